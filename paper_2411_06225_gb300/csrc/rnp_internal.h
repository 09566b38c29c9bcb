// rnp_internal.h -- shared declarations of librnp's kernels and launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rnp.h"

namespace rnp {

// Number of kernels this library has launched (all contexts, all threads).
long long launches_total();
void count_launches(long long n);

// Message returned by rnp_last_error(NULL) (calls without a context).
void set_global_error(const char* msg);

// Kernel-level PDE ids: the heat operator is split by dimension so that the
// stencil's dimensionality is a compile-time constant.
enum KPde {
  KP_BURGERS = 0, KP_ADVECT = 1, KP_HEAT1 = 2, KP_HEAT2 = 3, KP_HEAT3 = 4,
  KP_DIFFREACT = 5, KP_BRUSS2 = 6, KP_BRUSS3 = 7, KP_SWE = 8, KP_COUNT = 9
};

// Time integrators: forward Euler (G), classic RK4 (F, or G), and the
// eleven-stage eighth-order RK8 of Cooper & Verner (F, FP64 only).
enum Scheme { SCHEME_EULER = 0, SCHEME_RK4 = 1, SCHEME_RK8 = 2 };

// Geometry of one state vector.
struct Geom {
  int kp;          // KPde
  int nx, ny, nz;
  int ncomp;
  int dims;
  long long n;     // cells per component
  long long d;     // ncomp * n
  int outer;       // extent of the axis split across a cluster (x/y/z for 1/2/3D)
  long long plane; // cells per outer index
  int bc;          // rnp_bc: 0 periodic, 1 no-flux walls (wall neighbour = the cell)
  bool iso;        // equal grid spacing on every axis the operator has
};

// PDE constants, precomputed on the host in FP64 exactly as the plain
// serial formulas use them (coefficients, 1/h^2, 1/(2h), 1/h), and the
// shallow-water bottom term: bath[i] = g (b_E - b_W) (1 / (2 hx)) and
// bath[n + i] = g (b_N - b_S) (1 / (2 hy)) per cell (device, FP64; bath32
// the same rounded to FP32), or null for a flat bottom.
struct Coef {
  double k[12];
  const double* bath;
  const float* bath32;
};

// Work-item description of a stencil launch: item w reads the state at
// in + off(src, w) and writes out + off(dst, w) (and out2 + off(dst2, w)
// when out2 != nullptr), where off(x, w) = x_off[w] if the table is given,
// else x_base + w * x_stride.  gate (optional) skips items with
// gate[w] == 0.
struct Items {
  const long long* src_off; long long src_base, src_stride;
  const long long* dst_off; long long dst_base, dst_stride;
  const long long* dst2_off; long long dst2_base, dst2_stride;
  const int* gate;
  int n;
};

// Row offsets of the feature / scaling kernels: table or affine.
struct Rows {
  const long long* off; long long base, stride;
};

#ifdef __CUDACC__
__host__ __device__ __forceinline__ long long item_off(const long long* tab,
                                                       long long base,
                                                       long long stride, int w) {
  return tab ? tab[w] : base + (long long)w * stride;
}
#endif

struct StencilCfg {
  int cluster;   // CTAs per slice
  int threads;   // threads per CTA
  int R;         // cells per thread (FP64 kernel)
  int px, rs;    // x-points and outer rows per thread (mixed kernel)
  int tm;        // mixed kernel with the state in tensor memory (wide kernel)
};

Geom make_geom(const rnp_problem& p);
Coef make_coef(const rnp_problem& p, const Geom& g);

// Choose a fused-stencil configuration.  latency = true favours many SMs per
// item (sequential sweep), false favours throughput (many items).  rk8: the
// configuration runs the FP64 RK8 kernel (fp32 must be false).
bool pick_stencil(const Geom& g, bool fp32, int nitems, bool latency,
                  int want_cluster, int want_threads, StencilCfg* out,
                  char* why, int why_len, bool rk8 = false);

// Every launchable configuration (FP32 tiles when fp32, else the FP64
// kernel), at most maxn, for the autotuner.
int list_stencil_cfgs(const Geom& g, bool fp32, int nitems, StencilCfg* out, int maxn,
                      bool rk8 = false);

// Fused stencil: every item advances `steps` Euler/RK4/RK8 steps of size dt
// inside one launch, the slice resident in the cluster's shared memory.
cudaError_t launch_stencil_fused(const Geom& g, const Coef& c, bool fp32,
                                 int scheme, int steps, double dt,
                                 const double* in, double* out, double* out2,
                                 const Items& it, const StencilCfg& cfg,
                                 cudaStream_t st, int* err = nullptr);

// Plain stencil: one launch per Runge-Kutta stage over global memory.
// work must hold plain_work_doubles(scheme, n_items * d) doubles.
long long plain_work_doubles(int scheme, long long items_d);
cudaError_t launch_stencil_plain(const Geom& g, const Coef& c, int scheme,
                                 int steps, double dt, const double* in,
                                 double* out, double* out2, const Items& it,
                                 double* work, cudaStream_t st);

// ---------------- RandNet kernels (randnet.cu) -----------------------------

cudaError_t launch_weights(uint64_t seed, int M, long long d, double* A,
                           double* zeta, float* A32, uint16_t* Abf16,
                           float* zeta32, cudaStream_t st);

// Per-member, per-species min/max over `nstates` consecutive states starting
// at U + b * bstride, then c = (max + min) / 2, r = (max - min) / 2 (r = 1
// when 0), written to c[b*3 + q], r[b*3 + q].  none = identity scaling.
// nonfinite (optional) is set when a scanned value is NaN or Inf; mask
// (optional) restricts the update to members b with mask[b] != 0.
cudaError_t launch_scaling(const Geom& g, const double* U, long long bstride,
                           int nstates, int B, bool none, double* c, double* r,
                           double* work, int* nonfinite, const int* mask,
                           cudaStream_t st);

// Rows r = 0..R-1: S[dst(r)..] = (U[src(r)..] - c[b]) / r[b] with
// b = row_b[r] (or r / row_b_div); S (FP64) and S32 (rounded to FP32) are
// each optional.
cudaError_t launch_scale_rows(const Geom& g, const double* U, Rows src,
                              const int* row_b, int row_b_div,
                              const double* c, const double* r, double* S,
                              float* S32, Rows dst, int R, const int* gate,
                              cudaStream_t st);

// Random features phi = ReLU(A s + zeta) of R scaled rows S + s_off[r],
// written to phi + phi_off[r] (FP64).  part must hold R * M * nchunks.
cudaError_t launch_features64(const double* A, const double* zeta, int M,
                              long long d, const double* S, Rows s_rows, int R,
                              double* phi, Rows phi_rows, double* part,
                              const int* gate, cudaStream_t st);
cudaError_t launch_features32(const float* A, const double* zeta, int M,
                              long long d, const float* S, Rows s_rows, int R,
                              double* phi, Rows phi_rows, double* part,
                              const int* gate, cudaStream_t st);
int features_chunks(long long d);

// The same map with BF16 operands and FP32 accumulation: many rows on the
// tensor cores (tcgen05, split-K; M <= 128, part holds
// features_tc_part_floats(R, d) floats, err is set if a bounded wait gave
// up) or single rows on CUDA cores (part as for launch_features64).
size_t features_tc_part_floats(int R, long long d);
cudaError_t launch_features_tc(const __nv_bfloat16* A, const double* zeta, int M,
                               long long d, const float* S, Rows s_rows, int R,
                               double* phi, Rows phi_rows, float* part, int* err,
                               cudaStream_t st);
cudaError_t launch_features_bf16(const __nv_bfloat16* A, const double* zeta, int M,
                                 long long d, const float* S, Rows s_rows, int R,
                                 double* phi, Rows phi_rows, double* part,
                                 const int* gate, cudaStream_t st);

// Squared distances of the scaled query q[b] to the P[b] stored rows of
// member b (dataset rows at S + b * cap * d), partial over d-chunks.
cudaError_t launch_nn_partial(const double* q, const double* S, long long cap,
                              long long d, const int* P, int Pmax, int B,
                              double* part, const int* gate, cudaStream_t st);
cudaError_t launch_nn_partial32(const float* q, const float* S, long long cap,
                                long long d, const int* P, int Pmax, int B,
                                float* part, const int* gate, cudaStream_t st);
int nn_chunks(long long d);

// Both partial sums of a RandNet query in one launch: the feature partials
// of the B query rows q + b * d (fpart, as launch_features64's part) and the
// distance partials to the stored rows (npart, as launch_nn_partial's part).
cudaError_t launch_query64(const double* A, int M, long long d, const double* q, int B,
                           double* fpart, const double* S, long long cap, const int* P,
                           int Pmax, double* npart, const int* gate, cudaStream_t st);
cudaError_t launch_query32(const float* A, int M, long long d, const float* q, int B,
                           float* fpart, const float* S, long long cap, const int* P,
                           int Pmax, float* npart, const int* gate, cudaStream_t st);

// Per member: (if fpart != null) finish the query features phi_q from their
// chunk partials into phiq[b]; finish distances (d: the state dimension; the
// partials are chunked as the partial kernels chunk a member with P stored
// rows), select the m nearest (ties
// -> lower index), build the dual ridge system from the stored features and
// phi_q, solve by Cholesky (lambda x10 on a non-positive pivot, at most 4
// times) and write alpha[b*RNP_MAX_M + l], idx[b*RNP_MAX_M + l], meff[b].
cudaError_t launch_topm_ridge(const double* part, long long d, const double* Phi,
                              long long cap, int M, double* phiq,
                              long long phiq_bstride, const double* fpart, int fnch,
                              const double* zeta, const int* P, int Pmax,
                              int B, int m, double lambda,
                              double* dist, double* alpha, int* idx, int* meff,
                              int* esc_count, int* fail, const int* gate,
                              cudaStream_t st);
// The same with FP32 chunk partials (from launch_query32 / launch_nn_partial32).
cudaError_t launch_topm_ridge32(const float* part, long long d, const double* Phi,
                                long long cap, int M, double* phiq,
                                long long phiq_bstride, const float* fpart, int fnch,
                                const double* zeta, const int* P, int Pmax,
                                int B, int m, double lambda,
                                double* dist, double* alpha, int* idx, int* meff,
                                int* esc_count, int* fail, const int* gate,
                                cudaStream_t st);

// Optional second output of the update: the new state scaled per species,
// (out - c[b][q]) / r[b][q] (n cells per species), written to q64[b] and/or
// q32[b] (member stride d) -- the scaled query of the next sweep step.
struct QueryOut {
  const double* c;
  const double* r;
  long long n;
  double* q64;
  float* q32;
};

// out[b] = g[b] + sum_l alpha_l Y[b][idx_l]  (g may be null: out = sum).
// If err != null: err[b] = max |out_new - out_old| over the state (the old
// value is read before it is overwritten), and nonfinite is set on NaN/Inf.
cudaError_t launch_update(const double* g, long long g_bstride,
                          const double* Y, long long cap, long long d,
                          const double* alpha, const int* idx, const int* meff,
                          double* out, long long out_bstride,
                          unsigned long long* err, long long err_bstride,
                          int* nonfinite, int B, const int* gate,
                          cudaStream_t st, QueryOut qo = QueryOut{});

// Parareal (Eq. 4) update: out[b] = g[b] + Yv[b]; err / nonfinite as above.
cudaError_t launch_update_para(const double* g, long long g_bstride,
                               const double* Yv, long long yv_bstride,
                               long long d, double* out, long long out_bstride,
                               unsigned long long* err, long long err_bstride,
                               int* nonfinite, int B, const int* gate,
                               cudaStream_t st);

// Dataset append for item w = (b, j, p): y = F[b][j] - G[b][j] is written to
// Yv[b][j] and (randnet) to Yds[b][p]; the scaled start U[b][j] to Sds[b][p].
struct AppendItems {
  const int* b;
  const int* j;
  const int* p;
  int n;
};
cudaError_t launch_append(const Geom& g, const double* U, long long u_bstride,
                          const double* Fv, const double* Gc, long long n_bstride,
                          double* Yv, double* Sds, float* S32, double* Yds,
                          long long cap, const double* c, const double* r,
                          const AppendItems& it, bool randnet, cudaStream_t st);

// Copy feature rows: dst[b][p] = src[b][j] for each append item.
cudaError_t launch_copy_phi(const double* src, long long src_bstride,
                            double* dst, long long cap, int M,
                            const AppendItems& it, cudaStream_t st);

// Element-wise copy of `rows` rows of length d with per-row offsets.
cudaError_t launch_copy_rows(const double* src, const long long* src_off,
                             double* dst, const long long* dst_off, long long d,
                             int rows, cudaStream_t st);

// Up to RNP_MAX_BATCH segments [off, off + len) (in doubles) copied from src
// to dst at the same offsets; dst may be the device address of pinned host
// memory.
struct Segments {
  long long off[RNP_MAX_BATCH];
  long long len[RNP_MAX_BATCH];
  int n;
};
cudaError_t launch_copy_segments(const double* src, double* dst, const Segments& sg,
                                 cudaStream_t st);

}  // namespace rnp
