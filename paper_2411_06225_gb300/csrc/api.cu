// api.cu -- the C ABI of librnp (include/rnp.h) and the host orchestration
// of Alg. 1: the k = 0 coarse sweep, then per iteration the parallel fine
// step, the dataset append of Eq. 6, the exact leftmost slice, the
// sequential predictor-corrector sweep of Eq. 3 and the stopping rule of
// Eq. 5.  All arithmetic runs in the kernels of stencil.cu and randnet.cu;
// the host only builds work lists and reads back one norm vector per
// iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rnp_internal.h"

using namespace rnp;

struct rnp_ctx {
  rnp_problem p;
  Geom g;
  Coef coef;
  int dev = 0;
  cudaStream_t ust = nullptr;  // the caller's stream
  cudaStream_t st = nullptr;   // the context's own stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int B = 1, N = 1, M = 1, m = 1;
  long long d = 0, cap = 0;
  bool fp32 = false, plain = false, randnet = true;
  StencilCfg cfgF{}, cfgG{};
  bool tunedF = false, tunedG = false;
  double dtF = 0, dtG = 0;
  int schemeG = SCHEME_EULER;
  int schemeF = SCHEME_RK4;

  // device state
  double *U = nullptr, *Fv = nullptr, *Gc = nullptr, *Yv = nullptr, *gbuf = nullptr,
         *qbuf = nullptr, *phic = nullptr, *phiq = nullptr;
  double *Sds = nullptr, *Yds = nullptr, *Phi = nullptr;
  double *A = nullptr, *zeta = nullptr;
  float *A32 = nullptr, *S32 = nullptr, *q32 = nullptr;  // mixed precision copies
  __nv_bfloat16* Abf = nullptr;   // BF16 weights (MIXED_BF16)
  float* tc_part = nullptr;       // split-K partials of the tensor-core feature GEMM
  bool bf16 = false;
  double *sc = nullptr, *sr = nullptr, *scale_work = nullptr;
  double *feat_part = nullptr, *nn_part = nullptr, *dist = nullptr, *alpha = nullptr;
  int *idx = nullptr, *meff = nullptr, *flags = nullptr;  // flags: esc, fail, nonfinite
  int* dP = nullptr;
  unsigned long long* err = nullptr;
  double* plain_work = nullptr;
  double* bath = nullptr;         // shallow-water bottom term [2][n] (or null)
  float* bath32 = nullptr;
  long long* d_items = nullptr;   // src, dst, soff, phioff tables (4 * itemcap)
  int* d_app = nullptr;           // b, j, p (3 * itemcap)
  int* d_gate = nullptr;          // (N + 1) * B
  long long* d_qsrc = nullptr;    // [B] first sweep query of each member (offset in U)
  int* d_qgate = nullptr;         // [B] member has a sweep this iteration
  int itemcap = 0;
  int feat_rows_cap = 0;

  // host mirrors
  long long* h_items = nullptr;   // pinned
  int* h_app = nullptr;           // pinned
  int* h_gate = nullptr;          // pinned
  long long* h_qsrc = nullptr;    // pinned [B]
  int* h_qgate = nullptr;         // pinned [B]
  unsigned long long* h_err = nullptr;  // pinned (B * (N+1))
  int* h_flags = nullptr;         // pinned (4)
  std::vector<int> P;             // pairs per member
  // per-member iteration state (Alg. 1 split per iteration)
  std::vector<int> mL, mK, mstate;
  int* d_mask = nullptr;          // device [B] member mask
  int* h_mask = nullptr;          // pinned [B]
  rnp_stats run{};                // statistics accumulated since the last reset
  bool weights_ready = false, scaling_ready = false;
  double h_c[RNP_MAX_BATCH * 3], h_r[RNP_MAX_BATCH * 3];

  cudaEvent_t ev[6] = {};
  // side stream for the coarse step of the sweep, fork/join events, and the
  // CUDA graphs of the solve's sweep keyed by its first index
  cudaStream_t st2 = nullptr;
  cudaEvent_t evf = nullptr, evj = nullptr;
  // copy stream and its event: a solve into host memory sends each member's
  // converged states out while the next iteration computes
  cudaStream_t st3 = nullptr;
  cudaEvent_t evc = nullptr;
  std::vector<cudaGraphExec_t> sweep_graph;
  std::vector<long long> sweep_graph_launches;
  std::string msg;
};

static thread_local std::string g_create_error;

void rnp::set_global_error(const char* msg) { g_create_error = msg; }

namespace {

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Orders a call's work after what the caller enqueued on its stream, and
// the caller's later work after the call's: the context computes on its own
// stream (which, unlike the legacy default stream, can be captured into a
// graph) joined to the caller's stream by events.
struct StreamJoin {
  rnp_ctx* c;
  explicit StreamJoin(rnp_ctx* ctx) : c(ctx) {
    cudaEventRecord(c->ev_in, c->ust);
    cudaStreamWaitEvent(c->st, c->ev_in, 0);
  }
  ~StreamJoin() {
    cudaEventRecord(c->ev_out, c->st);
    cudaStreamWaitEvent(c->ust, c->ev_out, 0);
  }
};

rnp_status fail(rnp_ctx* c, rnp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->msg = buf; else g_create_error = buf;
  return s;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(c, RNP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                             \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  if (count == 0) { *p = nullptr; return cudaSuccess; }
  return cudaMalloc((void**)p, count * sizeof(T));
}

const char* validate(const rnp_problem* p) {
  if (!p) return "problem is NULL";
  if (p->pde < RNP_BURGERS1D || p->pde > RNP_ADVECT1D) return "unknown pde";
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "grid sizes must be >= 1";
  if ((p->pde == RNP_BURGERS1D || p->pde == RNP_ADVECT1D) && (p->ny != 1 || p->nz != 1))
    return "1D problems need ny = nz = 1";
  if ((p->pde == RNP_DIFFREACT2D || p->pde == RNP_BRUSS2D || p->pde == RNP_SWE2D) && p->nz != 1)
    return "2D problems need nz = 1";
  if (p->pde == RNP_HEAT && p->nz > 1 && p->ny < 2) return "3D heat needs ny > 1";
  if (p->nx < 3 || (p->ny > 1 && p->ny < 3) || (p->nz > 1 && p->nz < 3))
    return "every used axis needs >= 3 points";
  if (!(p->lx > 0) || !(p->ly > 0) || !(p->lz > 0)) return "domain lengths must be > 0";
  if (!(p->tN > p->t0)) return "tN must exceed t0";
  if (p->N < 1) return "N must be >= 1";
  if (p->nF < 1 || p->nG < 1) return "nF and nG must be >= 1";
  if (p->M < 1 || p->M > 4096) return "M must be in [1, 4096]";
  if (p->m < 1 || p->m > RNP_MAX_M) return "m must be in [1, 32]";
  if (!(p->lambda >= 0)) return "lambda must be >= 0";
  if (!(p->tol >= 0)) return "tol must be >= 0";
  if (p->max_iters < 1) return "max_iters must be >= 1";
  if (p->batch < 1 || p->batch > RNP_MAX_BATCH) return "batch must be in [1, 64]";
  if (p->corr != RNP_CORR_RANDNET && p->corr != RNP_CORR_PARAREAL) return "unknown corr";
  if (p->bc != RNP_BC_PERIODIC && p->bc != RNP_BC_NEUMANN) return "unknown bc";
  if (p->bathymetry && p->pde != RNP_SWE2D) return "bathymetry applies to shallow water only";
  if (p->scale_mode != RNP_SCALE_MINMAX && p->scale_mode != RNP_SCALE_NONE)
    return "unknown scale_mode";
  if (p->gscheme != RNP_G_EULER && p->gscheme != RNP_G_RK4) return "unknown gscheme";
  if (p->fscheme != RNP_F_RK4 && p->fscheme != RNP_F_RK8) return "unknown fscheme";
  if (p->fscheme == RNP_F_RK8 && p->precision != RNP_FP64)
    return "the RK8 fine solver runs in FP64 only";
  if (p->precision != RNP_FP64 && p->precision != RNP_MIXED && p->precision != RNP_MIXED_BF16)
    return "unknown precision";
  if (p->exec != RNP_EXEC_FUSED && p->exec != RNP_EXEC_PLAIN) return "unknown exec";
  if (p->cluster < 0 || p->cluster > 16 || p->threads < 0 || p->threads > 800 ||
      p->threads % 32)
    return "cluster must be in [0,16] and threads a multiple of 32 in [0,800]";
  if (p->max_pairs < 0) return "max_pairs must be >= 0";
  return nullptr;
}

// Shallow water over a bottom b (Sec. 5.3): the per-cell factors of the
// term -g h grad b, g (b_E - b_W) (1 / (2 hx)) and g (b_N - b_S) (1 / (2 hy))
// (across a wall the bottom's neighbour is the cell itself), in FP64 and
// rounded to FP32, on the device; the stencils read them through Coef.
bool upload_bathymetry(rnp_ctx* c, const rnp_problem& p) {
  const int nx = p.nx, ny = p.ny;
  const long long n = (long long)nx * ny;
  const double hx = p.lx / nx, hy = p.ly / ny, g = p.param[0];
  const bool wall = p.bc == RNP_BC_NEUMANN;
  auto nb = [&](int i, int dir, int len) {
    const int j = i + dir;
    if (j >= 0 && j < len) return j;
    if (wall) return i;
    return j < 0 ? j + len : j - len;
  };
  const double* b = p.bathymetry;
  std::vector<double> hb(2 * n);
  std::vector<float> hf(2 * n);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const long long i = (long long)y * nx + x;
      hb[i] = g * ((b[(long long)y * nx + nb(x, 1, nx)] - b[(long long)y * nx + nb(x, -1, nx)]) *
                   (0.5 / hx));
      hb[n + i] = g * ((b[(long long)nb(y, 1, ny) * nx + x] - b[(long long)nb(y, -1, ny) * nx + x]) *
                       (0.5 / hy));
    }
  for (long long i = 0; i < 2 * n; ++i) hf[i] = (float)hb[i];
  if (dalloc(&c->bath, (size_t)(2 * n)) != cudaSuccess ||
      dalloc(&c->bath32, (size_t)(2 * n)) != cudaSuccess)
    return false;
  if (cudaMemcpy(c->bath, hb.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(c->bath32, hf.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return false;
  c->coef.bath = c->bath;
  c->coef.bath32 = c->bath32;
  return true;
}

void destroy_buffers(rnp_ctx* c) {
  void* bufs[] = {c->U, c->Fv, c->Gc, c->Yv, c->gbuf, c->qbuf, c->phic, c->phiq, c->Sds,
                  c->Yds, c->Phi, c->A, c->zeta, c->sc, c->sr, c->scale_work, c->feat_part,
                  c->nn_part, c->dist, c->alpha, c->idx, c->meff, c->flags, c->dP, c->err,
                  c->plain_work, c->d_items, c->d_app, c->d_gate, c->A32, c->S32, c->q32,
                  c->d_mask, c->Abf, c->tc_part, c->d_qsrc, c->d_qgate, c->bath, c->bath32};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->h_items) cudaFreeHost(c->h_items);
  if (c->h_app) cudaFreeHost(c->h_app);
  if (c->h_gate) cudaFreeHost(c->h_gate);
  if (c->h_qsrc) cudaFreeHost(c->h_qsrc);
  if (c->h_qgate) cudaFreeHost(c->h_qgate);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->h_mask) cudaFreeHost(c->h_mask);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->evf) cudaEventDestroy(c->evf);
  if (c->evj) cudaEventDestroy(c->evj);
  for (auto& g : c->sweep_graph)
    if (g) cudaGraphExecDestroy(g);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->evc) cudaEventDestroy(c->evc);
  if (c->st3) cudaStreamDestroy(c->st3);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->st) cudaStreamDestroy(c->st);
}

// ---------------------------------------------------------------------------
// Building blocks
// ---------------------------------------------------------------------------
rnp_status run_stencil(rnp_ctx* c, bool fine, const double* in, double* out, double* out2,
                       const Items& it, cudaStream_t stream = nullptr) {
  cudaStream_t sx = stream ? stream : c->st;
  const int scheme = fine ? c->schemeF : c->schemeG;
  const int steps = fine ? c->p.nF : c->p.nG;
  const double dt = fine ? c->dtF : c->dtG;
  cudaError_t e;
  if (c->plain)
    e = launch_stencil_plain(c->g, c->coef, scheme, steps, dt, in, out, out2, it,
                             c->plain_work, sx);
  else
    e = launch_stencil_fused(c->g, c->coef, c->fp32, scheme, steps, dt, in, out, out2, it,
                             fine ? c->cfgF : c->cfgG, sx, c->flags + 3);
  if (e != cudaSuccess)
    return fail(c, RNP_ECUDA, "stencil launch failed: %s", cudaGetErrorString(e));
  return RNP_OK;
}

Items affine(int n, long long sb, long long ss, long long db, long long ds, const int* gate) {
  Items it{};
  it.src_off = nullptr; it.src_base = sb; it.src_stride = ss;
  it.dst_off = nullptr; it.dst_base = db; it.dst_stride = ds;
  it.dst2_off = nullptr; it.dst2_base = 0; it.dst2_stride = 0;
  it.gate = gate;
  it.n = n;
  return it;
}

rnp_status ensure_weights(rnp_ctx* c) {
  if (c->weights_ready) return RNP_OK;
  CK(launch_weights(c->p.seed, c->M, c->d, c->A, c->zeta, c->A32,
                    reinterpret_cast<uint16_t*>(c->Abf), nullptr, c->st));
  c->weights_ready = true;
  return RNP_OK;
}

rnp_status upload_P(rnp_ctx* c) {
  // small synchronous copy from a pinned staging word block
  for (int b = 0; b < c->B; ++b) c->h_flags[4 + b] = c->P[b];
  CK(cudaMemcpyAsync(c->dP, c->h_flags + 4, sizeof(int) * c->B, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return RNP_OK;
}

int Pmax(const rnp_ctx* c) {
  int x = 0;
  for (int b = 0; b < c->B; ++b) x = std::max(x, c->P[b]);
  return x;
}

// RandNet prediction for one query per member: the scaled query is written to
// qbuf, its features to phi_dst (member stride phi_bstride); alpha / idx /
// meff are left on the device for the update kernel.
rnp_status predict_core(rnp_ctx* c, const double* q, long long q_base, long long q_bstride,
                        double* phi_dst, long long phi_base, long long phi_bstride,
                        const int* gate, bool q_ready = false) {
  Rows src{nullptr, q_base, q_bstride};
  Rows qrows{nullptr, 0, c->d};
  Rows prow{nullptr, phi_base, phi_bstride};
  // the neighbour grid is sized for up to 256 rows (rows are strided), so a
  // captured sweep graph serves every later dataset size
  const int pm = Pmax(c) > 0 ? (int)std::max<long long>(Pmax(c), std::min<long long>(c->cap, 256))
                             : 0;
  // the query's feature partials are finished inside the ridge kernel
  // (except on the BF16 path); FP32 queries leave FP32 partials
  float* fpart32 = reinterpret_cast<float*>(c->feat_part);
  float* npart32 = reinterpret_cast<float*>(c->nn_part);
  if (c->fp32) {
    // mixed: FP32 query, FP32 features and FP32 distance screening
    if (!q_ready)
      CK(launch_scale_rows(c->g, q, src, nullptr, 1, c->sc, c->sr, nullptr, c->q32, qrows, c->B,
                           gate, c->st));
    if (c->bf16) {
      CK(launch_features_bf16(c->Abf, c->zeta, c->M, c->d, c->q32, qrows, c->B, phi_dst, prow,
                              c->feat_part, gate, c->st));
      CK(launch_nn_partial32(c->q32, c->S32, c->cap, c->d, c->dP, pm, c->B, npart32, gate,
                             c->st));
      fpart32 = nullptr;
    } else {
      CK(launch_query32(c->A32, c->M, c->d, c->q32, c->B, fpart32, c->S32, c->cap, c->dP, pm,
                        npart32, gate, c->st));
    }
    CK(launch_topm_ridge32(npart32, c->d, c->Phi, c->cap, c->M, phi_dst + phi_base,
                           phi_bstride, fpart32, features_chunks(c->d), c->zeta, c->dP, pm, c->B,
                           c->m, c->p.lambda, c->dist, c->alpha, c->idx, c->meff, c->flags + 0,
                           c->flags + 1, gate, c->st));
  } else {
    if (!q_ready)
      CK(launch_scale_rows(c->g, q, src, nullptr, 1, c->sc, c->sr, c->qbuf, nullptr, qrows, c->B,
                           gate, c->st));
    CK(launch_query64(c->A, c->M, c->d, c->qbuf, c->B, c->feat_part, c->Sds, c->cap, c->dP, pm,
                      c->nn_part, gate, c->st));
    CK(launch_topm_ridge(c->nn_part, c->d, c->Phi, c->cap, c->M, phi_dst + phi_base,
                         phi_bstride, c->feat_part, features_chunks(c->d), c->zeta, c->dP, pm,
                         c->B, c->m, c->p.lambda, c->dist, c->alpha, c->idx, c->meff,
                         c->flags + 0, c->flags + 1, gate, c->st));
  }
  return RNP_OK;
}

// One predictor-corrector step of Eq. 3 for every member, U[b][i] from
// U[b][i-1] (U with member stride ubs).  G runs on the side stream while the
// RandNet query (features, neighbours, ridge) runs on the main stream; both
// read only U[b][i-1] and join before the update.  Gc (optional) receives
// G(U[b][i-1]); err/gate as in launch_update.
rnp_status sweep_step(rnp_ctx* c, double* U, long long ubs, int i, double* Gc,
                      unsigned long long* err, const int* gate) {
  const long long d = c->d, nb = (long long)c->N * d;
  rnp_status s;
  CK(cudaEventRecord(c->evf, c->st));
  CK(cudaStreamWaitEvent(c->st2, c->evf, 0));
  Items it = affine(c->B, (long long)(i - 1) * d, ubs, 0, d, gate);
  if (Gc) {
    it.dst2_base = (long long)(i - 1) * d;
    it.dst2_stride = nb;
  }
  if ((s = run_stencil(c, false, U, c->gbuf, Gc, it, c->st2))) return s;
  CK(cudaEventRecord(c->evj, c->st2));
  if (c->randnet) {
    // the scaled query U[b][i-1] is already in q32 / qbuf: scaled before the
    // sweep for its first step, by the previous step's update otherwise
    if (Gc) {
      // the solve caches the query's features as the next dataset row
      if ((s = predict_core(c, U, (long long)(i - 1) * d, ubs, c->phic, (long long)(i - 1) * c->M,
                            (long long)c->N * c->M, gate, true)))
        return s;
    } else if ((s = predict_core(c, U, (long long)(i - 1) * d, ubs, c->phiq, 0, c->M, gate,
                                 true))) {
      return s;
    }
    CK(cudaStreamWaitEvent(c->st, c->evj, 0));
    const QueryOut qo{c->sc, c->sr, c->g.n, c->fp32 ? nullptr : c->qbuf,
                      c->fp32 ? c->q32 : nullptr};
    CK(launch_update(c->gbuf, d, c->Yds, c->cap, d, c->alpha, c->idx, c->meff,
                     U + (long long)i * d, ubs, err ? err + i : nullptr, c->N + 1, c->flags + 2,
                     c->B, gate, c->st, qo));
  } else {
    CK(cudaStreamWaitEvent(c->st, c->evj, 0));
    CK(launch_update_para(c->gbuf, d, c->Yv + (long long)(i - 1) * d, nb, d,
                          U + (long long)i * d, ubs, err ? err + i : nullptr, c->N + 1,
                          c->flags + 2, c->B, gate, c->st));
  }
  return RNP_OK;
}

// The solve's sweep i = i0 .. N.  In the fused path the whole range
// i = 2 .. N is captured once per context as a CUDA graph (every pointer is
// fixed per context; the gate table and the dataset size are read from
// device memory): steps below a member's L + 2 are gated off on the device,
// so one graph serves every iteration and every mix of members.  Steps
// below min(L) + 2 cost one empty launch per kernel.
rnp_status solve_sweep(rnp_ctx* c, int i0) {
  const long long sb = (long long)(c->N + 1) * c->d;
  rnp_status s;
  if (c->plain) {
    for (int i = i0; i <= c->N; ++i)
      if ((s = sweep_step(c, c->U, sb, i, c->Gc, c->err, c->d_gate + (long long)i * c->B)))
        return s;
    return RNP_OK;
  }
  i0 = 2;
  if (!c->sweep_graph[i0]) {
    const long long before = launches_total();
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    for (int i = i0; i <= c->N; ++i) {
      s = sweep_step(c, c->U, sb, i, c->Gc, c->err, c->d_gate + (long long)i * c->B);
      if (s) {
        cudaStreamEndCapture(c->st, &graph);
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
    }
    CK(cudaStreamEndCapture(c->st, &graph));
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
      return fail(c, RNP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    c->sweep_graph[i0] = exec;
    c->sweep_graph_launches[i0] = launches_total() - before;
    count_launches(-c->sweep_graph_launches[i0]);  // captured, not launched
  }
  CK(cudaGraphLaunch(c->sweep_graph[i0], c->st));
  count_launches(c->sweep_graph_launches[i0]);
  return RNP_OK;
}

// Features of R dataset rows (scaled rows at S64/S32 + s_rows, written to
// phi + phi_rows) in the context's precision: FP64, FP32, or BF16 operands on
// the tensor cores.
rnp_status batch_features(rnp_ctx* c, const double* S64, const float* S32, Rows s_rows, int R,
                          double* phi, Rows phi_rows) {
  if (R <= 0) return RNP_OK;
  if (c->bf16 && c->M <= 128)
    CK(launch_features_tc(c->Abf, c->zeta, c->M, c->d, S32, s_rows, R, phi, phi_rows,
                          c->tc_part, c->flags + 3, c->st));
  else if (c->bf16)
    CK(launch_features_bf16(c->Abf, c->zeta, c->M, c->d, S32, s_rows, R, phi, phi_rows,
                            c->feat_part, nullptr, c->st));
  else if (c->fp32)
    CK(launch_features32(c->A32, c->zeta, c->M, c->d, S32, s_rows, R, phi, phi_rows,
                         c->feat_part, nullptr, c->st));
  else
    CK(launch_features64(c->A, c->zeta, c->M, c->d, S64, s_rows, R, phi, phi_rows,
                         c->feat_part, nullptr, c->st));
  return RNP_OK;
}

static const char* const kTimeoutMsg =
    "a bounded device wait timed out (tensor-core feature GEMM or stencil halo exchange)";

rnp_status read_flags(rnp_ctx* c, int* esc, int* failf, int* nonfinite) {
  CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_flags[3]) return fail(c, RNP_ETIMEOUT, kTimeoutMsg);
  *esc = c->h_flags[0];
  *failf = c->h_flags[1];
  *nonfinite = c->h_flags[2];
  return RNP_OK;
}

// Times every launchable stencil tiling for the fine step (all B N slices)
// and the coarse step (one item per member) on the context's own buffers,
// a few dozen steps each, best of four after one untimed launch, and keeps
// the fastest.  The cost of a step does not depend on the state's values.
rnp_status autotune_stencils(rnp_ctx* c) {
  const int B = c->B, N = c->N;
  const long long d = c->d, sb = (long long)(N + 1) * d;
  CK(cudaMemsetAsync(c->U, 0, sizeof(double) * B * sb, c->st));
  CK(cudaMemsetAsync(c->Fv, 0, sizeof(double) * B * N * d, c->st));
  for (int which = 0; which < 2; ++which) {
    const bool fine = which == 0;
    const int nitems = fine ? B * N : B;
    StencilCfg cands[64];
    const int n = list_stencil_cfgs(c->g, c->fp32, nitems, cands, 64,
                                    fine && c->schemeF == SCHEME_RK8);
    if (n <= 1) continue;
    // long enough (about half a millisecond for a fine step) that launch and
    // cluster-scheduling noise do not decide the ranking
    const int steps = std::min(fine ? c->p.nF : c->p.nG, fine ? 64 : 16);
    Items it = affine(nitems, 0, d, 0, d, nullptr);
    float best = 1e30f;
    int besti = -1;
    for (int k = 0; k < n; ++k) {
      float tmin = 1e30f;
      for (int rep = 0; rep < 5; ++rep) {
        CK(cudaEventRecord(c->ev[4], c->st));
        CK(launch_stencil_fused(c->g, c->coef, c->fp32, fine ? c->schemeF : c->schemeG, steps,
                                fine ? c->dtF : c->dtG, c->U, c->Fv, nullptr, it, cands[k],
                                c->st, c->flags + 3));
        CK(cudaEventRecord(c->ev[5], c->st));
        CK(cudaEventSynchronize(c->ev[5]));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
        if (rep > 0 && ms < tmin) tmin = ms;
      }
      if (tmin < best) { best = tmin; besti = k; }
    }
    if (besti >= 0) {
      if (fine) { c->cfgF = cands[besti]; c->tunedF = true; }
      else { c->cfgG = cands[besti]; c->tunedG = true; }
    }
  }
  return RNP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

long long rnp_dim(const rnp_problem* p) {
  if (!p) return 0;
  const int nc = (p->pde == RNP_SWE2D) ? 3
                 : (p->pde == RNP_DIFFREACT2D || p->pde == RNP_BRUSS2D || p->pde == RNP_BRUSS3D)
                     ? 2
                     : 1;
  return (long long)nc * p->nx * p->ny * p->nz;
}

const char* rnp_last_error(const rnp_ctx* ctx) {
  return ctx ? ctx->msg.c_str() : g_create_error.c_str();
}

rnp_status rnp_create(const rnp_problem* prob, void* cuda_stream, rnp_ctx** out) {
  rnp_ctx* c = nullptr;
  if (!out) return fail(nullptr, RNP_EINVAL, "out is NULL");
  *out = nullptr;
  if (const char* why = validate(prob)) return fail(nullptr, RNP_EINVAL, "%s", why);
  c = new (std::nothrow) rnp_ctx();
  if (!c) return fail(nullptr, RNP_ENOMEM, "host allocation failed");
  c->p = *prob;
  if (cudaGetDevice(&c->dev) != cudaSuccess) {
    delete c;
    return fail(nullptr, RNP_ECUDA, "no CUDA device");
  }
  c->ust = (cudaStream_t)cuda_stream;
  c->g = make_geom(*prob);
  c->coef = make_coef(*prob, c->g);
  c->B = prob->batch; c->N = prob->N; c->M = prob->M; c->m = prob->m;
  c->d = c->g.d;
  c->fp32 = prob->precision != RNP_FP64;
  c->bf16 = prob->precision == RNP_MIXED_BF16;
  c->plain = prob->exec == RNP_EXEC_PLAIN;
  c->randnet = prob->corr == RNP_CORR_RANDNET;
  c->schemeG = prob->gscheme == RNP_G_RK4 ? SCHEME_RK4 : SCHEME_EULER;
  c->schemeF = prob->fscheme == RNP_F_RK8 ? SCHEME_RK8 : SCHEME_RK4;
  const double dT = (prob->tN - prob->t0) / prob->N;
  c->dtF = dT / prob->nF;
  c->dtG = dT / prob->nG;
  const int Kmax = std::min(prob->max_iters, prob->N);
  long long cap = 0;
  for (int k = 1; k <= Kmax; ++k) cap += prob->N - k + 1;
  if (prob->max_pairs > 0) cap = prob->max_pairs;
  c->cap = cap;
  c->P.assign(c->B, 0);
  c->mL.assign(c->B, 0);
  c->mK.assign(c->B, 0);
  c->mstate.assign(c->B, RNP_MEMBER_FREE);
  const int B = c->B, N = c->N, M = c->M;
  const long long d = c->d;
  char why[256] = {0};
  rnp_ctx* cc = c;
  auto bail = [&](rnp_status s, const char* m) {
    g_create_error = m;
    destroy_buffers(cc);
    delete cc;
    return s;
  };
  if (!c->plain) {
    if (!pick_stencil(c->g, c->fp32, B * N, false, prob->cluster, prob->threads, &c->cfgF, why,
                      sizeof(why), c->schemeF == SCHEME_RK8))
      return bail(RNP_EINVAL, why);
    if (!pick_stencil(c->g, c->fp32, B, true, prob->cluster, prob->threads, &c->cfgG, why,
                      sizeof(why)))
      return bail(RNP_EINVAL, why);
  }
  c->itemcap = B * (N + 1);
  c->feat_rows_cap = std::max(B * N, B);
  const int nchF = features_chunks(d), nchN = nn_chunks(d);
  bool ok = true;
  ok &= dalloc(&c->U, (size_t)B * (N + 1) * d) == cudaSuccess;
  ok &= dalloc(&c->Fv, (size_t)B * N * d) == cudaSuccess;
  ok &= dalloc(&c->Gc, (size_t)B * N * d) == cudaSuccess;
  ok &= dalloc(&c->Yv, (size_t)B * N * d) == cudaSuccess;
  ok &= dalloc(&c->gbuf, (size_t)B * d) == cudaSuccess;
  ok &= dalloc(&c->qbuf, (size_t)B * d) == cudaSuccess;
  ok &= dalloc(&c->phic, (size_t)B * N * M) == cudaSuccess;
  ok &= dalloc(&c->phiq, (size_t)B * M) == cudaSuccess;
  if (c->bf16) {
    ok &= dalloc(&c->Abf, (size_t)M * d) == cudaSuccess;
    ok &= dalloc(&c->tc_part, features_tc_part_floats(c->feat_rows_cap, d)) == cudaSuccess;
  }
  if (c->fp32) {
    ok &= dalloc(&c->A32, (size_t)M * d) == cudaSuccess;
    ok &= dalloc(&c->S32, (size_t)B * cap * d) == cudaSuccess;
    ok &= dalloc(&c->q32, (size_t)B * d) == cudaSuccess;
  }
  {
    if (!c->fp32) ok &= dalloc(&c->Sds, (size_t)B * cap * d) == cudaSuccess;
    ok &= dalloc(&c->Yds, (size_t)B * cap * d) == cudaSuccess;
    ok &= dalloc(&c->Phi, (size_t)B * cap * M) == cudaSuccess;
    ok &= dalloc(&c->dist, (size_t)B * cap) == cudaSuccess;
    ok &= dalloc(&c->nn_part, (size_t)B * cap * nchN) == cudaSuccess;
  }
  ok &= dalloc(&c->A, (size_t)M * d) == cudaSuccess;
  ok &= dalloc(&c->zeta, (size_t)M) == cudaSuccess;
  ok &= dalloc(&c->sc, (size_t)B * 3) == cudaSuccess;
  ok &= dalloc(&c->sr, (size_t)B * 3) == cudaSuccess;
  ok &= dalloc(&c->scale_work, (size_t)B * 3 * 64 * 2) == cudaSuccess;
  ok &= dalloc(&c->feat_part, (size_t)c->feat_rows_cap * M * nchF) == cudaSuccess;
  ok &= dalloc(&c->alpha, (size_t)B * RNP_MAX_M) == cudaSuccess;
  ok &= dalloc(&c->idx, (size_t)B * RNP_MAX_M) == cudaSuccess;
  ok &= dalloc(&c->meff, (size_t)B) == cudaSuccess;
  ok &= dalloc(&c->flags, (size_t)4) == cudaSuccess;
  ok &= dalloc(&c->dP, (size_t)B) == cudaSuccess;
  ok &= dalloc(&c->err, (size_t)B * (N + 1)) == cudaSuccess;
  if (c->plain)
    ok &= dalloc(&c->plain_work, (size_t)plain_work_doubles(c->schemeF, (long long)B * N * d)) ==
          cudaSuccess;
  ok &= dalloc(&c->d_items, (size_t)4 * c->itemcap) == cudaSuccess;
  ok &= dalloc(&c->d_app, (size_t)3 * c->itemcap) == cudaSuccess;
  ok &= dalloc(&c->d_gate, (size_t)(N + 1) * B) == cudaSuccess;
  ok &= dalloc(&c->d_mask, (size_t)B) == cudaSuccess;
  ok &= dalloc(&c->d_qsrc, (size_t)B) == cudaSuccess;
  ok &= dalloc(&c->d_qgate, (size_t)B) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_qsrc, sizeof(long long) * B) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_qgate, sizeof(int) * B) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_mask, sizeof(int) * B) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_items, sizeof(long long) * 4 * c->itemcap) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_app, sizeof(int) * 3 * c->itemcap) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_gate, sizeof(int) * (N + 1) * B) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_err, sizeof(unsigned long long) * B * (N + 1)) == cudaSuccess;
  ok &= cudaMallocHost((void**)&c->h_flags, sizeof(int) * (4 + RNP_MAX_BATCH)) == cudaSuccess;
  for (auto& e : c->ev) ok &= cudaEventCreate(&e) == cudaSuccess;
  ok &= cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&c->evf, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&c->evj, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaStreamCreateWithFlags(&c->st3, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&c->evc, cudaEventDisableTiming) == cudaSuccess;
  c->sweep_graph.assign(N + 2, nullptr);
  c->sweep_graph_launches.assign(N + 2, 0);
  if (!ok) {
    cudaGetLastError();
    char m[256];
    snprintf(m, sizeof(m),
             "device allocation failed (dataset arena of %lld rows x %lld unknowns per member; "
             "lower max_iters or max_pairs)",
             cap, d);
    return bail(RNP_ENOMEM, m);
  }
  if (cudaMemsetAsync(c->dP, 0, sizeof(int) * B, c->st) != cudaSuccess ||
      cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    cudaGetLastError();
    return bail(RNP_ECUDA, "initialisation failed");
  }
  if (prob->bathymetry) {
    if (!upload_bathymetry(c, *prob)) {
      cudaGetLastError();
      return bail(RNP_ENOMEM, "bathymetry upload failed");
    }
  }
  for (int i = 0; i < B * 3; ++i) { c->h_c[i] = 0.0; c->h_r[i] = 1.0; }
  if (prob->autotune && !c->plain && prob->cluster == 0 && prob->threads == 0) {
    if (autotune_stencils(c) != RNP_OK) {
      std::string m = "autotune: " + c->msg;
      return bail(RNP_ECUDA, m.c_str());
    }
  }
  *out = c;
  return RNP_OK;
}

rnp_status rnp_destroy(rnp_ctx* c) {
  if (!c) return RNP_OK;
  DevGuard gd(c->dev);
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->st2) cudaStreamSynchronize(c->st2);
  if (c->st3) cudaStreamSynchronize(c->st3);
  destroy_buffers(c);
  delete c;
  return RNP_OK;
}

rnp_status rnp_fine_batch(rnp_ctx* c, const double* U_in, int n, double* U_out) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!U_in || !U_out || n < 1 || n > c->N) return fail(c, RNP_EINVAL, "bad arguments");
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  Items it = affine(c->B * n, 0, c->d, 0, c->d, nullptr);
  if (!c->plain && c->B * n > c->B * c->N) return fail(c, RNP_EINVAL, "too many items");
  CK(cudaMemsetAsync(c->flags + 3, 0, sizeof(int), c->st));
  rnp_status s = run_stencil(c, true, U_in, U_out, nullptr, it);
  if (s) return s;
  CK(cudaMemcpyAsync(c->h_flags + 3, c->flags + 3, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_flags[3]) return fail(c, RNP_ETIMEOUT, kTimeoutMsg);
  return RNP_OK;
}

rnp_status rnp_get_weights(rnp_ctx* c, double* A, double* zeta) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  rnp_status s = ensure_weights(c);
  if (s) return s;
  if (A) CK(cudaMemcpyAsync(A, c->A, sizeof(double) * c->M * c->d, cudaMemcpyDeviceToDevice, c->st));
  if (zeta) CK(cudaMemcpyAsync(zeta, c->zeta, sizeof(double) * c->M, cudaMemcpyDeviceToDevice, c->st));
  return RNP_OK;
}

rnp_status rnp_set_scaling(rnp_ctx* c, const double* hc, const double* hr) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!hc || !hr) return fail(c, RNP_EINVAL, "NULL scaling");
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  for (int i = 0; i < c->B * 3; ++i) {
    if (!(hr[i] != 0.0)) return fail(c, RNP_EINVAL, "scale r must be nonzero");
    c->h_c[i] = hc[i];
    c->h_r[i] = hr[i];
  }
  CK(cudaMemcpyAsync(c->sc, c->h_c, sizeof(double) * c->B * 3, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->sr, c->h_r, sizeof(double) * c->B * 3, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->scaling_ready = true;
  return RNP_OK;
}

rnp_status rnp_get_scaling(rnp_ctx* c, double* hc, double* hr) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  if (!c->scaling_ready) {
    for (int i = 0; i < c->B * 3; ++i) { hc[i] = 0.0; hr[i] = 1.0; }
    return RNP_OK;
  }
  CK(cudaMemcpyAsync(hc, c->sc, sizeof(double) * c->B * 3, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hr, c->sr, sizeof(double) * c->B * 3, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return RNP_OK;
}

rnp_status rnp_reset(rnp_ctx* c) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  std::fill(c->P.begin(), c->P.end(), 0);
  c->scaling_ready = false;
  return upload_P(c);
}

rnp_status rnp_stencil_config(const rnp_ctx* c, int which, int* out) {
  if (!c || !out || (which != 0 && which != 1)) return RNP_EINVAL;
  const StencilCfg& s = which == 0 ? c->cfgF : c->cfgG;
  out[0] = c->plain ? 0 : s.cluster;
  out[1] = c->plain ? 256 : s.threads;
  out[2] = s.px;
  out[3] = s.px ? s.rs : s.R;
  out[4] = which == 0 ? c->tunedF : c->tunedG;
  out[5] = s.px ? s.tm : 0;
  return RNP_OK;
}

static rnp_status ensure_scaling_identity(rnp_ctx* c);

rnp_status rnp_features(rnp_ctx* c, const double* U, int R, double* phi) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!U || !phi || R < 1 || R > c->feat_rows_cap || R > c->itemcap)
    return fail(c, RNP_EINVAL, "bad arguments (1 <= R <= %d)", std::min(c->feat_rows_cap, c->itemcap));
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  rnp_status s = ensure_weights(c);
  if (s) return s;
  if ((s = ensure_scaling_identity(c))) return s;
  for (int r = 0; r < R; ++r) c->h_app[r] = 0;  // member 0's scaling
  CK(cudaMemcpyAsync(c->d_app, c->h_app, sizeof(int) * R, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st));
  Rows src{nullptr, 0, c->d}, dst{nullptr, 0, c->d}, prow{nullptr, 0, c->M};
  double* S64 = c->Fv;                                // scratch rows
  float* S32 = reinterpret_cast<float*>(c->Fv);
  CK(launch_scale_rows(c->g, U, src, c->d_app, 1, c->sc, c->sr, c->fp32 ? nullptr : S64,
                       c->fp32 ? S32 : nullptr, dst, R, nullptr, c->st));
  if ((s = batch_features(c, S64, S32, dst, R, phi, prow))) return s;
  CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_flags[3]) return fail(c, RNP_ETIMEOUT, kTimeoutMsg);
  return RNP_OK;
}

rnp_status rnp_get_pairs(rnp_ctx* c, long long* pairs) {
  if (!c || !pairs) return RNP_EINVAL;
  for (int b = 0; b < c->B; ++b) pairs[b] = c->P[b];
  return RNP_OK;
}

static rnp_status ensure_scaling_identity(rnp_ctx* c) {
  if (c->scaling_ready) return RNP_OK;
  double hc[RNP_MAX_BATCH * 3], hr[RNP_MAX_BATCH * 3];
  for (int i = 0; i < c->B * 3; ++i) { hc[i] = 0.0; hr[i] = 1.0; }
  return rnp_set_scaling(c, hc, hr);
}

rnp_status rnp_randnet_fit(rnp_ctx* c, const double* Uin, const double* Y, int P) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!Uin || !Y || P < 0) return fail(c, RNP_EINVAL, "bad arguments");
  if (P == 0) return RNP_OK;
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  for (int b = 0; b < c->B; ++b)
    if (c->P[b] + (long long)P > c->cap)
      return fail(c, RNP_ENOMEM, "dataset arena full (%lld rows per member)", c->cap);
  rnp_status s = ensure_weights(c);
  if (s) return s;
  if ((s = ensure_scaling_identity(c))) return s;
  // rows in chunks that fit the offset tables and the feature workspace
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st));
  const int chunk = std::min(c->itemcap, c->feat_rows_cap);
  const int R = c->B * P;
  long long* src = c->h_items;
  long long* sdst = c->h_items + c->itemcap;
  long long* pdst = c->h_items + 2 * c->itemcap;
  int* rowb = c->h_app;
  for (int r0 = 0; r0 < R; r0 += chunk) {
    const int n = std::min(chunk, R - r0);
    for (int r = 0; r < n; ++r) {
      const int b = (r0 + r) / P, t = (r0 + r) % P;
      src[r] = ((long long)b * P + t) * c->d;
      sdst[r] = ((long long)b * c->cap + c->P[b] + t) * c->d;
      pdst[r] = ((long long)b * c->cap + c->P[b] + t) * c->M;
      rowb[r] = b;
    }
    CK(cudaMemcpyAsync(c->d_items, c->h_items, sizeof(long long) * 3 * c->itemcap,
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_app, c->h_app, sizeof(int) * c->itemcap, cudaMemcpyHostToDevice,
                       c->st));
    Rows rsrc{c->d_items, 0, 0}, rdst{c->d_items + c->itemcap, 0, 0};
    CK(launch_scale_rows(c->g, Uin, rsrc, c->d_app, 1, c->sc, c->sr, c->fp32 ? nullptr : c->Sds,
                         c->fp32 ? c->S32 : nullptr, rdst, n, nullptr, c->st));
    CK(launch_copy_rows(Y, c->d_items, c->Yds, c->d_items + c->itemcap, c->d, n, c->st));
    Rows prow{c->d_items + 2 * c->itemcap, 0, 0};
    {
      rnp_status fs = batch_features(c, c->Sds, c->S32, rdst, n, c->Phi, prow);
      if (fs) return fs;
    }
    CK(cudaStreamSynchronize(c->st));  // the staging tables are reused
  }
  CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_flags[3]) return fail(c, RNP_ETIMEOUT, kTimeoutMsg);
  for (int b = 0; b < c->B; ++b) c->P[b] += P;
  return upload_P(c);
}

rnp_status rnp_randnet_predict(rnp_ctx* c, const double* q, double* out) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!q || !out) return fail(c, RNP_EINVAL, "bad arguments");
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  rnp_status s = ensure_weights(c);
  if (s) return s;
  if ((s = ensure_scaling_identity(c))) return s;
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st));
  if ((s = predict_core(c, q, 0, c->d, c->phiq, 0, c->M, nullptr))) return s;
  CK(launch_update(nullptr, 0, c->Yds, c->cap, c->d, c->alpha, c->idx, c->meff, out, c->d,
                   nullptr, 0, c->flags + 2, c->B, nullptr, c->st));
  int esc, fl, nf;
  if ((s = read_flags(c, &esc, &fl, &nf))) return s;
  if (fl) return fail(c, RNP_ENONFINITE, "ridge system not positive definite");
  return RNP_OK;
}

rnp_status rnp_coarse_sweep(rnp_ctx* c, int first, const double* U_first, double* U) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!U_first || !U || first < 0 || first > c->N) return fail(c, RNP_EINVAL, "bad arguments");
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  const long long d = c->d, sb = (long long)(c->N + 1) * d;
  CK(cudaMemcpy2DAsync(U + (long long)first * d, sizeof(double) * sb, U_first,
                       sizeof(double) * d, sizeof(double) * d, c->B, cudaMemcpyDeviceToDevice,
                       c->st));
  const bool use_fhat = c->randnet && Pmax(c) > 0;
  rnp_status s;
  if (use_fhat) {
    if ((s = ensure_weights(c))) return s;
    if ((s = ensure_scaling_identity(c))) return s;
  }
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st));
  if (use_fhat && first < c->N)  // the first step's scaled query (later: from the update)
    CK(launch_scale_rows(c->g, U, Rows{nullptr, (long long)first * d, sb}, nullptr, 1, c->sc,
                         c->sr, c->fp32 ? nullptr : c->qbuf, c->fp32 ? c->q32 : nullptr,
                         Rows{nullptr, 0, d}, c->B, nullptr, c->st));
  for (int i = first + 1; i <= c->N; ++i) {
    if (!use_fhat) {
      Items it = affine(c->B, (long long)(i - 1) * d, sb, (long long)i * d, sb, nullptr);
      if ((s = run_stencil(c, false, U, U, nullptr, it))) return s;
      continue;
    }
    if ((s = sweep_step(c, U, sb, i, nullptr, nullptr, nullptr))) return s;
  }
  if (first == 0 && !use_fhat && c->p.scale_mode == RNP_SCALE_MINMAX) {
    CK(launch_scaling(c->g, U, sb, c->N + 1, c->B, false, c->sc, c->sr, c->scale_work,
                      c->flags + 2, nullptr, c->st));
    c->scaling_ready = true;
  }
  int esc, fl, nf;
  if ((s = read_flags(c, &esc, &fl, &nf))) return s;
  if (fl) return fail(c, RNP_ENONFINITE, "ridge system not positive definite");
  if (nf) return fail(c, RNP_ENONFINITE, "non-finite state in the sweep");
  return RNP_OK;
}

}  // extern "C"

namespace {

// k = 0 of Alg. 1 for the members with want[b]: U_b,0 = u0 (row b of u0,
// member stride u0_bstride; device or host memory), U_b,i = G(U_b,i-1) for
// i = 1..N with the G values kept for the first targets, then the member's
// scaling.  The members become active with an empty dataset.
rnp_status start_members(rnp_ctx* c, const std::vector<int>& want, const double* u0,
                         long long u0_bstride, rnp_stats* st) {
  const int B = c->B, N = c->N;
  const long long d = c->d, sb = (long long)(N + 1) * d, nb = (long long)N * d;
  rnp_status s;
  float ms;
  for (int b = 0; b < B; ++b) {
    c->h_mask[b] = want[b] ? 1 : 0;
    if (want[b]) c->P[b] = 0;
  }
  if ((s = upload_P(c))) return s;
  CK(cudaMemcpyAsync(c->d_mask, c->h_mask, sizeof(int) * B, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st));
  for (int b = 0; b < B; ++b)
    if (want[b])
      CK(cudaMemcpyAsync(c->U + (long long)b * sb, u0 + (long long)b * u0_bstride,
                         sizeof(double) * d, cudaMemcpyDefault, c->st));
  CK(cudaEventRecord(c->ev[0], c->st));
  for (int i = 1; i <= N; ++i) {
    Items it = affine(B, (long long)(i - 1) * d, sb, (long long)i * d, sb, c->d_mask);
    it.dst2_base = (long long)(i - 1) * d;
    it.dst2_stride = nb;
    if ((s = run_stencil(c, false, c->U, c->U, c->Gc, it))) return s;
  }
  CK(launch_scaling(c->g, c->U, sb, N + 1, B, c->p.scale_mode == RNP_SCALE_NONE, c->sc, c->sr,
                    c->scale_work, c->flags + 2, c->d_mask, c->st));
  c->scaling_ready = true;
  if (c->randnet && (s = ensure_weights(c))) return s;
  CK(cudaEventRecord(c->ev[1], c->st));
  CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_flags[3]) return fail(c, RNP_ETIMEOUT, kTimeoutMsg);
  if (c->h_flags[2]) return fail(c, RNP_ENONFINITE, "non-finite state in the k = 0 sweep");
  CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  if (st) st->t_sweep_ms += ms;
  for (int b = 0; b < B; ++b)
    if (want[b]) {
      c->mL[b] = 0;
      c->mK[b] = 0;
      c->mstate[b] = RNP_MEMBER_ACTIVE;
    }
  return RNP_OK;
}

// Where a buffer lives: host memory (pinned, or pageable and unknown to
// CUDA), and for pinned memory its device address (null if it has none).
struct HostMem {
  bool host = false;
  double* dptr = nullptr;
};
HostMem host_memory(void* p) {
  HostMem h;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    h.host = true;
    return h;
  }
  h.host = a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
  if (a.type == cudaMemoryTypeHost) h.dptr = static_cast<double*>(a.devicePointer);
  return h;
}

// Sends states sent[b] + 1 .. upto[b] of every member from the context's U
// to Uout (member stride (N + 1) d) on the copy stream, after the work on
// the main stream so far.  States U_0 .. U_L of a member are final once
// Eq. 5 has set L: later iterations only read them.
rnp_status send_states(rnp_ctx* c, double* Uout, std::vector<int>& sent,
                       const std::vector<int>& upto) {
  const long long d = c->d, sb = (long long)(c->N + 1) * d;
  bool any = false;
  for (int b = 0; b < c->B; ++b) any |= upto[b] > sent[b];
  if (!any) return RNP_OK;
  CK(cudaEventRecord(c->evc, c->st));
  CK(cudaStreamWaitEvent(c->st3, c->evc, 0));
  for (int b = 0; b < c->B; ++b) {
    if (upto[b] <= sent[b]) continue;
    const long long off = (long long)b * sb + (long long)(sent[b] + 1) * d;
    CK(cudaMemcpyAsync(Uout + off, c->U + off,
                       sizeof(double) * d * (upto[b] - sent[b]), cudaMemcpyDefault, c->st3));
    sent[b] = upto[b];
  }
  return RNP_OK;
}

// Waits for the copy stream when a solve into host memory leaves, also on
// an error, so that no copy into the caller's buffer outlives the call.
struct CopyDrain {
  rnp_ctx* c;
  ~CopyDrain() { cudaStreamSynchronize(c->st3); }
};

// One iteration of Alg. 1 for every active member: the parallel fine step
// over all their unconverged starts (one launch), the dataset append of
// Eq. 6, the exact leftmost slice, the sweep of Eq. 3 and the stopping rule
// of Eq. 5.  Members may be at different iterations.
rnp_status iterate_once(rnp_ctx* c, rnp_stats* st, int* n_active) {
  const int B = c->B, N = c->N, M = c->M;
  const long long d = c->d, sb = (long long)(N + 1) * d, nb = (long long)N * d;
  rnp_status s;
  float ms;
  std::vector<int>& L = c->mL;
  auto active = [&](int b) { return c->mstate[b] == RNP_MEMBER_ACTIVE; };
  // ---- work list: first-iteration members' rows first --------------------
  int nit = 0, nfirst = 0;
  long long* srco = c->h_items;
  long long* dsto = c->h_items + c->itemcap;
  long long* soff = c->h_items + 2 * c->itemcap;
  long long* poff = c->h_items + 3 * c->itemcap;
  int* ab = c->h_app;
  int* aj = c->h_app + c->itemcap;
  int* ap = c->h_app + 2 * c->itemcap;
  for (int pass = 0; pass < 2; ++pass)
    for (int b = 0; b < B; ++b) {
      if (!active(b) || (c->mK[b] == 0) != (pass == 0)) continue;
      if (c->randnet && c->P[b] + (N - L[b]) > c->cap)
        return fail(c, RNP_ENOMEM, "dataset arena full (%lld rows per member)", c->cap);
      for (int j = L[b]; j < N; ++j) {
        const int p = c->P[b] + (j - L[b]);
        srco[nit] = (long long)b * sb + (long long)j * d;
        dsto[nit] = (long long)b * nb + (long long)j * d;
        soff[nit] = ((long long)b * c->cap + p) * d;
        poff[nit] = ((long long)b * c->cap + p) * M;
        ab[nit] = b; aj[nit] = j; ap[nit] = p;
        ++nit;
      }
      if (pass == 0) nfirst = nit;
    }
  if (nit == 0) { *n_active = 0; return RNP_OK; }
  for (int i = 0; i <= N; ++i)
    for (int b = 0; b < B; ++b) c->h_gate[i * B + b] = (active(b) && i >= L[b] + 2) ? 1 : 0;
  CK(cudaMemcpyAsync(c->d_items, c->h_items, sizeof(long long) * 4 * c->itemcap,
                     cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_app, c->h_app, sizeof(int) * 3 * c->itemcap, cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaMemcpyAsync(c->d_gate, c->h_gate, sizeof(int) * (N + 1) * B, cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned long long) * B * (N + 1), c->st));
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, c->st));
  // ---- parallel fine step --------------------------------------------------
  CK(cudaEventRecord(c->ev[0], c->st));
  Items fit{};
  fit.src_off = c->d_items;
  fit.dst_off = c->d_items + c->itemcap;
  fit.n = nit;
  if ((s = run_stencil(c, true, c->U, c->Fv, nullptr, fit))) return s;
  CK(cudaEventRecord(c->ev[1], c->st));
  for (int b = 0; b < B; ++b)
    if (active(b)) st->fine_cell_updates += (long long)(N - L[b]) * c->p.nF * d;
  // ---- dataset append (Eq. 6) and features of the new rows -----------------
  AppendItems ai{c->d_app, c->d_app + c->itemcap, c->d_app + 2 * c->itemcap, nit};
  CK(launch_append(c->g, c->U, sb, c->Fv, c->Gc, nb, c->Yv, c->fp32 ? nullptr : c->Sds,
                   c->fp32 ? c->S32 : nullptr, c->Yds, c->cap, c->sc, c->sr, ai, c->randnet,
                   c->st));
  if (c->randnet) {
    if (nfirst > 0) {  // first iteration: features of the k = 0 starts
      Rows srows{c->d_items + 2 * c->itemcap, 0, 0};
      Rows prow{c->d_items + 3 * c->itemcap, 0, 0};
      if ((s = batch_features(c, c->Sds, c->S32, srows, nfirst, c->Phi, prow))) return s;
    }
    if (nit > nfirst) {  // later iterations: the sweep already computed them
      AppendItems rest{c->d_app + nfirst, c->d_app + c->itemcap + nfirst,
                       c->d_app + 2 * c->itemcap + nfirst, nit - nfirst};
      CK(launch_copy_phi(c->phic, (long long)N * M, c->Phi, c->cap, M, rest, c->st));
    }
    for (int b = 0; b < B; ++b)
      if (active(b)) c->P[b] += N - L[b];
    for (int b = 0; b < B; ++b) c->h_flags[4 + b] = c->P[b];
    CK(cudaMemcpyAsync(c->dP, c->h_flags + 4, sizeof(int) * B, cudaMemcpyHostToDevice, c->st));
  }
  // ---- exact leftmost slice: U_{L+1} = F(U_L) ------------------------------
  for (int b = 0; b < B; ++b)
    if (active(b))
      CK(cudaMemcpyAsync(c->U + (long long)b * sb + (long long)(L[b] + 1) * d,
                         c->Fv + (long long)b * nb + (long long)L[b] * d, sizeof(double) * d,
                         cudaMemcpyDeviceToDevice, c->st));
  CK(cudaEventRecord(c->ev[2], c->st));
  // ---- sequential predictor-corrector sweep (Eq. 3) ------------------------
  int imin = N + 1;
  for (int b = 0; b < B; ++b)
    if (active(b)) imin = std::min(imin, L[b] + 2);
  if (c->randnet && imin <= N) {
    // the first step's scaled query U[b][L+1]; later steps get theirs from
    // the update of the step before
    for (int b = 0; b < B; ++b) {
      c->h_qgate[b] = (active(b) && L[b] + 2 <= N) ? 1 : 0;
      c->h_qsrc[b] = (long long)b * sb + (long long)(L[b] + 1) * d;
    }
    CK(cudaMemcpyAsync(c->d_qsrc, c->h_qsrc, sizeof(long long) * B, cudaMemcpyHostToDevice,
                       c->st));
    CK(cudaMemcpyAsync(c->d_qgate, c->h_qgate, sizeof(int) * B, cudaMemcpyHostToDevice, c->st));
    CK(launch_scale_rows(c->g, c->U, Rows{c->d_qsrc, 0, 0}, nullptr, 1, c->sc, c->sr,
                         c->fp32 ? nullptr : c->qbuf, c->fp32 ? c->q32 : nullptr,
                         Rows{nullptr, 0, d}, B, c->d_qgate, c->st));
  }
  if (imin <= N && (s = solve_sweep(c, imin))) return s;
  CK(cudaEventRecord(c->ev[3], c->st));
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(unsigned long long) * B * (N + 1),
                     cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_flags[3]) return fail(c, RNP_ETIMEOUT, kTimeoutMsg);
  CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  st->t_fine_ms += ms;
  CK(cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]));
  st->t_fit_ms += ms;
  CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
  st->t_sweep_ms += ms;
  st->lambda_escalations += c->h_flags[0];
  if (c->h_flags[1]) return fail(c, RNP_ENONFINITE, "ridge system not positive definite");
  if (c->h_flags[2]) return fail(c, RNP_ENONFINITE, "non-finite state");
  // ---- stopping rule (Eq. 5) -----------------------------------------------
  const int Kmax = std::min(c->p.max_iters, N);
  int left = 0;
  for (int b = 0; b < B; ++b) {
    if (!active(b)) continue;
    int Ln = L[b] + 1;
    for (int i = L[b] + 2; i <= N; ++i) {
      double e;
      memcpy(&e, &c->h_err[(long long)b * (N + 1) + i], sizeof(double));
      if (e < c->p.tol) Ln = i; else break;
    }
    L[b] = Ln;
    c->mK[b] += 1;
    if (L[b] == N) c->mstate[b] = RNP_MEMBER_CONVERGED;
    else if (c->mK[b] >= Kmax) c->mstate[b] = RNP_MEMBER_NOTCONV;
    else ++left;
  }
  *n_active = left;
  return RNP_OK;
}

}  // namespace

extern "C" {

rnp_status rnp_solve(rnp_ctx* c, const double* u0, double* Uout, rnp_stats* stats) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!u0 || !Uout) return fail(c, RNP_EINVAL, "bad arguments");
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  auto t_start = std::chrono::steady_clock::now();
  const long long launches0 = launches_total();
  const int B = c->B, N = c->N;
  const long long d = c->d, sb = (long long)(N + 1) * d;
  rnp_stats st;
  memset(&st, 0, sizeof(st));
  rnp_status s;
  const std::vector<int> all(B, 1);
  // U in host memory: each member's converged states go out on the copy
  // stream after every iteration, overlapping the next one; the rest at the
  // end, into pinned memory by SM stores through its device address (after
  // the iterations the destination's address translations are cold, and the
  // copy engine resolves them a few at a time: 2.1 GB took 240 ms that way
  // and 57 ms by SM stores on GB300; 11 ms either way when warm)
  const HostMem out = host_memory(Uout);
  const bool host_out = out.host;
  CopyDrain drain{c};
  std::vector<int> sent(B, -1);
  s = start_members(c, all, u0, d, &st);
  if (s != RNP_OK) return s;
  int n_active = B;
  while (n_active > 0) {
    s = iterate_once(c, &st, &n_active);
    if (s != RNP_OK) return s;
    if (host_out && n_active > 0 && (s = send_states(c, Uout, sent, c->mL))) return s;
  }
  if (host_out && out.dptr) {
    Segments sg;
    sg.n = 0;
    for (int b = 0; b < B; ++b) {
      if (sent[b] >= N) continue;
      sg.off[sg.n] = (long long)b * sb + (long long)(sent[b] + 1) * d;
      sg.len[sg.n] = (long long)(N - sent[b]) * d;
      ++sg.n;
      sent[b] = N;
    }
    CK(launch_copy_segments(c->U, out.dptr, sg, c->st));
    CK(cudaStreamSynchronize(c->st3));
  } else if (host_out) {
    if ((s = send_states(c, Uout, sent, std::vector<int>(B, N)))) return s;
    CK(cudaStreamSynchronize(c->st3));
  } else {
    CK(cudaMemcpyAsync(Uout, c->U, sizeof(double) * B * sb, cudaMemcpyDeviceToDevice, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  st.converged = 1;
  st.L = N;
  for (int b = 0; b < B; ++b) {
    st.K = std::max(st.K, c->mK[b]);
    st.K_each[b] = c->mK[b];
    st.L = std::min(st.L, c->mL[b]);
    st.converged &= c->mstate[b] == RNP_MEMBER_CONVERGED;
    st.pairs += c->P[b];
    c->mstate[b] = RNP_MEMBER_FREE;
  }
  st.t_total_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  st.kernel_launches = launches_total() - launches0;
  if (stats) *stats = st;
  if (!st.converged)
    return fail(c, RNP_ENOTCONV, "not converged after %d iterations",
                std::min(c->p.max_iters, N));
  return RNP_OK;
}

rnp_status rnp_member_start(rnp_ctx* c, int member, const double* u0) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!u0 || member < 0 || member >= c->B) return fail(c, RNP_EINVAL, "bad arguments");
  if (c->mstate[member] == RNP_MEMBER_ACTIVE)
    return fail(c, RNP_EBUSY, "member %d is still iterating", member);
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  std::vector<int> want(c->B, 0);
  want[member] = 1;
  // member stride 0: row `member` of the source is u0 itself
  return start_members(c, want, u0, 0, &c->run);
}

rnp_status rnp_iterate(rnp_ctx* c, int* active) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  int n = 0;
  rnp_status s = iterate_once(c, &c->run, &n);
  if (active) *active = n;
  return s;
}

rnp_status rnp_member_status(const rnp_ctx* c, int member, int* state, int* K, int* L) {
  if (!c || member < 0 || member >= c->B) return RNP_EINVAL;
  if (state) *state = c->mstate[member];
  if (K) *K = c->mK[member];
  if (L) *L = c->mL[member];
  return RNP_OK;
}

rnp_status rnp_member_result(rnp_ctx* c, int member, double* U) {
  if (!c) return RNP_EINVAL;
  c->msg.clear();
  if (!U || member < 0 || member >= c->B) return fail(c, RNP_EINVAL, "bad arguments");
  if (c->mstate[member] == RNP_MEMBER_ACTIVE || c->mstate[member] == RNP_MEMBER_FREE)
    return fail(c, RNP_EINVAL, "member %d has no finished result", member);
  DevGuard gd(c->dev);
  StreamJoin sj(c);
  const long long sb = (long long)(c->N + 1) * c->d;
  CK(cudaMemcpyAsync(U, c->U + (long long)member * sb, sizeof(double) * sb,
                     cudaMemcpyDeviceToDevice, c->st));
  const int st = c->mstate[member];
  c->mstate[member] = RNP_MEMBER_FREE;
  return st == RNP_MEMBER_CONVERGED ? RNP_OK : RNP_ENOTCONV;
}

}  // extern "C"
