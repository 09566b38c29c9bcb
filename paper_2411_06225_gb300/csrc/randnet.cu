// randnet.cu -- the RandNet correction of Eq. randnet: seeded random weights
// (Alg. 3), per-species rescaling (Alg. 1 initialisation), random features
// phi = ReLU(A s + zeta) (Eq. HA), the m-nearest-neighbour restriction of
// App. B, the ridge readout of Eq. ridgeless in its dual m x m form, and
// the predictor-corrector update of Eq. 3 fused with the max-norm of Eq. 5.
//
// Reductions over the state dimension d are split into fixed chunks whose
// partial sums are combined in a fixed order, so every result is
// reproducible run to run.  The m x m ridge system is assembled and solved
// with explicitly rounded FP64 operations in the order of the plain serial
// formulas.
#include <atomic>
#include <cstdint>

#include "rnp_internal.h"

namespace rnp {

static std::atomic<long long> g_launches{0};
long long launches_total() { return g_launches.load(); }
void count_launches(long long n) { g_launches += n; }

static int grid_cap(long long tot, int threads, int cap = 152 * 16) {
  long long b = (tot + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Weights: SplitMix64 (Steele, Lea & Flood 2014) in counter form.  Draw
// number (stream * 2^40 + idx + 1) of the generator seeded with `seed` is
// mix(seed + n * gamma); u = top 53 bits * 2^-53;  value = 2u - 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double sm64_uniform(uint64_t seed, uint32_t stream,
                                               uint64_t idx) {
  const uint64_t n = ((uint64_t)stream << 40) + idx + 1;
  const uint64_t z = sm64_mix(seed + n * 0x9e3779b97f4a7c15ULL);
  return __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
}

// Round-to-nearest-even of a double to bfloat16 (8 significant bits), done
// on the double's bits so that there is a single rounding.
__device__ __forceinline__ uint16_t to_bf16_rne(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint64_t lsb = (b >> 45) & 1ULL;
  b += 0x00000FFFFFFFFFFFULL + lsb;
  b &= ~((1ULL << 45) - 1ULL);
  const float f = (float)__longlong_as_double((long long)b);  // exact
  return (uint16_t)(__float_as_uint(f) >> 16);
}

__global__ void k_weights(uint64_t seed, int M, long long d, double* A, double* zeta,
                          float* A32, uint16_t* Abf, float* zeta32) {
  const long long tot = (long long)M * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = __dsub_rn(__dmul_rn(2.0, sm64_uniform(seed, 0, (uint64_t)t)), 1.0);
    if (A) A[t] = v;
    if (A32) A32[t] = (float)v;
    if (Abf) Abf[t] = to_bf16_rne(v);
    if (t < M) {
      const double z = __dsub_rn(__dmul_rn(2.0, sm64_uniform(seed, 1, (uint64_t)t)), 1.0);
      if (zeta) zeta[t] = z;
      if (zeta32) zeta32[t] = (float)z;
    }
  }
}

cudaError_t launch_weights(uint64_t seed, int M, long long d, double* A, double* zeta,
                           float* A32, uint16_t* Abf16, float* zeta32, cudaStream_t st) {
  const long long tot = (long long)M * d;
  count_launches(1);
  k_weights<<<grid_cap(tot, 256), 256, 0, st>>>(seed, M, d, A, zeta, A32, Abf16, zeta32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-species scaling
// ---------------------------------------------------------------------------
__global__ void k_minmax_partial(const double* U, long long bstride, int nstates,
                                 long long n, long long d, int ncomp, double* work,
                                 int nchunk, int* nonfinite, const int* mask) {
  // blockIdx.y = b * ncomp + q ; blockIdx.x = chunk
  const int bq = blockIdx.y;
  const int b = bq / ncomp, q = bq - b * ncomp;
  if (mask && !mask[b]) return;
  const long long tot = (long long)nstates * n;
  double mn = 1.0 / 0.0, mx = -1.0 / 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)nchunk * blockDim.x) {
    const long long s = t / n, j = t - s * n;
    const double v = U[b * bstride + s * d + q * n + j];
    if (nonfinite && !isfinite(v)) *nonfinite = 1;
    mn = v < mn ? v : mn;
    mx = v > mx ? v : mx;
  }
  __shared__ double smn[256], smx[256];
  smn[threadIdx.x] = mn;
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = smn[threadIdx.x + o], c = smx[threadIdx.x + o];
      if (a < smn[threadIdx.x]) smn[threadIdx.x] = a;
      if (c > smx[threadIdx.x]) smx[threadIdx.x] = c;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    work[(bq * (long long)nchunk + blockIdx.x) * 2] = smn[0];
    work[(bq * (long long)nchunk + blockIdx.x) * 2 + 1] = smx[0];
  }
}

__global__ void k_minmax_finish(const double* work, int nchunk, int B, int ncomp,
                                bool none, double* c, double* r, const int* mask) {
  const int bq = blockIdx.x * blockDim.x + threadIdx.x;
  if (bq >= B * ncomp) return;
  const int b = bq / ncomp, q = bq - b * ncomp;
  if (mask && !mask[b]) return;
  if (none) {
    c[b * 3 + q] = 0.0;
    r[b * 3 + q] = 1.0;
    return;
  }
  double mn = work[(bq * (long long)nchunk) * 2], mx = work[(bq * (long long)nchunk) * 2 + 1];
  for (int k = 1; k < nchunk; ++k) {
    const double a = work[(bq * (long long)nchunk + k) * 2];
    const double e = work[(bq * (long long)nchunk + k) * 2 + 1];
    if (a < mn) mn = a;
    if (e > mx) mx = e;
  }
  const double cc = __dmul_rn(0.5, __dadd_rn(mx, mn));
  double rr = __dmul_rn(0.5, __dsub_rn(mx, mn));
  if (rr == 0.0) rr = 1.0;
  c[b * 3 + q] = cc;
  r[b * 3 + q] = rr;
}

static const int kScaleChunks = 64;

cudaError_t launch_scaling(const Geom& g, const double* U, long long bstride, int nstates,
                           int B, bool none, double* c, double* r, double* work,
                           int* nonfinite, const int* mask, cudaStream_t st) {
  dim3 grid(kScaleChunks, B * g.ncomp);
  count_launches(1);
  k_minmax_partial<<<grid, 256, 0, st>>>(U, bstride, nstates, g.n, g.d, g.ncomp, work,
                                         kScaleChunks, nonfinite, mask);
  count_launches(1);
  k_minmax_finish<<<(B * g.ncomp + 63) / 64, 64, 0, st>>>(work, kScaleChunks, B, g.ncomp,
                                                          none, c, r, mask);
  return cudaGetLastError();
}

__global__ void k_scale_rows(const double* U, Rows src, const int* row_b, int row_b_div,
                             const double* c, const double* r, double* S, float* S32,
                             Rows dst, int R, long long n, long long d, const int* gate) {
  const long long tot = (long long)R * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / d);
    if (gate && !gate[row]) continue;
    const long long e = t - (long long)row * d;
    const int q = (int)(e / n);
    const int b = row_b ? row_b[row] : row / row_b_div;
    const double u = U[item_off(src.off, src.base, src.stride, row) + e];
    const double v = __ddiv_rn(__dsub_rn(u, c[b * 3 + q]), r[b * 3 + q]);
    const long long o = item_off(dst.off, dst.base, dst.stride, row) + e;
    if (S) S[o] = v;
    if (S32) S32[o] = (float)v;
  }
}

cudaError_t launch_scale_rows(const Geom& g, const double* U, Rows src, const int* row_b,
                              int row_b_div, const double* c, const double* r, double* S,
                              float* S32, Rows dst, int R, const int* gate, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  count_launches(1);
  k_scale_rows<<<grid_cap((long long)R * g.d, 256), 256, 0, st>>>(
      U, src, row_b, row_b_div, c, r, S, S32, dst, R, g.n, g.d, gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Random features (Eq. HA), FP64 or FP32 operands.  Stage 1: a CTA takes a
// chunk of CH coordinates, TR rows and FW neurons; every warp owns two
// neurons and computes their TR partial dot products A[w, chunk] . s[r, chunk]
// (lanes stride the chunk, then a fixed butterfly reduction).  Stage 2 sums
// the chunk partials in chunk order (FP64), adds zeta and applies ReLU.
// ---------------------------------------------------------------------------
static const int kFeatCH = 1024;
static const int kFeatTR = 4;
static const int kFeatFW = 16;

int features_chunks(long long d) { return (int)((d + kFeatCH - 1) / kFeatCH); }

// Partials of row r, neuron w, chunk ch at part[(r * M + w) * nch + ch]
// (row-major, CM = false) or at part[(ch * R + r) * M + w] (chunk-major: the
// finishing threads, one per neuron, then read consecutive addresses).
template <typename T, typename TP, bool CM>
__device__ __forceinline__ void feat_partial_body(T (&sS)[kFeatTR][kFeatCH], const T* A, int M,
                                                  long long d, const T* S, Rows rows, int R,
                                                  TP* part, int nch, const int* gate,
                                                  int ch, int ry, int wz) {
  const int r0 = ry * kFeatTR;
  const int w0 = wz * kFeatFW;
  const long long j0 = (long long)ch * kFeatCH;
  const int len = (int)((d - j0) < kFeatCH ? (d - j0) : kFeatCH);
  bool any = false;
  for (int r = 0; r < kFeatTR; ++r) {
    const int row = r0 + r;
    const bool on = row < R && (!gate || gate[row]);
    any |= on;
    const T* src = on ? S + item_off(rows.off, rows.base, rows.stride, row) + j0 : nullptr;
    for (int j = threadIdx.x; j < kFeatCH; j += blockDim.x)
      sS[r][j] = (on && j < len) ? src[j] : T(0);
  }
  if (!any) return;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = w0 + warp; w < M && w < w0 + kFeatFW; w += 8) {
    const T* Aw = A + (long long)w * d + j0;
    // (loops unrolled so that a lane's loads of a chunk are in flight together)
    T acc[kFeatTR];
#pragma unroll
    for (int r = 0; r < kFeatTR; ++r) acc[r] = T(0);
#pragma unroll 16
    for (int j = lane; j < len; j += 32) {
      const T a = Aw[j];
#pragma unroll
      for (int r = 0; r < kFeatTR; ++r) acc[r] = fma(a, sS[r][j], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kFeatTR; ++r) {
      T v = acc[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[r] = v;
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < kFeatTR; ++r)
        if (r0 + r < R) {
          const long long at = CM ? ((long long)ch * R + (r0 + r)) * M + w
                                  : ((long long)(r0 + r) * M + w) * nch + ch;
          part[at] = (TP)acc[r];
        }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_feat_partial(const T* A, int M, long long d,
                                                      const T* S, Rows rows, int R,
                                                      double* part, int nch,
                                                      const int* gate) {
  __shared__ T sS[kFeatTR][kFeatCH];
  feat_partial_body<T, double, false>(sS, A, M, d, S, rows, R, part, nch, gate, blockIdx.x,
                                      blockIdx.y, blockIdx.z);
}

__global__ void k_feat_finish(const double* part, int nch, int R, int M, const double* zeta,
                              double* phi, Rows prow, const int* gate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * M) return;
  const int row = t / M, w = t - row * M;
  if (gate && !gate[row]) return;
  const double* p = part + (long long)t * nch;
  double acc = 0.0;
  for (int k = 0; k < nch; ++k) acc = acc + p[k];
  const double v = acc + zeta[w];
  phi[item_off(prow.off, prow.base, prow.stride, row) + w] = v > 0.0 ? v : 0.0;
}

template <typename T>
static cudaError_t launch_features_t(const T* A, const double* zeta, int M, long long d,
                                     const T* S, Rows s_rows, int R, double* phi,
                                     Rows phi_rows, double* part, const int* gate,
                                     cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int nch = features_chunks(d);
  dim3 grid(nch, (R + kFeatTR - 1) / kFeatTR, (M + kFeatFW - 1) / kFeatFW);
  count_launches(2);
  k_feat_partial<T><<<grid, 256, 0, st>>>(A, M, d, S, s_rows, R, part, nch, gate);
  k_feat_finish<<<(R * M + 255) / 256, 256, 0, st>>>(part, nch, R, M, zeta, phi, phi_rows,
                                                     gate);
  return cudaGetLastError();
}

cudaError_t launch_features64(const double* A, const double* zeta, int M, long long d,
                              const double* S, Rows s_rows, int R, double* phi,
                              Rows phi_rows, double* part, const int* gate,
                              cudaStream_t st) {
  return launch_features_t<double>(A, zeta, M, d, S, s_rows, R, phi, phi_rows, part, gate, st);
}

cudaError_t launch_features32(const float* A, const double* zeta, int M, long long d,
                              const float* S, Rows s_rows, int R, double* phi,
                              Rows phi_rows, double* part, const int* gate,
                              cudaStream_t st) {
  return launch_features_t<float>(A, zeta, M, d, S, s_rows, R, phi, phi_rows, part, gate, st);
}

// ---------------------------------------------------------------------------
// Nearest-neighbour distances (App. B): delta_p = sum_j (q_j - S_pj)^2.
// One warp per stored row and chunk (at most 32 chunks per state); chunk
// partials are summed in chunk order by the selection kernel.
// ---------------------------------------------------------------------------
static const int kNnRows = 8;

__host__ __device__ inline long long nn_chunk_len(long long d) {
  long long ch = (d + 31) / 32;
  ch = ((ch + 255) / 256) * 256;
  return ch < 1024 ? 1024 : ch;
}

int nn_chunks(long long d) { return (int)((d + nn_chunk_len(d) - 1) / nn_chunk_len(d)); }

// Chunking of the distance sums for P stored rows: nn_chunks(d) chunks of
// nn_chunk_len(d) while P x chunks stays within the task budget; beyond,
// fewer and longer chunks (about that many tasks, never more chunks than
// nn_chunks(d)), so the selection kernel finishes fewer partials per row.
// The budget is kNnTasks warp tasks per member, half that for states of
// 65536 unknowns or more (the scan then streams from HBM, and longer tasks
// keep more of it in flight per warp).  The partial and the selection
// kernels both derive the chunking from (d, P).
static constexpr int kNnTasks = 8192;
__host__ __device__ inline void nn_split(long long d, int P, long long* chl, int* nch) {
  const long long c0 = nn_chunk_len(d);
  const int n0 = (int)((d + c0 - 1) / c0);
  const int tasks = d >= 65536 ? kNnTasks / 2 : kNnTasks;
  if ((long long)P * n0 <= tasks) {
    *chl = c0;
    *nch = n0;
    return;
  }
  const int want = P < tasks ? tasks / P : 1;
  long long c = (d + want - 1) / want;
  c = ((c + 255) / 256) * 256;
  *chl = c;
  *nch = (int)((d + c - 1) / c);
}

// sum over j in [j0, j1) of (q_j - S_j)^2 by one warp, fixed lane order
template <typename T>
__device__ __forceinline__ T warp_dist(const T* qb, const T* Sp, long long j0, long long j1,
                                       int lane) {
  T acc0 = T(0), acc1 = T(0);
  long long j = j0 + lane;
#pragma unroll 16
  for (; j + 32 < j1; j += 64) {
    const T t0 = qb[j] - Sp[j];
    const T t1 = qb[j + 32] - Sp[j + 32];
    acc0 = fma(t0, t0, acc0);
    acc1 = fma(t1, t1, acc1);
  }
  if (j < j1) {
    const T t0 = qb[j] - Sp[j];
    acc0 = fma(t0, t0, acc0);
  }
  T acc = acc0 + acc1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Partial of member b, stored row p, chunk ch at part[(ch * B + b) * cap + p]
// (chunk-major: the finishing threads, one per stored row, read consecutive
// addresses).  The grid (nch x gy blocks of kNnRows warps per member) does
// not depend on P; with the default chunking block (ch, by) takes chunk ch
// of rows by * kNnRows + warp (stride gy * kNnRows), otherwise the member's
// warps stride over the (row, chunk) tasks of nn_split.
template <typename T>
__device__ __forceinline__ void nn_partial_body(const T* q, const T* S, long long cap,
                                                long long d, long long chl, const int* P,
                                                T* part, int nch, const int* gate,
                                                int ch, int by, int gy, int b, int B) {
  if (gate && !gate[b]) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Pb = P[b];
  const T* qb = q + (long long)b * d;
  long long chl_e;
  int nch_e;
  nn_split(d, Pb, &chl_e, &nch_e);
  if (nch_e == nch) {
    const long long j0 = (long long)ch * chl;
    const long long j1 = (j0 + chl) < d ? j0 + chl : d;
    for (int p = by * kNnRows + warp; p < Pb; p += gy * kNnRows) {
      const T acc = warp_dist<T>(qb, S + ((long long)b * cap + p) * d, j0, j1, lane);
      if (lane == 0) part[((long long)ch * B + b) * cap + p] = acc;
    }
  } else {
    const long long W = (long long)nch * gy * kNnRows;
    const long long ntask = (long long)Pb * nch_e;
    for (long long t = ((long long)by * nch + ch) * kNnRows + warp; t < ntask; t += W) {
      const int p = (int)(t / nch_e);
      const int c = (int)(t - (long long)p * nch_e);
      const long long j0 = (long long)c * chl_e;
      const long long j1 = (j0 + chl_e) < d ? j0 + chl_e : d;
      const T acc = warp_dist<T>(qb, S + ((long long)b * cap + p) * d, j0, j1, lane);
      if (lane == 0) part[((long long)c * B + b) * cap + p] = acc;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_nn_partial(const T* q, const T* S, long long cap,
                                                    long long d, long long chl,
                                                    const int* P, T* part, int nch,
                                                    const int* gate) {
  nn_partial_body<T>(q, S, cap, d, chl, P, part, nch, gate, blockIdx.x, blockIdx.y, gridDim.y,
                     blockIdx.z, gridDim.z);
}

// One launch for both halves of a RandNet query: blocks [0, nfb) compute the
// feature partials of the B query rows (grid nch_f x nry x nwz, flattened),
// the rest the distance partials (grid nch_n x gy x B, flattened).
template <typename T>
__global__ void __launch_bounds__(256) k_query_partials(
    const T* A, int M, long long d, const T* q, Rows qrows, int R, T* fpart, int fnch,
    int nry, int nfb, const T* S, long long cap, long long chl, const int* P, T* npart,
    int nnch, int gy, const int* gate) {
  __shared__ T sS[kFeatTR][kFeatCH];
  int bid = blockIdx.x;
  if (bid < nfb) {
    const int ch = bid % fnch, rest = bid / fnch;
    feat_partial_body<T, T, true>(sS, A, M, d, q, qrows, R, fpart, fnch, gate, ch, rest % nry,
                                  rest / nry);
    return;
  }
  bid -= nfb;
  const int ch = bid % nnch, rest = bid / nnch;
  nn_partial_body<T>(q, S, cap, d, chl, P, npart, nnch, gate, ch, rest % gy, gy, rest / gy, R);
}

template <typename T>
static cudaError_t launch_nn_t(const T* q, const T* S, long long cap, long long d, const int* P,
                               int Pmax, int B, T* part, const int* gate,
                               cudaStream_t st) {
  if (Pmax <= 0 || B <= 0) return cudaSuccess;
  const int nch = nn_chunks(d);
  // Pmax only sizes the grid (rows are strided), so a graph captured with
  // the arena capacity stays valid as the dataset grows
  int gy = (Pmax + kNnRows - 1) / kNnRows;
  if (gy > 32) gy = 32;
  dim3 grid(nch, gy, B);
  count_launches(1);
  k_nn_partial<T><<<grid, 256, 0, st>>>(q, S, cap, d, nn_chunk_len(d), P, part, nch, gate);
  return cudaGetLastError();
}

cudaError_t launch_nn_partial(const double* q, const double* S, long long cap, long long d,
                              const int* P, int Pmax, int B, double* part, const int* gate,
                              cudaStream_t st) {
  return launch_nn_t<double>(q, S, cap, d, P, Pmax, B, part, gate, st);
}

cudaError_t launch_nn_partial32(const float* q, const float* S, long long cap, long long d,
                                const int* P, int Pmax, int B, float* part, const int* gate,
                                cudaStream_t st) {
  return launch_nn_t<float>(q, S, cap, d, P, Pmax, B, part, gate, st);
}

template <typename T>
static cudaError_t launch_query_t(const T* A, int M, long long d, const T* q, int B,
                                  T* fpart, const T* S, long long cap, const int* P,
                                  int Pmax, T* npart, const int* gate, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int fnch = features_chunks(d);
  const int nry = (B + kFeatTR - 1) / kFeatTR, nwz = (M + kFeatFW - 1) / kFeatFW;
  const int nfb = fnch * nry * nwz;
  const int nnch = nn_chunks(d);
  // distance blocks: enough that the whole query fits one wave of resident
  // blocks (rows are strided, so fewer blocks each take more rows); the
  // grid does not depend on the dataset size, so a captured graph stays valid
  static int slots[2] = {0, 0};   // resident blocks on the device, per T
  int& sl = slots[sizeof(T) == 8 ? 1 : 0];
  if (sl == 0) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_query_partials<T>, 256, 0) ==
            cudaSuccess)
      sl = sms * per;
    else
      sl = -1;
    cudaGetLastError();
  }
  int gy = (Pmax + kNnRows - 1) / kNnRows;
  if (gy > 32) gy = 32;
  if (sl > 0) {
    const int fit = (sl - nfb) / (nnch * B);
    if (fit >= 1 && fit < gy) gy = fit;
  }
  if (Pmax <= 0) gy = 0;
  const long long nblocks = (long long)nfb + (long long)nnch * gy * B;
  count_launches(1);
  k_query_partials<T><<<(unsigned)nblocks, 256, 0, st>>>(
      A, M, d, q, Rows{nullptr, 0, d}, B, fpart, fnch, nry, nfb, S, cap, nn_chunk_len(d), P,
      npart, nnch, gy > 0 ? gy : 1, gate);
  return cudaGetLastError();
}

cudaError_t launch_query64(const double* A, int M, long long d, const double* q, int B,
                           double* fpart, const double* S, long long cap, const int* P,
                           int Pmax, double* npart, const int* gate, cudaStream_t st) {
  return launch_query_t<double>(A, M, d, q, B, fpart, S, cap, P, Pmax, npart, gate, st);
}

cudaError_t launch_query32(const float* A, int M, long long d, const float* q, int B,
                           float* fpart, const float* S, long long cap, const int* P,
                           int Pmax, float* npart, const int* gate, cudaStream_t st) {
  return launch_query_t<float>(A, M, d, q, B, fpart, S, cap, P, Pmax, npart, gate, st);
}

// ---------------------------------------------------------------------------
// Top-m selection + dual ridge solve, one CTA per member.
// ---------------------------------------------------------------------------
// Distances are sums of squares (>= 0 or NaN), so their bit patterns order
// like the values and a NaN orders after +inf: the selection compares 64-bit
// integer keys (ties -> lower index).  Minimum of (key, index) over a warp
// with three 32-bit reductions; lanes without a candidate pass key ~0.
__device__ __forceinline__ void warp_min_key(unsigned long long key, unsigned idx,
                                             unsigned long long* okey, unsigned* oidx) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
  *oidx = __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? idx : 0xffffffffu);
  *okey = ((unsigned long long)mhi << 32) | mlo;
}

// Cholesky solve of (K + lam I) x = r for a small system held in registers
// (n <= 4 after unrolling): one reciprocal square root per pivot scales its
// column and both triangular solves.  Returns false on a non-positive pivot.
template <int N>
__device__ __forceinline__ bool chol_small(const double* Kraw, const double* r, double lam,
                                           double* x) {
  double L[N][N], li[N], y[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double s = __dadd_rn(Kraw[j * RNP_MAX_M + j], lam);
#pragma unroll
    for (int k = 0; k < j; ++k) s = __dsub_rn(s, __dmul_rn(L[j][k], L[j][k]));
    if (!(s > 0.0)) return false;
    const double inv = rsqrt(s);
    li[j] = inv;
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      double t = Kraw[i * RNP_MAX_M + j];
#pragma unroll
      for (int k = 0; k < j; ++k) t = __dsub_rn(t, __dmul_rn(L[i][k], L[j][k]));
      L[i][j] = __dmul_rn(t, inv);
    }
    L[j][j] = __dmul_rn(s, inv);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double t = r[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t = __dsub_rn(t, __dmul_rn(L[i][k], y[k]));
    y[i] = __dmul_rn(t, li[i]);
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    double t = y[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) t = __dsub_rn(t, __dmul_rn(L[k][i], x[k]));
    x[i] = __dmul_rn(t, li[i]);
  }
  return true;
}

// The same for any n <= RNP_MAX_M with the factor in shared memory.
__device__ bool chol_general(const double* Kraw, const double* r, double lam, int n, double* L,
                             double* li, double* y, double* x) {
  for (int j = 0; j < n; ++j) {
    double s = __dadd_rn(Kraw[j * RNP_MAX_M + j], lam);
    for (int k = 0; k < j; ++k) s = __dsub_rn(s, __dmul_rn(L[j * RNP_MAX_M + k], L[j * RNP_MAX_M + k]));
    if (!(s > 0.0)) return false;
    const double inv = rsqrt(s);
    li[j] = inv;
    for (int i = j + 1; i < n; ++i) {
      double t = Kraw[i * RNP_MAX_M + j];
      for (int k = 0; k < j; ++k) t = __dsub_rn(t, __dmul_rn(L[i * RNP_MAX_M + k], L[j * RNP_MAX_M + k]));
      L[i * RNP_MAX_M + j] = __dmul_rn(t, inv);
    }
    L[j * RNP_MAX_M + j] = __dmul_rn(s, inv);
  }
  for (int i = 0; i < n; ++i) {
    double t = r[i];
    for (int k = 0; k < i; ++k) t = __dsub_rn(t, __dmul_rn(L[i * RNP_MAX_M + k], y[k]));
    y[i] = __dmul_rn(t, li[i]);
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < n; ++k) t = __dsub_rn(t, __dmul_rn(L[k * RNP_MAX_M + i], x[k]));
    x[i] = __dmul_rn(t, li[i]);
  }
  return true;
}

// TP: type of the chunk partials (double in the FP64 path, float where the
// query was computed in FP32; their sums are kept in TP).
template <typename TP>
__global__ void __launch_bounds__(256) k_topm_ridge(const TP* part, long long d,
                                                    const double* Phi, long long cap, int M,
                                                    double* phiq, long long phiq_bstride,
                                                    const TP* fpart, int fnch,
                                                    const double* zeta, const int* Pn, int m,
                                                    double lambda, double* dist, double* alpha,
                                                    int* idx, int* meff, int* esc_count,
                                                    int* fail, const int* gate) {
  const int b = blockIdx.x;
  if (gate && !gate[b]) return;
  const int P = Pn[b];
  const int me = m < P ? m : P;
  long long chl_unused;
  int nch;                     // chunks of the distance partials (nn_split)
  nn_split(d, P, &chl_unused, &nch);
  constexpr int kWarps = 8;  // blockDim.x == 256
  __shared__ int sel[RNP_MAX_M];
  __shared__ unsigned long long ck[kWarps * RNP_MAX_M];
  __shared__ unsigned ci[kWarps * RNP_MAX_M];
  __shared__ double Kraw[RNP_MAX_M * RNP_MAX_M];
  __shared__ double Lsh[RNP_MAX_M * RNP_MAX_M];
  __shared__ double rhs[RNP_MAX_M], ysh[RNP_MAX_M], xsh[RNP_MAX_M], lish[RNP_MAX_M];
  double* pq = phiq + (long long)b * phiq_bstride;
  // Distances first (their partial loads are issued before the feature
  // partials', so both are in flight together): four interleaved partial
  // sums over the chunks, then combined; two stored rows per iteration
  // (p and p + 256) so that twice the loads are in flight.  Each thread
  // keeps its kTop best (distance key, index) pairs in a sorted register
  // list (insertion by compare-and-swap with static indices; candidates
  // arrive in increasing index, so a strict comparison keeps the lower
  // index first among equal keys).
  constexpr int kTop = 8;
  const bool in_regs = me <= kTop;
  unsigned long long tk[kTop];
  unsigned ti[kTop];
#pragma unroll
  for (int t = 0; t < kTop; ++t) { tk[t] = ~0ULL; ti[t] = 0xffffffffu; }
  auto insert = [&](unsigned long long k, unsigned i) {
#pragma unroll
    for (int t = 0; t < kTop; ++t) {
      const bool lt = k < tk[t];
      const unsigned long long ok = tk[t];
      const unsigned oi = ti[t];
      tk[t] = lt ? k : ok;
      ti[t] = lt ? i : oi;
      k = lt ? ok : k;
      i = lt ? oi : i;
    }
  };
  double* db = dist + (long long)b * cap;
  const int B = gridDim.x;                          // members (one CTA each)
  const long long cstride = (long long)B * cap;     // chunk k of row p at pp[k * cstride]
  if (P <= (int)blockDim.x) {
    // one stored row per thread: its key starts the (otherwise empty) list
    const int p = threadIdx.x;
    if (p < P) {
      const TP* pa = part + (long long)b * cap + p;
      TP a0 = TP(0), a1 = TP(0), a2 = TP(0), a3 = TP(0);
      int k = 0;
#pragma unroll 4
      for (; k + 3 < nch; k += 4) {
        a0 = a0 + pa[k * cstride];
        a1 = a1 + pa[(k + 1) * cstride];
        a2 = a2 + pa[(k + 2) * cstride];
        a3 = a3 + pa[(k + 3) * cstride];
      }
      for (; k < nch; ++k) a0 = a0 + pa[k * cstride];
      const double d0 = (double)((a0 + a1) + (a2 + a3));
      db[p] = d0;
      tk[0] = (unsigned long long)__double_as_longlong(d0);
      ti[0] = (unsigned)p;
    }
  } else {
    for (int p0 = threadIdx.x; p0 < P; p0 += 2 * blockDim.x) {
      const int p1 = p0 + blockDim.x;
      const bool two = p1 < P;
      const TP* pa = part + (long long)b * cap + p0;
      const TP* pb = part + (long long)b * cap + (two ? p1 : p0);
      TP a0 = TP(0), a1 = TP(0), a2 = TP(0), a3 = TP(0);
      TP c0 = TP(0), c1 = TP(0), c2 = TP(0), c3 = TP(0);
      int k = 0;
#pragma unroll 2
      for (; k + 3 < nch; k += 4) {
        a0 = a0 + pa[k * cstride];
        a1 = a1 + pa[(k + 1) * cstride];
        a2 = a2 + pa[(k + 2) * cstride];
        a3 = a3 + pa[(k + 3) * cstride];
        c0 = c0 + pb[k * cstride];
        c1 = c1 + pb[(k + 1) * cstride];
        c2 = c2 + pb[(k + 2) * cstride];
        c3 = c3 + pb[(k + 3) * cstride];
      }
      for (; k < nch; ++k) {
        a0 = a0 + pa[k * cstride];
        c0 = c0 + pb[k * cstride];
      }
      const double d0 = (double)((a0 + a1) + (a2 + a3));
      db[p0] = d0;
      if (in_regs) insert((unsigned long long)__double_as_longlong(d0), (unsigned)p0);
      if (two) {
        const double d1 = (double)((c0 + c1) + (c2 + c3));
        db[p1] = d1;
        if (in_regs) insert((unsigned long long)__double_as_longlong(d1), (unsigned)p1);
      }
    }
  }
  // query features (when their partials are given): the chunk partials in
  // chunk order, + zeta, ReLU
  if (fpart) {
    for (int w = threadIdx.x; w < M; w += blockDim.x) {
      const TP* fp = fpart + (long long)b * M + w;   // chunk k at fp[k * B * M]
      TP acc = TP(0);
#pragma unroll 16
      for (int k = 0; k < fnch; ++k) acc = acc + fp[(long long)k * B * M];
      const double v = (double)acc + zeta[w];
      pq[w] = v > 0.0 ? v : 0.0;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (in_regs) {
    // m nearest from the register lists: each warp takes its me best (the
    // winning lane pops its list head), then warp 0 takes the me best of
    // those
    for (int r = 0; r < me; ++r) {
      unsigned long long wkey;
      unsigned widx;
      warp_min_key(tk[0], ti[0], &wkey, &widx);
      if (widx != 0xffffffffu && ti[0] == widx) {
#pragma unroll
        for (int t = 0; t + 1 < kTop; ++t) { tk[t] = tk[t + 1]; ti[t] = ti[t + 1]; }
        tk[kTop - 1] = ~0ULL;
        ti[kTop - 1] = 0xffffffffu;
      }
      if (lane == 0) { ck[warp * RNP_MAX_M + r] = wkey; ci[warp * RNP_MAX_M + r] = widx; }
    }
  } else {
    // more neighbours than the register lists hold: the same selection
    // reading the distances back, with the warp's picks as the taken list
    __syncthreads();
    for (int r = 0; r < me; ++r) {
      unsigned long long bk = ~0ULL;
      unsigned bi = 0xffffffffu;
      for (int p = threadIdx.x; p < P; p += blockDim.x) {
        bool taken = false;
        for (int k = 0; k < r; ++k) taken |= (ci[warp * RNP_MAX_M + k] == (unsigned)p);
        if (taken) continue;
        const unsigned long long v = (unsigned long long)__double_as_longlong(db[p]);
        if (v < bk || (v == bk && (unsigned)p < bi)) { bk = v; bi = (unsigned)p; }
      }
      unsigned long long wkey;
      unsigned widx;
      warp_min_key(bk, bi, &wkey, &widx);
      if (lane == 0) { ck[warp * RNP_MAX_M + r] = wkey; ci[warp * RNP_MAX_M + r] = widx; }
      __syncwarp();
    }
  }
  __syncthreads();
  if (warp == 0) {
    // the warps' picks, at most RNP_MAX_M per lane slot: lane c holds
    // candidates c, c + 32, ... of the nw * me list; the winner drops its own
    const int nc = kWarps * me;
    unsigned long long lk[kWarps];
    unsigned li2[kWarps];
#pragma unroll
    for (int t = 0; t < kWarps; ++t) {
      const int c = lane + 32 * t;
      if (c < nc) {
        const int w = c / me, k = c - w * me;
        lk[t] = ck[w * RNP_MAX_M + k];
        li2[t] = ci[w * RNP_MAX_M + k];
        if (li2[t] == 0xffffffffu) lk[t] = ~0ULL;
      } else {
        lk[t] = ~0ULL;
        li2[t] = 0xffffffffu;
      }
    }
    for (int r = 0; r < me; ++r) {
      unsigned long long bk = ~0ULL;
      unsigned bi = 0xffffffffu;
      int bt = -1;
#pragma unroll
      for (int t = 0; t < kWarps; ++t)
        if (lk[t] != ~0ULL && (lk[t] < bk || (lk[t] == bk && li2[t] < bi))) {
          bk = lk[t]; bi = li2[t]; bt = t;
        }
      unsigned long long wkey;
      unsigned widx;
      warp_min_key(bk, bi, &wkey, &widx);
      if (bt >= 0 && bi == widx) {
#pragma unroll
        for (int t = 0; t < kWarps; ++t)
          if (t == bt) lk[t] = ~0ULL;
      }
      if (lane == 0) sel[r] = (int)widx;
    }
  }
  __syncthreads();
  // Gram entries K[i][j] = sum_w X_i,w X_j,w (i >= j) and rhs_i = X_i . phi_q:
  // one warp per entry, lanes stride w, fixed butterfly reduction.
  const double* X = Phi + (long long)b * cap * M;
  const int nK = me * (me + 1) / 2;
  for (int t = warp; t < nK + me; t += kWarps) {
    const double *xa, *xb;
    int i, j = -1;
    if (t < nK) {
      i = 0;
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      j = t - i * (i + 1) / 2;
      xa = X + (long long)sel[i] * M;
      xb = X + (long long)sel[j] * M;
    } else {
      i = t - nK;
      xa = X + (long long)sel[i] * M;
      xb = pq;
    }
    double acc = 0.0;
#pragma unroll 4
    for (int w = lane; w < M; w += 32) acc = fma(xa[w], xb[w], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (j >= 0) Kraw[i * RNP_MAX_M + j] = acc;
      else rhs[i] = acc;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  meff[b] = me;
  for (int l = 0; l < me; ++l) idx[b * RNP_MAX_M + l] = sel[l];
  if (me == 0) return;
  // Cholesky of K + lambda I; lambda x10 on a non-positive pivot
  double lam = lambda;
  double x[4];
  bool ok = false;
  int tries = 0;
  for (tries = 0; tries <= 4 && !ok; ++tries) {
    switch (me) {
      case 1: ok = chol_small<1>(Kraw, rhs, lam, x); break;
      case 2: ok = chol_small<2>(Kraw, rhs, lam, x); break;
      case 3: ok = chol_small<3>(Kraw, rhs, lam, x); break;
      case 4: ok = chol_small<4>(Kraw, rhs, lam, x); break;
      default: ok = chol_general(Kraw, rhs, lam, me, Lsh, lish, ysh, xsh);
    }
    if (!ok) lam = __dmul_rn(lam, 10.0);
  }
  if (!ok) {
    atomicExch(fail, 1);
    for (int l = 0; l < me; ++l) alpha[b * RNP_MAX_M + l] = 0.0;
    return;
  }
  if (tries - 1 > 0) atomicAdd(esc_count, tries - 1);
  if (me <= 4) {
#pragma unroll
    for (int l = 0; l < 4; ++l)
      if (l < me) alpha[b * RNP_MAX_M + l] = x[l];
  } else {
    for (int l = 0; l < me; ++l) alpha[b * RNP_MAX_M + l] = xsh[l];
  }
}

template <typename TP>
static cudaError_t launch_topm_t(const TP* part, long long d, const double* Phi, long long cap,
                                 int M, double* phiq, long long phiq_bstride, const TP* fpart,
                                 int fnch, const double* zeta, const int* P, int B, int m,
                                 double lambda, double* dist, double* alpha, int* idx,
                                 int* meff, int* esc_count, int* fail, const int* gate,
                                 cudaStream_t st) {
  count_launches(1);
  k_topm_ridge<TP><<<B, 256, 0, st>>>(part, d, Phi, cap, M, phiq, phiq_bstride, fpart, fnch,
                                      zeta, P, m, lambda, dist, alpha, idx, meff, esc_count,
                                      fail, gate);
  return cudaGetLastError();
}

cudaError_t launch_topm_ridge(const double* part, long long d, const double* Phi, long long cap,
                              int M, double* phiq, long long phiq_bstride, const double* fpart,
                              int fnch, const double* zeta, const int* P, int Pmax, int B,
                              int m, double lambda, double* dist, double* alpha, int* idx,
                              int* meff, int* esc_count, int* fail, const int* gate,
                              cudaStream_t st) {
  (void)Pmax;
  return launch_topm_t<double>(part, d, Phi, cap, M, phiq, phiq_bstride, fpart, fnch, zeta, P,
                               B, m, lambda, dist, alpha, idx, meff, esc_count, fail, gate, st);
}

cudaError_t launch_topm_ridge32(const float* part, long long d, const double* Phi, long long cap,
                                int M, double* phiq, long long phiq_bstride, const float* fpart,
                                int fnch, const double* zeta, const int* P, int Pmax, int B,
                                int m, double lambda, double* dist, double* alpha, int* idx,
                                int* meff, int* esc_count, int* fail, const int* gate,
                                cudaStream_t st) {
  (void)Pmax;
  return launch_topm_t<float>(part, d, Phi, cap, M, phiq, phiq_bstride, fpart, fnch, zeta, P,
                              B, m, lambda, dist, alpha, idx, meff, esc_count, fail, gate, st);
}

// ---------------------------------------------------------------------------
// Update of Eq. 3 with the max-norm of Eq. 5 fused in.
// ---------------------------------------------------------------------------
// Block maximum of non-negative doubles (or NaN) given as their bit
// patterns, which order like the values; one atomicMax per block.
__device__ __forceinline__ void block_max_to(unsigned long long* dst, unsigned long long v) {
  __shared__ unsigned long long red[32];
  const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32));
  const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32) == hi ? (unsigned)v : 0u);
  v = ((unsigned long long)hi << 32) | lo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long x = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) x = red[k] > x ? red[k] : x;
    atomicMax(dst, x);
  }
}

// FAST (mixed-precision contexts, whose next query is kept in FP32 only):
// the correction by fused multiply-adds and the scaled query by the
// reciprocal of the range; otherwise every operation rounded separately, as
// the oracle's Eq. 3 update and scaling do.  (GB300's FP64 pipe makes the
// separate operations and the division the kernel's cost.)
template <bool FAST>
__global__ void __launch_bounds__(256) k_update(const double* g, long long g_bstride,
                                                const double* Y, long long cap, long long d,
                                                const double* alpha, const int* idx,
                                                const int* meff, double* out,
                                                long long out_bstride, unsigned long long* err,
                                                long long err_bstride, int* nonfinite,
                                                const int* gate, QueryOut qo) {
  const int b = blockIdx.y;
  if (gate && !gate[b]) return;
  const int me = meff[b];
  __shared__ double a[RNP_MAX_M];
  __shared__ const double* Yl[RNP_MAX_M];
  __shared__ double rinv[3];
  if (threadIdx.x < me) {
    a[threadIdx.x] = alpha[b * RNP_MAX_M + threadIdx.x];
    Yl[threadIdx.x] = Y + ((long long)b * cap + idx[b * RNP_MAX_M + threadIdx.x]) * d;
  }
  if (FAST && qo.q32 && threadIdx.x >= 32 && threadIdx.x < 35)
    rinv[threadIdx.x - 32] = 1.0 / qo.r[b * 3 + threadIdx.x - 32];
  __syncthreads();
  const double* gb = g ? g + (long long)b * g_bstride : nullptr;
  double* ob = out + (long long)b * out_bstride;
  unsigned long long emax = 0ULL;  // bits of a non-negative double
  bool bad = false;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < d;
       j += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if constexpr (FAST) {
      for (int l = 0; l < me; ++l) acc = fma(a[l], Yl[l][j], acc);
    } else {
      for (int l = 0; l < me; ++l) acc = __dadd_rn(acc, __dmul_rn(a[l], Yl[l][j]));
    }
    const double v = gb ? __dadd_rn(gb[j], acc) : acc;
    if (err) {
      const unsigned long long e = (unsigned long long)__double_as_longlong(fabs(v - ob[j]));
      emax = e > emax ? e : emax;
    }
    bad |= !isfinite(v);
    ob[j] = v;
    if (qo.q64 || qo.q32) {
      // the next step's scaled query, as k_scale_rows computes it (FAST:
      // times the reciprocal); component q of at most three
      const int q = j >= qo.n ? (j >= 2 * qo.n ? 2 : 1) : 0;
      if constexpr (FAST) {
        qo.q32[(long long)b * d + j] = (float)(__dsub_rn(v, qo.c[b * 3 + q]) * rinv[q]);
      } else {
        const double sv = __ddiv_rn(__dsub_rn(v, qo.c[b * 3 + q]), qo.r[b * 3 + q]);
        if (qo.q64) qo.q64[(long long)b * d + j] = sv;
        if (qo.q32) qo.q32[(long long)b * d + j] = (float)sv;
      }
    }
  }
  if (bad) atomicExch(nonfinite, 1);
  if (err) block_max_to(err + (long long)b * err_bstride, emax);
}

__global__ void __launch_bounds__(256) k_update_para(const double* g, long long g_bstride,
                                                     const double* Yv, long long yv_bstride,
                                                     long long d, double* out,
                                                     long long out_bstride,
                                                     unsigned long long* err,
                                                     long long err_bstride, int* nonfinite,
                                                     const int* gate) {
  const int b = blockIdx.y;
  if (gate && !gate[b]) return;
  const double* gb = g + (long long)b * g_bstride;
  const double* yb = Yv + (long long)b * yv_bstride;
  double* ob = out + (long long)b * out_bstride;
  unsigned long long emax = 0ULL;  // bits of a non-negative double
  bool bad = false;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < d;
       j += (long long)gridDim.x * blockDim.x) {
    const double v = __dadd_rn(gb[j], yb[j]);
    if (err) {
      const unsigned long long e = (unsigned long long)__double_as_longlong(fabs(v - ob[j]));
      emax = e > emax ? e : emax;
    }
    bad |= !isfinite(v);
    ob[j] = v;
  }
  if (bad) atomicExch(nonfinite, 1);
  if (err) block_max_to(err + (long long)b * err_bstride, emax);
}

static dim3 update_grid(long long d, int B) {
  long long bx = (d + 255) / 256;
  if (bx > 1024) bx = 1024;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, B);
}

cudaError_t launch_update(const double* g, long long g_bstride, const double* Y,
                          long long cap, long long d, const double* alpha, const int* idx,
                          const int* meff, double* out, long long out_bstride,
                          unsigned long long* err, long long err_bstride, int* nonfinite,
                          int B, const int* gate, cudaStream_t st, QueryOut qo) {
  count_launches(1);
  if (qo.q32 && !qo.q64)
    k_update<true><<<update_grid(d, B), 256, 0, st>>>(g, g_bstride, Y, cap, d, alpha, idx, meff,
                                                      out, out_bstride, err, err_bstride,
                                                      nonfinite, gate, qo);
  else
    k_update<false><<<update_grid(d, B), 256, 0, st>>>(g, g_bstride, Y, cap, d, alpha, idx, meff,
                                                       out, out_bstride, err, err_bstride,
                                                       nonfinite, gate, qo);
  return cudaGetLastError();
}

cudaError_t launch_update_para(const double* g, long long g_bstride, const double* Yv,
                               long long yv_bstride, long long d, double* out,
                               long long out_bstride, unsigned long long* err,
                               long long err_bstride, int* nonfinite, int B, const int* gate,
                               cudaStream_t st) {
  count_launches(1);
  k_update_para<<<update_grid(d, B), 256, 0, st>>>(g, g_bstride, Yv, yv_bstride, d, out,
                                                   out_bstride, err, err_bstride, nonfinite,
                                                   gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dataset append (Eq. 6) and row copies
// ---------------------------------------------------------------------------
__global__ void k_append(const double* U, long long u_bstride, const double* Fv,
                         const double* Gc, long long n_bstride, double* Yv, double* Sds,
                         float* S32, double* Yds, long long cap, const double* c,
                         const double* r, AppendItems it, bool randnet, long long n,
                         long long d) {
  const long long tot = (long long)it.n * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t / d);
    const long long e = t - (long long)w * d;
    const int b = it.b[w], j = it.j[w];
    const long long ns = (long long)b * n_bstride + (long long)j * d + e;
    const double y = __dsub_rn(Fv[ns], Gc[ns]);
    Yv[ns] = y;
    if (randnet) {
      const long long ds = ((long long)b * cap + it.p[w]) * d + e;
      Yds[ds] = y;
      const int q = (int)(e / n);
      const double u = U[(long long)b * u_bstride + (long long)j * d + e];
      const double v = __ddiv_rn(__dsub_rn(u, c[b * 3 + q]), r[b * 3 + q]);
      if (Sds) Sds[ds] = v;
      if (S32) S32[ds] = (float)v;
    }
  }
}

cudaError_t launch_append(const Geom& g, const double* U, long long u_bstride, const double* Fv,
                          const double* Gc, long long n_bstride, double* Yv, double* Sds,
                          float* S32, double* Yds, long long cap, const double* c,
                          const double* r, const AppendItems& it, bool randnet,
                          cudaStream_t st) {
  if (it.n <= 0) return cudaSuccess;
  count_launches(1);
  k_append<<<grid_cap((long long)it.n * g.d, 256), 256, 0, st>>>(
      U, u_bstride, Fv, Gc, n_bstride, Yv, Sds, S32, Yds, cap, c, r, it, randnet, g.n, g.d);
  return cudaGetLastError();
}

__global__ void k_copy_phi(const double* src, long long src_bstride, double* dst,
                           long long cap, int M, AppendItems it) {
  const long long tot = (long long)it.n * M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t / M);
    const int k = (int)(t - (long long)w * M);
    const int b = it.b[w];
    dst[((long long)b * cap + it.p[w]) * M + k] =
        src[(long long)b * src_bstride + (long long)it.j[w] * M + k];
  }
}

cudaError_t launch_copy_phi(const double* src, long long src_bstride, double* dst,
                            long long cap, int M, const AppendItems& it, cudaStream_t st) {
  if (it.n <= 0) return cudaSuccess;
  count_launches(1);
  k_copy_phi<<<grid_cap((long long)it.n * M, 256), 256, 0, st>>>(src, src_bstride, dst, cap, M,
                                                                it);
  return cudaGetLastError();
}

__global__ void k_copy_rows(const double* src, const long long* src_off, double* dst,
                            const long long* dst_off, long long d, int rows) {
  const long long tot = (long long)rows * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t / d);
    const long long e = t - (long long)w * d;
    dst[dst_off[w] + e] = src[src_off[w] + e];
  }
}

cudaError_t launch_copy_rows(const double* src, const long long* src_off, double* dst,
                             const long long* dst_off, long long d, int rows, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  count_launches(1);
  k_copy_rows<<<grid_cap((long long)rows * d, 256), 256, 0, st>>>(src, src_off, dst, dst_off, d,
                                                                 rows);
  return cudaGetLastError();
}

// Segment s: dst[off[s] .. off[s] + len[s]) = src[same range].  Used to
// write states into pinned host memory through its device address: SM
// stores keep many address translations of the destination in flight at
// once, where the copy engine takes them a few at a time.
__global__ void k_copy_segments(const double* __restrict__ src, double* __restrict__ dst,
                                Segments sg) {
  const int s = blockIdx.y;
  const long long off = sg.off[s], len = sg.len[s];
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < len;
       j += (long long)gridDim.x * blockDim.x)
    dst[off + j] = src[off + j];
}

cudaError_t launch_copy_segments(const double* src, double* dst, const Segments& sg,
                                 cudaStream_t st) {
  if (sg.n <= 0) return cudaSuccess;
  long long lmax = 0;
  for (int s = 0; s < sg.n; ++s) lmax = sg.len[s] > lmax ? sg.len[s] : lmax;
  if (lmax <= 0) return cudaSuccess;
  // about 16 blocks of 512 threads per SM over all segments
  const int bx = grid_cap(lmax, 512, (152 * 16 + sg.n - 1) / sg.n);
  count_launches(1);
  k_copy_segments<<<dim3(bx, sg.n), 512, 0, st>>>(src, dst, sg);
  return cudaGetLastError();
}

}  // namespace rnp
