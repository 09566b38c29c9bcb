// features_tc.cu -- the random-feature map of Eq. HA, phi = ReLU(A s + zeta),
// for many rows at once on the 5th-generation tensor cores (tcgen05), with
// BF16 operands and FP32 accumulation in tensor memory.
//
//   C[R x M] = S[R x d] . A[M x d]^T     (both operands K-major: d contiguous)
//
// One CTA computes a 128-row x 128-neuron tile over one chunk of the
// reduction dimension d (deterministic split-K): its 4 warps convert the FP32
// scaled rows and copy the BF16 weights into 128-byte-swizzled shared memory
// (the canonical K-major layout of the tensor core), one thread issues
// tcgen05.mma for each 16-wide K step and commits to an mbarrier, and after
// the chunk the accumulator is read from tensor memory with tcgen05.ld and
// written as FP32 partials.  A second kernel sums the partials in chunk order
// (FP64), adds zeta and applies ReLU.  Every wait on the mbarrier is bounded:
// on timeout the CTA records an error flag and skips the rest of its work
// (after waiting, again boundedly, for its own MMAs to drain) instead of
// hanging.
//
// Single queries (one row per member) use k_feat_bf16_gemv below: CUDA cores
// on the same BF16-rounded operands with FP32 accumulation, so that every row
// of the dataset and every query see the same feature map.
#include <cuda_bf16.h>

#include <cstdint>

#include "rnp_internal.h"

namespace rnp {

static const int kTcM = 128;      // rows per tile (tcgen05 M)
static const int kTcN = 128;      // neurons per tile (tcgen05 N); M <= 128
static const int kTcKB = 64;      // K elements per shared-memory block (128 B of BF16)
static const int kTcChunk = 256;  // K elements per CTA (split-K chunk)
// Bound of a wait on the MMA-commit mbarrier: kPolls polls of at most
// kPollNs suspension each.
static const unsigned kPollNs = 1000;
static const unsigned kPolls = 2u << 20;

int features_tc_chunks(long long d) { return (int)((d + kTcChunk - 1) / kTcChunk); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): K-major, 128-byte swizzle,
// 8-row core groups 1024 B apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused)
  d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset
  d |= (uint64_t)1 << 46;                            // descriptor version
  d |= (uint64_t)2 << 61;                            // SWIZZLE_128B
  return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulator,
// both K-major, shape M x N.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
  return (1u << 4)                       // D format: F32
         | (1u << 7)                     // A format: BF16
         | (1u << 10)                    // B format: BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// Byte offset of element (row r, k) of a K-major, 128-byte-swizzled tile
// whose rows hold kTcKB BF16 values: 16-byte chunk c of row r is stored at
// chunk c ^ (r % 8) of that row; rows are 128 B apart.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
  const int chunk = (k * 2) >> 4;
  return (uint32_t)(r * 128 + ((chunk ^ (r & 7)) << 4) + ((k * 2) & 15));
}

// Polls until the phase completes; every poll may suspend the thread for at
// most kPollNs (the suspend-time hint), so kPolls polls bound the wait at
// about 2 s.  Returns false when the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned it = 0; it < kPolls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity), "r"(kPollNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Stages K-block [kb, kb + kTcKB) of the S tile (rows r0.., FP32 -> BF16)
// and of the A tile (neurons 0.., BF16) into the 128-byte-swizzled K-major
// buffers sA / sB, zero-padded beyond R, M and d.
//  * A: each 16-byte swizzle chunk (8 BF16) is copied global -> shared by
//    cp.async without passing through registers (zero-filled beyond M);
//    element copies where d does not allow 16-byte chunks.  The caller
//    waits for the copies (tc_stage_wait) before the tile is used.
//  * S: all of the thread's 16-byte loads (4 FP32 values each) are issued
//    before any is converted, so they are in flight together; each becomes
//    an 8-byte half chunk of BF16.  Element loads where the row start or d
//    do not allow 16-byte loads.
__device__ __forceinline__ void tc_stage(const float* S, Rows rows, int R,
                                         const __nv_bfloat16* A, int M, long long d, int r0,
                                         long long kb, unsigned char* sA, unsigned char* sB,
                                         int tid) {
  constexpr int kAPer = kTcN * (kTcKB / 8) / 128;   // 8 chunks per thread
#pragma unroll
  for (int i = 0; i < kAPer; ++i) {
    const int e = tid + i * 128;
    const int w = e >> 3, kk = (e & 7) * 8;
    unsigned char* dst = sB + sw128_offset(w, kk);
    if ((d & 7) == 0 && kb + kk + 8 <= d) {
      const __nv_bfloat16* src = A + (long long)(w < M ? w : 0) * d + kb + kk;
      const uint32_t n = w < M ? 16u : 0u;   // 0: zero fill
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                   "l"(src), "r"(n)
                   : "memory");
    } else {
      __nv_bfloat16 t[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        t[j] = (w < M && kb + kk + j < d) ? A[(long long)w * d + kb + kk + j]
                                          : __float2bfloat16(0.f);
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(t);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  constexpr int kSPer = kTcM * (kTcKB / 4) / 128;   // 16 groups of 4 per thread
  float4 v[kSPer];
#pragma unroll
  for (int i = 0; i < kSPer; ++i) {
    const int e = tid + i * 128;
    const int r = e >> 4, kk = (e & 15) * 4;
    const int row = r0 + r;
    v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < R) {
      const long long off = item_off(rows.off, rows.base, rows.stride, row);
      const float* src = S + off + kb + kk;
      if (((off | d) & 3) == 0 && kb + kk + 4 <= d) {
        v[i] = *reinterpret_cast<const float4*>(src);
      } else {
        if (kb + kk + 0 < d) v[i].x = src[0];
        if (kb + kk + 1 < d) v[i].y = src[1];
        if (kb + kk + 2 < d) v[i].z = src[2];
        if (kb + kk + 3 < d) v[i].w = src[3];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kSPer; ++i) {
    const int e = tid + i * 128;
    const int r = e >> 4, kk = (e & 15) * 4;
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v[i].x, v[i].y);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(v[i].z, v[i].w);
    uint2 pk2;
    pk2.x = *reinterpret_cast<const uint32_t*>(&lo);
    pk2.y = *reinterpret_cast<const uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(sA + sw128_offset(r, kk)) = pk2;
  }
}

// Waits for this thread's cp.async copies of the last staged tile.
__device__ __forceinline__ void tc_stage_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// One CTA: the 128-row x 128-neuron tile of rows r0.. over the K chunk
// [k0, k0 + chunk).  Two operand stages: while the tensor core runs the MMAs
// of K-block j (from stage j & 1), the threads load K-block j + 1 into the
// other stage; a stage is refilled only after the commit of the MMAs that
// read it (mbarrier j & 1, one phase per use).
__global__ void __launch_bounds__(128, 1) k_feat_tc(const float* S, Rows rows, int R,
                                                    const __nv_bfloat16* A, int M, long long d,
                                                    int chunk_len, float* part, int nchunk,
                                                    int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned operand stages: [stage][S tile 16 KB | A tile 16 KB]
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int kStage = (kTcM + kTcN) * kTcKB * 2;   // 32 KB
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int aborted;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int chunk = blockIdx.x;
  const int r0 = blockIdx.y * kTcM;
  const long long k0 = (long long)chunk * chunk_len;
  const long long k1 = (k0 + chunk_len) < d ? k0 + chunk_len : d;
  const int nblk = (int)((k1 - k0 + kTcKB - 1) / kTcKB);
  const uint32_t mb[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};

  if (tid == 0) {
    aborted = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb[0]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb[1]) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // 128 columns of tensor memory: the 128 x 128 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = bf16_idesc(kTcM, kTcN);

  if (nblk > 0) tc_stage(S, rows, R, A, M, d, r0, k0, base, base + kTcM * kTcKB * 2, tid);
  int done = 0;   // K-blocks whose MMAs are known complete
  for (int j = 0; j < nblk; ++j) {
    unsigned char* sA = base + (j & 1) * kStage;
    unsigned char* sB = sA + kTcM * kTcKB * 2;
    // make this thread's copies and generic-proxy writes of stage j & 1
    // visible to the tensor core
    tc_stage_wait();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (aborted) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = sw128_desc(smem_u32(sA)), db = sw128_desc(smem_u32(sB));
#pragma unroll
      for (int ks = 0; ks < kTcKB / 16; ++ks) {
        // advance 16 BF16 (32 B) along K inside the swizzled rows
        const uint64_t a = da + (uint64_t)((ks * 32) >> 4);
        const uint64_t b = db + (uint64_t)((ks * 32) >> 4);
        const uint32_t acc = (j > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mb[j & 1])
          : "memory");
    }
    if (j + 1 < nblk) {
      // stage (j + 1) & 1 was last read by the MMAs of block j - 1
      if (j >= 1) {
        if (!mbar_wait(mb[(j + 1) & 1], (uint32_t)(((j - 1) >> 1) & 1))) {
          if (tid == 0) { atomicExch(err, 1); aborted = 1; }
        } else {
          done = j;
        }
      }
      __syncthreads();
      if (aborted) break;
      unsigned char* nA = base + ((j + 1) & 1) * kStage;
      tc_stage(S, rows, R, A, M, d, r0, k0 + (long long)(j + 1) * kTcKB, nA,
               nA + kTcM * kTcKB * 2, tid);
    }
  }
  // every MMA of this CTA complete (the commits of the last one or two
  // blocks not yet waited for), bounded; on a timeout the accumulator is
  // not read
  for (int j = done; j < nblk; ++j)
    if (!mbar_wait(mb[j & 1], (uint32_t)((j >> 1) & 1)) && tid == 0) {
      atomicExch(err, 1);
      aborted = 1;
    }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!aborted && nblk > 0) {
    // warp w owns tensor-memory lanes 32w .. 32w + 31 = tile rows
    const int r = warp * 32 + (tid & 31);
    const int row = r0 + r;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < kTcN; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < R) {
        float* dst = part + ((long long)row * nchunk + chunk) * kTcN + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < M) dst[j] = __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

__global__ void k_feat_tc_finish(const float* part, int nchunk, int R, int M,
                                 const double* zeta, double* phi, Rows prow) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * M) return;
  const int row = t / M, w = t - row * M;
  double acc = 0.0;
  for (int c = 0; c < nchunk; ++c) acc += (double)part[((long long)row * nchunk + c) * kTcN + w];
  const double v = acc + zeta[w];
  phi[item_off(prow.off, prow.base, prow.stride, row) + w] = v > 0.0 ? v : 0.0;
}

size_t features_tc_part_floats(int R, long long d) {
  return (size_t)R * features_tc_chunks(d) * kTcN;
}

// K-chunk length of one CTA: the longest multiple of kTcChunk (up to 8 x)
// that still gives about two CTAs per SM over the row tiles, so that long
// reductions pipeline their loads while small ones still fill the GPU.
static int tc_chunk_len(int R, long long d) {
  const long long tiles = (R + kTcM - 1) / kTcM;
  int len = kTcChunk;
  while (len < 8 * kTcChunk && tiles * ((d + 2 * len - 1) / (2 * len)) >= 2 * 152) len *= 2;
  return len;
}

cudaError_t launch_features_tc(const __nv_bfloat16* A, const double* zeta, int M, long long d,
                               const float* S, Rows s_rows, int R, double* phi, Rows phi_rows,
                               float* part, int* err, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  if (M > kTcN) return cudaErrorInvalidValue;
  const int len = tc_chunk_len(R, d);
  const int nch = (int)((d + len - 1) / len);   // <= features_tc_chunks(d)
  // two 32 KB operand stages plus alignment: at most three CTAs (3 x 128
  // tensor-memory columns of the SM's 512) resident per SM
  const size_t smem = 2 * (kTcM + kTcN) * kTcKB * 2 + 1024;
  cudaError_t e = cudaFuncSetAttribute((const void*)k_feat_tc,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(nch, (R + kTcM - 1) / kTcM);
  count_launches(2);
  k_feat_tc<<<grid, 128, smem, st>>>(S, s_rows, R, A, M, d, len, part, nch, err);
  k_feat_tc_finish<<<(R * M + 255) / 256, 256, 0, st>>>(part, nch, R, M, zeta, phi, phi_rows);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single queries on CUDA cores with the same BF16 operands (FP32 accumulate)
// ---------------------------------------------------------------------------
static const int kBfCH = 1024;
static const int kBfFW = 16;

int features_bf16_chunks(long long d) { return (int)((d + kBfCH - 1) / kBfCH); }

__global__ void __launch_bounds__(256) k_feat_bf16_gemv(const __nv_bfloat16* A, int M,
                                                        long long d, const float* S, Rows rows,
                                                        int R, double* part, int nch,
                                                        const int* gate) {
  __shared__ float sS[kBfCH];
  const int row = blockIdx.y;
  if (row >= R || (gate && !gate[row])) return;
  const int ch = blockIdx.x, w0 = blockIdx.z * kBfFW;
  const long long j0 = (long long)ch * kBfCH;
  const int len = (int)((d - j0) < kBfCH ? (d - j0) : kBfCH);
  const float* src = S + item_off(rows.off, rows.base, rows.stride, row) + j0;
  for (int j = threadIdx.x; j < kBfCH; j += blockDim.x)
    sS[j] = j < len ? __bfloat162float(__float2bfloat16_rn(src[j])) : 0.f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = w0 + warp; w < M && w < w0 + kBfFW; w += 8) {
    const __nv_bfloat16* Aw = A + (long long)w * d + j0;
    float acc = 0.f;
    for (int j = lane; j < len; j += 32) acc = fmaf(__bfloat162float(Aw[j]), sS[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[((long long)row * M + w) * nch + ch] = (double)acc;
  }
}

__global__ void k_feat_bf16_finish(const double* part, int nch, int R, int M, const double* zeta,
                                   double* phi, Rows prow, const int* gate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * M) return;
  const int row = t / M, w = t - row * M;
  if (gate && !gate[row]) return;
  double acc = 0.0;
  for (int k = 0; k < nch; ++k) acc += part[(long long)t * nch + k];
  const double v = acc + zeta[w];
  phi[item_off(prow.off, prow.base, prow.stride, row) + w] = v > 0.0 ? v : 0.0;
}

cudaError_t launch_features_bf16(const __nv_bfloat16* A, const double* zeta, int M, long long d,
                                 const float* S, Rows s_rows, int R, double* phi, Rows phi_rows,
                                 double* part, const int* gate, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int nch = features_bf16_chunks(d);
  dim3 grid(nch, R, (M + kBfFW - 1) / kBfFW);
  count_launches(2);
  k_feat_bf16_gemv<<<grid, 256, 0, st>>>(A, M, d, S, s_rows, R, part, nch, gate);
  k_feat_bf16_finish<<<(R * M + 255) / 256, 256, 0, st>>>(part, nch, R, M, zeta, phi, phi_rows,
                                                          gate);
  return cudaGetLastError();
}

}  // namespace rnp
