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

__global__ void __launch_bounds__(128, 1) k_feat_tc(const float* S, Rows rows, int R,
                                                    const __nv_bfloat16* A, int M, long long d,
                                                    float* part, int nchunk, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned operand tiles: S tile (128 x 64 BF16) then A tile
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                       // 16 KB
  unsigned char* sB = base + kTcM * kTcKB * 2;    // 16 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int aborted;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int chunk = blockIdx.x;
  const int r0 = blockIdx.y * kTcM;
  const long long k0 = (long long)chunk * kTcChunk;
  const long long k1 = (k0 + kTcChunk) < d ? k0 + kTcChunk : d;
  const uint32_t mbar_a = smem_u32(&mbar);

  if (tid == 0) {
    aborted = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
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

  uint32_t phase = 0;
  int nblk = 0;
  for (long long kb = k0; kb < k1; kb += kTcKB, ++nblk) {
    // stage: S rows (FP32 -> BF16) and A rows (BF16), zero-padded
    for (int e = tid; e < kTcM * (kTcKB / 2); e += blockDim.x) {
      const int r = e / (kTcKB / 2), kk = (e % (kTcKB / 2)) * 2;
      const int row = r0 + r;
      float v0 = 0.f, v1 = 0.f;
      if (row < R) {
        const float* src = S + item_off(rows.off, rows.base, rows.stride, row);
        if (kb + kk < d) v0 = src[kb + kk];
        if (kb + kk + 1 < d) v1 = src[kb + kk + 1];
      }
      *reinterpret_cast<__nv_bfloat162*>(sA + sw128_offset(r, kk)) = __floats2bfloat162_rn(v0, v1);
    }
    for (int e = tid; e < kTcN * (kTcKB / 2); e += blockDim.x) {
      const int w = e / (kTcKB / 2), kk = (e % (kTcKB / 2)) * 2;
      __nv_bfloat162 v = __floats2bfloat162_rn(0.f, 0.f);
      if (w < M) {
        const __nv_bfloat16* src = A + (long long)w * d;
        __nv_bfloat16 a0 = kb + kk < d ? src[kb + kk] : __float2bfloat16(0.f);
        __nv_bfloat16 a1 = kb + kk + 1 < d ? src[kb + kk + 1] : __float2bfloat16(0.f);
        v = __halves2bfloat162(a0, a1);
      }
      *reinterpret_cast<__nv_bfloat162*>(sB + sw128_offset(w, kk)) = v;
    }
    // make the generic-proxy writes visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = sw128_desc(smem_u32(sA)), db = sw128_desc(smem_u32(sB));
#pragma unroll
      for (int ks = 0; ks < kTcKB / 16; ++ks) {
        // advance 16 BF16 (32 B) along K inside the swizzled rows
        const uint64_t a = da + (uint64_t)((ks * 32) >> 4);
        const uint64_t b = db + (uint64_t)((ks * 32) >> 4);
        const uint32_t acc = (nblk > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mbar_a)
          : "memory");
    }
    // the staging buffers are reused: wait until these MMAs have read them
    if (!mbar_wait(mbar_a, phase)) {
      if (tid == 0) { atomicExch(err, 1); aborted = 1; }
    }
    __syncthreads();
    if (aborted) {
      // give the MMAs already issued one more bounded chance to finish before
      // the tensor memory they write is released
      mbar_wait(mbar_a, phase);
      break;
    }
    phase ^= 1;
  }
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

cudaError_t launch_features_tc(const __nv_bfloat16* A, const double* zeta, int M, long long d,
                               const float* S, Rows s_rows, int R, double* phi, Rows phi_rows,
                               float* part, int* err, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  if (M > kTcN) return cudaErrorInvalidValue;
  const int nch = features_tc_chunks(d);
  // operand tiles need 33 KB; asking for 50 KB keeps at most four CTAs (4 x
  // 128 tensor-memory columns = the SM's 512) resident per SM
  const size_t smem = 50 * 1024;
  cudaError_t e = cudaFuncSetAttribute((const void*)k_feat_tc,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(nch, (R + kTcM - 1) / kTcM);
  count_launches(2);
  k_feat_tc<<<grid, 128, smem, st>>>(S, s_rows, R, A, M, d, part, nch, err);
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
