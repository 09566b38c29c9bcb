// stencil_impl.cuh -- device code of the fine/coarse propagators (Sec. 2)
// over the right-hand sides h(u) of Eq. 1: arithmetic policy, right-hand
// sides, the fused cluster-resident kernel and the plain per-stage kernel.
// Included by one small translation unit per PDE (stencil_<pde>.cu) so that
// the instantiations compile in parallel; the host side is in stencil.cu.
#pragma once

#include <cooperative_groups.h>

#include "rnp_internal.h"

namespace cg = cooperative_groups;

namespace rnp {

// ---------------------------------------------------------------------------
// Arithmetic policy
// ---------------------------------------------------------------------------
template <typename T, bool EX>
struct Ar {
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T div(T a, T b) { return a / b; }
  static __device__ __forceinline__ T sqr(T a) { return sqrt(a); }
};
template <>
struct Ar<double, true> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqr(double a) { return __dsqrt_rn(a); }
};

template <int KP> struct KT;
template <> struct KT<KP_BURGERS> { static constexpr int NC = 1, DIMS = 1; };
template <> struct KT<KP_ADVECT> { static constexpr int NC = 1, DIMS = 1; };
template <> struct KT<KP_HEAT1> { static constexpr int NC = 1, DIMS = 1; };
template <> struct KT<KP_HEAT2> { static constexpr int NC = 1, DIMS = 2; };
template <> struct KT<KP_HEAT3> { static constexpr int NC = 1, DIMS = 3; };
template <> struct KT<KP_DIFFREACT> { static constexpr int NC = 2, DIMS = 2; };
template <> struct KT<KP_BRUSS2> { static constexpr int NC = 2, DIMS = 2; };
template <> struct KT<KP_BRUSS3> { static constexpr int NC = 2, DIMS = 3; };
template <> struct KT<KP_SWE> { static constexpr int NC = 3, DIMS = 2; };

// Second differences summed over the axes: ((e - 2c) + w) / h^2 per axis.
template <int DIMS, typename T, bool EX>
__device__ __forceinline__ T lapl(T c, T e, T w, T n, T s, T up, T dn, T ix2,
                                  T iy2, T iz2) {
  using A = Ar<T, EX>;
  const T two = T(2);
  T r = A::mul(A::add(A::sub(e, A::mul(two, c)), w), ix2);
  if (DIMS >= 2) r = A::add(r, A::mul(A::add(A::sub(n, A::mul(two, c)), s), iy2));
  if (DIMS >= 3) r = A::add(r, A::mul(A::add(A::sub(up, A::mul(two, c)), dn), iz2));
  return r;
}

// Rusanov flux of the shallow-water system across one face (dir 0: x, 1: y).
template <typename T, bool EX>
__device__ __forceinline__ void swe_flux(T g, T hg, int dir, const T* L,
                                         const T* R, T* F) {
  using A = Ar<T, EX>;
  T uL = A::div(L[1], L[0]), vL = A::div(L[2], L[0]);
  T uR = A::div(R[1], R[0]), vR = A::div(R[2], R[0]);
  T FL[3], FR[3], sL, sR;
  if (dir == 0) {
    FL[0] = L[1];
    FL[1] = A::add(A::mul(L[1], uL), A::mul(A::mul(hg, L[0]), L[0]));
    FL[2] = A::mul(L[2], uL);
    FR[0] = R[1];
    FR[1] = A::add(A::mul(R[1], uR), A::mul(A::mul(hg, R[0]), R[0]));
    FR[2] = A::mul(R[2], uR);
    sL = A::add(fabs(uL), A::sqr(A::mul(g, L[0])));
    sR = A::add(fabs(uR), A::sqr(A::mul(g, R[0])));
  } else {
    FL[0] = L[2];
    FL[1] = A::mul(L[1], vL);
    FL[2] = A::add(A::mul(L[2], vL), A::mul(A::mul(hg, L[0]), L[0]));
    FR[0] = R[2];
    FR[1] = A::mul(R[1], vR);
    FR[2] = A::add(A::mul(R[2], vR), A::mul(A::mul(hg, R[0]), R[0]));
    sL = A::add(fabs(vL), A::sqr(A::mul(g, L[0])));
    sR = A::add(fabs(vR), A::sqr(A::mul(g, R[0])));
  }
  const T a = sL > sR ? sL : sR;
  const T half = T(0.5);
  const T ha = A::mul(half, a);
  for (int q = 0; q < 3; ++q)
    F[q] = A::sub(A::mul(half, A::add(FL[q], FR[q])), A::mul(ha, A::sub(R[q], L[q])));
}

// h(u) at one point from its own and its neighbours' component values.
// E/W: x +- 1; Nn/S: y +- 1; Up/Dn: z +- 1.
template <int KP, typename T, bool EX>
__device__ __forceinline__ void rhs_point(const T* C, const T* E, const T* W,
                                          const T* Nn, const T* S, const T* Up,
                                          const T* Dn, const T* k, T* out) {
  using A = Ar<T, EX>;
  constexpr int DIMS = KT<KP>::DIMS;
  if constexpr (KP == KP_BURGERS) {
    T diff = A::mul(k[0], lapl<1, T, EX>(C[0], E[0], W[0], T(0), T(0), T(0), T(0), k[1], T(0), T(0)));
    out[0] = A::sub(diff, A::mul(C[0], A::mul(A::sub(E[0], W[0]), k[2])));
  } else if constexpr (KP == KP_ADVECT) {
    out[0] = -(A::mul(k[0], A::mul(A::sub(E[0], W[0]), k[1])));
  } else if constexpr (KP == KP_HEAT1 || KP == KP_HEAT2 || KP == KP_HEAT3) {
    out[0] = A::mul(k[0], lapl<DIMS, T, EX>(C[0], E[0], W[0], Nn[0], S[0], Up[0], Dn[0], k[1], k[2], k[3]));
  } else if constexpr (KP == KP_DIFFREACT) {
    const T a = C[0], b = C[1];
    T lu = lapl<2, T, EX>(C[0], E[0], W[0], Nn[0], S[0], T(0), T(0), k[3], k[4], T(0));
    T lv = lapl<2, T, EX>(C[1], E[1], W[1], Nn[1], S[1], T(0), T(0), k[3], k[4], T(0));
    out[0] = A::add(A::mul(k[0], lu), A::sub(A::sub(A::sub(a, A::mul(A::mul(a, a), a)), k[2]), b));
    out[1] = A::add(A::mul(k[1], lv), A::sub(a, b));
  } else if constexpr (KP == KP_BRUSS2 || KP == KP_BRUSS3) {
    const T a = C[0], b = C[1];
    T lu = lapl<DIMS, T, EX>(C[0], E[0], W[0], Nn[0], S[0], Up[0], Dn[0], k[5], k[6], k[7]);
    T lv = lapl<DIMS, T, EX>(C[1], E[1], W[1], Nn[1], S[1], Up[1], Dn[1], k[5], k[6], k[7]);
    T a2 = A::mul(a, a);
    out[0] = A::add(A::mul(k[2], lu), A::add(A::sub(k[0], A::mul(k[4], a)), A::mul(b, a2)));
    out[1] = A::add(A::mul(k[3], lv), A::sub(A::mul(k[1], a), A::mul(b, a2)));
  } else if constexpr (KP == KP_SWE) {
    T Fe[3], Fw[3], Gn[3], Gs[3];
    swe_flux<T, EX>(k[0], k[1], 0, C, E, Fe);
    swe_flux<T, EX>(k[0], k[1], 0, W, C, Fw);
    swe_flux<T, EX>(k[0], k[1], 1, C, Nn, Gn);
    swe_flux<T, EX>(k[0], k[1], 1, S, C, Gs);
    for (int q = 0; q < 3; ++q)
      out[q] = A::add(A::mul(A::sub(Fw[q], Fe[q]), k[2]), A::mul(A::sub(Gs[q], Gn[q]), k[3]));
  }
}

// ---------------------------------------------------------------------------
// Fused, cluster-resident kernel
// ---------------------------------------------------------------------------
struct FusedParams {
  const double* in;
  double* out;
  double* out2;
  Items it;
  int nx, ny;
  long long n;
  int outer;
  int plane;
  int cluster;
  int steps;
  int scheme;
  double dt, h2, h6;
  Coef coef;
  float kf[12];      // coefficients rounded to FP32 (mixed kernel)
  float fdt, fh2, fh6;
};

template <int KP, typename T, bool EX, int R>
__global__ void __launch_bounds__(512, 1) k_stencil_fused(const FusedParams P) {
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  using A = Ar<T, EX>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CS = P.cluster;
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int item = blockIdx.x / CS;
  if (item >= P.it.n) return;                // uniform over the cluster
  if (P.it.gate && !P.it.gate[item]) return; // uniform over the cluster
  const int plane = P.plane, nx = P.nx, ny = P.ny;
  const int nloc = P.outer / CS;
  const int ncell = nloc * plane;
  T* const buf0 = reinterpret_cast<T*>(smem_raw);
  T* const buf1 = buf0 + NC * ncell;
  const T *rp0 = buf0, *rp1 = buf1, *rn0 = buf0, *rn1 = buf1;
  if (CS > 1) {
    cg::cluster_group cl = cg::this_cluster();
    const int rp = (rank + CS - 1) % CS, rn = (rank + 1) % CS;
    rp0 = cl.map_shared_rank(buf0, rp);
    rp1 = cl.map_shared_rank(buf1, rp);
    rn0 = cl.map_shared_rank(buf0, rn);
    rn1 = cl.map_shared_rank(buf1, rn);
  }
  T kk[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) kk[i] = T(P.coef.k[i]);
  const T dt = T(P.dt), h2 = T(P.h2), h6 = T(P.h6);
  const long long base = (long long)rank * ncell;
  const double* in = P.in + item_off(P.it.src_off, P.it.src_base, P.it.src_stride, item) + base;
  const int tid = threadIdx.x, TT = blockDim.x;

  T u[R][NC], acc[R][NC];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int c = tid + j * TT;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      T v = T(0);
      if (c < ncell) {
        v = T(in[q * P.n + c]);
        buf0[q * ncell + c] = v;
      }
      u[j][q] = v;
      acc[j][q] = T(0);
    }
  }
  if (CS > 1) cg::this_cluster().sync(); else __syncthreads();

  const int S = P.scheme == SCHEME_RK4 ? 4 : 1;
  int cur = 0;
  for (int step = 0; step < P.steps; ++step) {
    for (int s = 0; s < S; ++s) {
      const T* B = cur ? buf1 : buf0;
      T* Bn = cur ? buf0 : buf1;
      const T* BP = cur ? rp1 : rp0;
      const T* BN = cur ? rn1 : rn0;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int c = tid + j * TT;
        if (c >= ncell) continue;
        const int o = c / plane;
        const int ii = c - o * plane;
        int x, y;
        if (DIMS == 3) { y = ii / nx; x = ii - y * nx; } else { x = ii; y = 0; }
        const int xe = (x + 1 == nx) ? 0 : x + 1;
        const int xw = (x == 0) ? nx - 1 : x - 1;
        const int rowb = o * plane + (DIMS == 3 ? y * nx : 0);
        T Cv[NC], Ev[NC], Wv[NC], Nv[NC], Sv[NC], Uv[NC], Dv[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          const T* Bq = B + q * ncell;
          Cv[q] = Bq[c];
          Ev[q] = Bq[rowb + xe];
          Wv[q] = Bq[rowb + xw];
          Nv[q] = Sv[q] = Uv[q] = Dv[q] = T(0);
          if (DIMS == 3) {
            const int yn = (y + 1 == ny) ? 0 : y + 1;
            const int ys = (y == 0) ? ny - 1 : y - 1;
            Nv[q] = Bq[o * plane + yn * nx + x];
            Sv[q] = Bq[o * plane + ys * nx + x];
          }
          if (DIMS >= 2) {
            // outer neighbours: local, or the neighbouring CTA's first/last plane
            T vp, vm;
            if (o + 1 < nloc) vp = Bq[c + plane];
            else vp = BN[q * ncell + ii];
            if (o > 0) vm = Bq[c - plane];
            else vm = BP[q * ncell + (nloc - 1) * plane + ii];
            if (DIMS == 2) { Nv[q] = vp; Sv[q] = vm; } else { Uv[q] = vp; Dv[q] = vm; }
          }
        }
        T k[NC];
        rhs_point<KP, T, EX>(Cv, Ev, Wv, Nv, Sv, Uv, Dv, kk, k);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          T w;
          if (S == 1) {
            u[j][q] = A::add(u[j][q], A::mul(dt, k[q]));
            w = u[j][q];
          } else if (s == 0) {
            acc[j][q] = k[q];
            w = A::add(u[j][q], A::mul(h2, k[q]));
          } else if (s == 1) {
            acc[j][q] = A::add(acc[j][q], A::mul(T(2), k[q]));
            w = A::add(u[j][q], A::mul(h2, k[q]));
          } else if (s == 2) {
            acc[j][q] = A::add(acc[j][q], A::mul(T(2), k[q]));
            w = A::add(u[j][q], A::mul(dt, k[q]));
          } else {
            acc[j][q] = A::add(acc[j][q], k[q]);
            u[j][q] = A::add(u[j][q], A::mul(h6, acc[j][q]));
            w = u[j][q];
          }
          Bn[q * ncell + c] = w;
        }
      }
      cur ^= 1;
      if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    }
  }
  double* out = P.out + item_off(P.it.dst_off, P.it.dst_base, P.it.dst_stride, item) + base;
  double* out2 = P.out2 ? P.out2 + item_off(P.it.dst2_off, P.it.dst2_base, P.it.dst2_stride, item) + base
                        : nullptr;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int c = tid + j * TT;
    if (c >= ncell) continue;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      out[q * P.n + c] = double(u[j][q]);
      if (out2) out2[q * P.n + c] = double(u[j][q]);
    }
  }
}

// ---------------------------------------------------------------------------
// Plain per-stage kernels
// ---------------------------------------------------------------------------
struct PlainParams {
  const double* Wc;   // stage input [items][d]
  double* Wn;         // next stage input
  double* U;          // step state
  double* Acc;        // stage accumulator
  const int* gate;
  int nitems;
  int nx, ny, nz;
  long long n, d;
  int stage, scheme;
  double dt, h2, h6;
  Coef coef;
};

template <int KP>
__global__ void k_stage_plain(const PlainParams P) {
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  using A = Ar<double, true>;
  const long long tot = (long long)P.nitems * P.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int item = (int)(t / P.n);
    if (P.gate && !P.gate[item]) continue;
    const long long cell = t - (long long)item * P.n;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(cell % nx);
    const int y = (int)((cell / nx) % ny);
    const int z = (int)(cell / ((long long)nx * ny));
    const int xe = (x + 1) % nx, xw = (x + nx - 1) % nx;
    const int yn = (y + 1) % ny, ys = (y + ny - 1) % ny;
    const int zu = (z + 1) % nz, zd = (z + nz - 1) % nz;
    auto at = [&](int xx, int yy, int zz) { return ((long long)zz * ny + yy) * nx + xx; };
    const double* W = P.Wc + (long long)item * P.d;
    double Cv[NC], Ev[NC], Wv[NC], Nv[NC], Sv[NC], Uv[NC], Dv[NC];
    for (int q = 0; q < NC; ++q) {
      const double* Wq = W + q * P.n;
      Cv[q] = Wq[cell];
      Ev[q] = Wq[at(xe, y, z)];
      Wv[q] = Wq[at(xw, y, z)];
      Nv[q] = DIMS >= 2 ? Wq[at(x, yn, z)] : 0.0;
      Sv[q] = DIMS >= 2 ? Wq[at(x, ys, z)] : 0.0;
      Uv[q] = DIMS >= 3 ? Wq[at(x, y, zu)] : 0.0;
      Dv[q] = DIMS >= 3 ? Wq[at(x, y, zd)] : 0.0;
    }
    double k[NC];
    rhs_point<KP, double, true>(Cv, Ev, Wv, Nv, Sv, Uv, Dv, P.coef.k, k);
    for (int q = 0; q < NC; ++q) {
      const long long e = (long long)item * P.d + q * P.n + cell;
      double w;
      const double u = P.U[e];
      if (P.scheme == SCHEME_EULER) {
        w = A::add(u, A::mul(P.dt, k[q]));
        P.U[e] = w;
      } else if (P.stage == 0) {
        P.Acc[e] = k[q];
        w = A::add(u, A::mul(P.h2, k[q]));
      } else if (P.stage == 1) {
        P.Acc[e] = A::add(P.Acc[e], A::mul(2.0, k[q]));
        w = A::add(u, A::mul(P.h2, k[q]));
      } else if (P.stage == 2) {
        P.Acc[e] = A::add(P.Acc[e], A::mul(2.0, k[q]));
        w = A::add(u, A::mul(P.dt, k[q]));
      } else {
        const double a = A::add(P.Acc[e], k[q]);
        w = A::add(u, A::mul(P.h6, a));
        P.U[e] = w;
      }
      P.Wn[e] = w;
    }
  }
}


// ---------------------------------------------------------------------------
// Mixed-precision fused kernel: FP32 arithmetic, compensated state.
//
// Same residency scheme as k_stencil_fused, with three differences:
//  * the step state is an unevaluated sum u = uh + ul of two FP32 numbers;
//    each step's increment is added with an error-free TwoSum (Knuth), so the
//    state keeps ~48 bits over thousands of steps while every right-hand
//    side is evaluated in FP32 (uh in registers, ul in shared memory);
//  * thread t owns PX adjacent x-points (vector shared-memory accesses) over
//    RS consecutive outer rows: the outer-axis neighbours come from a rolling
//    window of registers, only the x neighbours (and y in 3D) are loaded;
//  * the four Runge-Kutta stages are unrolled at compile time.
// Requires nx % PX == 0 and (outer / cluster) % RS == 0.
// ---------------------------------------------------------------------------
template <int PX> struct VecT;
template <> struct VecT<1> { typedef float T; };
template <> struct VecT<2> { typedef float2 T; };
template <> struct VecT<4> { typedef float4 T; };

template <int PX>
__device__ __forceinline__ void ld_vec(const float* p, float* v) {
  if constexpr (PX == 1) { v[0] = p[0]; }
  else if constexpr (PX == 2) { float2 t = *reinterpret_cast<const float2*>(p); v[0] = t.x; v[1] = t.y; }
  else { float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
}
template <int PX>
__device__ __forceinline__ void st_vec(float* p, const float* v) {
  if constexpr (PX == 1) { p[0] = v[0]; }
  else if constexpr (PX == 2) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
  else { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
}

// (uh, ul) += x without rounding error in the sum (TwoSum, then renormalise).
__device__ __forceinline__ void two_sum_acc(float& uh, float& ul, float x) {
  const float s = __fadd_rn(uh, x);
  const float bb = __fsub_rn(s, uh);
  const float err = __fadd_rn(__fsub_rn(uh, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  const float l = __fadd_rn(ul, err);
  const float h = __fadd_rn(s, l);
  ul = __fsub_rn(l, __fsub_rn(h, s));
  uh = h;
}

template <int KP, int PX, int RS, int STAGE>
__device__ __forceinline__ void mixed_stage(const FusedParams& P, const float* __restrict__ B,
                                            float* __restrict__ Bn, const float* BP,
                                            const float* BN, float* ulo,
                                            float (&uh)[RS][KT<KP>::NC][PX],
                                            float (&acc)[RS][KT<KP>::NC][PX],
                                            int ncell, int plane, int nloc, int o0,
                                            int rowoff, int woff, int eoff, int yn_off, int ys_off,
                                            bool euler) {
  const float* kk = P.kf;
  const float dt = P.fdt, h2 = P.fh2, h6 = P.fh6;
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  float prv[NC][PX], cur[NC][PX], nxt[NC][PX];
  // rolling window along the outer axis (rows o0-1, o0, o0+1, ...)
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    ld_vec<PX>(B + q * ncell + o0 * plane + rowoff, cur[q]);
    if (DIMS >= 2) {
      if (o0 > 0) ld_vec<PX>(B + q * ncell + (o0 - 1) * plane + rowoff, prv[q]);
      else ld_vec<PX>(BP + q * ncell + (nloc - 1) * plane + rowoff, prv[q]);
    }
  }
#pragma unroll
  for (int r = 0; r < RS; ++r) {
    const int o = o0 + r;
    const int cb = o * plane + rowoff;  // first cell of this tile row
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      if (DIMS >= 2) {
        if (o + 1 < nloc) ld_vec<PX>(B + q * ncell + cb + plane, nxt[q]);
        else ld_vec<PX>(BN + q * ncell + rowoff, nxt[q]);
      }
    }
    float ew[NC], ee[NC];
    float yn[NC][PX], ys[NC][PX];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const float* Bq = B + q * ncell + o * plane;
      // x neighbours: aligned vector loads of the adjacent tiles (lanes read
      // consecutive vectors, so there is no bank conflict); keep the edge
      float vw[PX], ve[PX];
      ld_vec<PX>(Bq + woff, vw);
      ld_vec<PX>(Bq + eoff, ve);
      ew[q] = vw[PX - 1];
      ee[q] = ve[0];
      if (DIMS == 3) {
        ld_vec<PX>(Bq + yn_off, yn[q]);
        ld_vec<PX>(Bq + ys_off, ys[q]);
      }
    }
    float wout[NC][PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      float Cv[NC], Ev[NC], Wv[NC], Nv[NC], Sv[NC], Uv[NC], Dv[NC], k[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        Cv[q] = cur[q][p];
        Ev[q] = (p + 1 < PX) ? cur[q][p + 1] : ee[q];
        Wv[q] = (p > 0) ? cur[q][p - 1] : ew[q];
        if (DIMS == 2) { Nv[q] = nxt[q][p]; Sv[q] = prv[q][p]; Uv[q] = Dv[q] = 0.f; }
        else if (DIMS == 3) { Nv[q] = yn[q][p]; Sv[q] = ys[q][p]; Uv[q] = nxt[q][p]; Dv[q] = prv[q][p]; }
        else { Nv[q] = Sv[q] = Uv[q] = Dv[q] = 0.f; }
      }
      rhs_point<KP, float, false>(Cv, Ev, Wv, Nv, Sv, Uv, Dv, kk, k);
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        float w;
        if (euler) {
          float l = ulo[q * ncell + cb + p];
          two_sum_acc(uh[r][q][p], l, __fmul_rn(dt, k[q]));
          ulo[q * ncell + cb + p] = l;
          w = uh[r][q][p];
        } else if (STAGE == 0) {
          acc[r][q][p] = k[q];
          w = uh[r][q][p] + h2 * k[q];
        } else if (STAGE == 1) {
          acc[r][q][p] = acc[r][q][p] + 2.f * k[q];
          w = uh[r][q][p] + h2 * k[q];
        } else if (STAGE == 2) {
          acc[r][q][p] = acc[r][q][p] + 2.f * k[q];
          w = uh[r][q][p] + dt * k[q];
        } else {
          const float a = acc[r][q][p] + k[q];
          float l = ulo[q * ncell + cb + p];
          two_sum_acc(uh[r][q][p], l, __fmul_rn(h6, a));
          ulo[q * ncell + cb + p] = l;
          w = uh[r][q][p];
        }
        wout[q][p] = w;
      }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      st_vec<PX>(Bn + q * ncell + cb, wout[q]);
      if (DIMS >= 2) {
#pragma unroll
        for (int p = 0; p < PX; ++p) { prv[q][p] = cur[q][p]; cur[q][p] = nxt[q][p]; }
      }
    }
  }
}

template <int KP, int PX, int RS>
__global__ void __launch_bounds__(512, 1) k_stencil_mixed(const __grid_constant__ FusedParams P) {
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CS = P.cluster;
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int item = blockIdx.x / CS;
  if (item >= P.it.n) return;                // uniform over the cluster
  if (P.it.gate && !P.it.gate[item]) return; // uniform over the cluster
  const int plane = P.plane, nx = P.nx, ny = P.ny;
  const int nloc = P.outer / CS;
  const int ncell = nloc * plane;
  float* const buf0 = reinterpret_cast<float*>(smem_raw);
  float* const buf1 = buf0 + NC * ncell;
  float* const ulo = buf1 + NC * ncell;
  const float *rp0 = buf0, *rp1 = buf1, *rn0 = buf0, *rn1 = buf1;
  if (CS > 1) {
    cg::cluster_group cl = cg::this_cluster();
    const int rp = (rank + CS - 1) % CS, rn = (rank + 1) % CS;
    rp0 = cl.map_shared_rank(buf0, rp);
    rp1 = cl.map_shared_rank(buf1, rp);
    rn0 = cl.map_shared_rank(buf0, rn);
    rn1 = cl.map_shared_rank(buf1, rn);
  }
  // tile of this thread: PX x-points at inner offset rowoff, rows o0 .. o0+RS-1
  const int tiles = plane / PX;
  const int ti = threadIdx.x % tiles;
  const int o0 = (threadIdx.x / tiles) * RS;
  const int rowoff = ti * PX;                  // offset inside the plane
  const int x0 = rowoff % nx;
  const int yrow = rowoff / nx;                // y index in 3D (0 otherwise)
  const int xw = x0 == 0 ? nx - 1 : x0 - 1;
  const int xe = x0 + PX == nx ? 0 : x0 + PX;
  const int yn_off = (DIMS == 3 ? ((yrow + 1 == ny ? 0 : yrow + 1) * nx) : 0) + x0;
  const int ys_off = (DIMS == 3 ? ((yrow == 0 ? ny - 1 : yrow - 1) * nx) : 0) + x0;
  // first cells of the tiles west and east of this one (periodic in x)
  const int woff = yrow * nx + (xw + 1 - PX), eoff = yrow * nx + xe;

  const long long base = (long long)rank * ncell;
  const double* in = P.in + item_off(P.it.src_off, P.it.src_base, P.it.src_stride, item) + base;
  float uh[RS][NC][PX], acc[RS][NC][PX];
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        const int cell = (o0 + r) * plane + rowoff + p;
        const double v = in[q * P.n + cell];
        const float h = (float)v;
        uh[r][q][p] = h;
        acc[r][q][p] = 0.f;
        buf0[q * ncell + cell] = h;
        ulo[q * ncell + cell] = (float)(v - (double)h);
      }
  if (CS > 1) cg::this_cluster().sync(); else __syncthreads();

  const bool rk4 = P.scheme == SCHEME_RK4;
  for (int step = 0; step < P.steps; ++step) {
    if (rk4) {
      mixed_stage<KP, PX, RS, 0>(P, buf0, buf1, rp0, rn0, ulo, uh, acc, ncell, plane, nloc, o0,
                                 rowoff, woff, eoff, yn_off, ys_off, false);
      if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
      mixed_stage<KP, PX, RS, 1>(P, buf1, buf0, rp1, rn1, ulo, uh, acc, ncell, plane, nloc, o0,
                                 rowoff, woff, eoff, yn_off, ys_off, false);
      if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
      mixed_stage<KP, PX, RS, 2>(P, buf0, buf1, rp0, rn0, ulo, uh, acc, ncell, plane, nloc, o0,
                                 rowoff, woff, eoff, yn_off, ys_off, false);
      if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
      mixed_stage<KP, PX, RS, 3>(P, buf1, buf0, rp1, rn1, ulo, uh, acc, ncell, plane, nloc, o0,
                                 rowoff, woff, eoff, yn_off, ys_off, false);
      if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    } else {
      // forward Euler: buffers alternate every step
      if ((step & 1) == 0)
        mixed_stage<KP, PX, RS, 0>(P, buf0, buf1, rp0, rn0, ulo, uh, acc, ncell, plane, nloc, o0,
                                 rowoff, woff, eoff, yn_off, ys_off, true);
      else
        mixed_stage<KP, PX, RS, 0>(P, buf1, buf0, rp1, rn1, ulo, uh, acc, ncell, plane, nloc, o0,
                                 rowoff, woff, eoff, yn_off, ys_off, true);
      if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
    }
  }
  double* out = P.out + item_off(P.it.dst_off, P.it.dst_base, P.it.dst_stride, item) + base;
  double* out2 = P.out2 ? P.out2 + item_off(P.it.dst2_off, P.it.dst2_base, P.it.dst2_stride, item) + base
                        : nullptr;
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        const int cell = (o0 + r) * plane + rowoff + p;
        const double v = (double)uh[r][q][p] + (double)ulo[q * ncell + cell];
        out[q * P.n + cell] = v;
        if (out2) out2[q * P.n + cell] = v;
      }
}

typedef void (*FusedFn)(const FusedParams);
typedef void (*PlainFn)(const PlainParams);

template <int KP, typename T, bool EX>
inline FusedFn fused_for_R(int R) {
  switch (R) {
    case 1: return k_stencil_fused<KP, T, EX, 1>;
    case 2: return k_stencil_fused<KP, T, EX, 2>;
    case 4: return k_stencil_fused<KP, T, EX, 4>;
    case 8: return k_stencil_fused<KP, T, EX, 8>;
    case 16: return k_stencil_fused<KP, T, EX, 16>;
    default: return nullptr;
  }
}

template <int KP, int PX>
inline FusedFn mixed_for_RS(int RS) {
  switch (RS) {
    case 1: return k_stencil_mixed<KP, PX, 1>;
    case 2: return k_stencil_mixed<KP, PX, 2>;
    case 4: return k_stencil_mixed<KP, PX, 4>;
    case 5: return k_stencil_mixed<KP, PX, 5>;
    case 8: return k_stencil_mixed<KP, PX, 8>;
    default: return nullptr;
  }
}

// Per-PDE entry points, defined in stencil_<pde>.cu.
#define RNP_STENCIL_DECL(NAME)                 \
  FusedFn fused_fn_##NAME(bool fp32, int R);   \
  FusedFn mixed_fn_##NAME(int PX, int RS);     \
  PlainFn plain_fn_##NAME();
RNP_STENCIL_DECL(burgers)
RNP_STENCIL_DECL(advect)
RNP_STENCIL_DECL(heat1)
RNP_STENCIL_DECL(heat2)
RNP_STENCIL_DECL(heat3)
RNP_STENCIL_DECL(diffreact)
RNP_STENCIL_DECL(bruss2)
RNP_STENCIL_DECL(bruss3)
RNP_STENCIL_DECL(swe)
#undef RNP_STENCIL_DECL

#define RNP_STENCIL_DEFINE(KPV, NAME)                                                \
  FusedFn fused_fn_##NAME(bool fp32, int R) {                                        \
    return fp32 ? fused_for_R<KPV, float, false>(R) : fused_for_R<KPV, double, true>(R); \
  }                                                                                  \
  FusedFn mixed_fn_##NAME(int PX, int RS) {                                         \
    return PX == 2 ? mixed_for_RS<KPV, 2>(RS) : PX == 4 ? mixed_for_RS<KPV, 4>(RS) : nullptr; \
  }                                                                                  \
  PlainFn plain_fn_##NAME() { return k_stage_plain<KPV>; }

}  // namespace rnp
