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
  int* err;          // set to 1 when a halo wait times out (mixed kernel)
  int bc;            // 0 periodic, 1 no-flux walls (the wall neighbour is the cell)
  // mixed kernel, per launch: outer rows per CTA and the component strides
  // of its stage buffers (with ghost rows) and low words, read from the
  // parameter space instead of being kept in registers
  int nloc, mcell, mcl;
  int moff;          // byte offset of the mbarriers in the dynamic shared memory
  int tmcols;        // tensor-memory columns the CTA allocates (wide kernel)
  // eighth-order fine solver (FP64 kernel): a_{s,j} at rk[s*(s-1)/2 + j] for
  // stages s = 1..10, j < s, then b_0..b_10 at rk[55..65]
  double rk[66];
};

// Neighbours of cell c of this CTA's block (periodic wrap, or the cell
// itself across a no-flux wall; outer neighbours across a CTA boundary from
// the adjacent CTA's block BP / BN) and h(u) there.
template <int KP, typename T, bool EX>
__device__ __forceinline__ void fused_cell_rhs(const FusedParams& P, const T* B, const T* BP,
                                               const T* BN, int c, int ncell, int nloc,
                                               int rank, int CS, const T* kk, T* k) {
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  const int plane = P.plane, nx = P.nx, ny = P.ny;
  const int o = c / plane;
  const int ii = c - o * plane;
  int x, y;
  if (DIMS == 3) { y = ii / nx; x = ii - y * nx; } else { x = ii; y = 0; }
  // neighbours: periodic wrap, or the cell itself across a no-flux wall
  const bool wall = P.bc != 0;
  const int xe = (x + 1 == nx) ? (wall ? x : 0) : x + 1;
  const int xw = (x == 0) ? (wall ? 0 : nx - 1) : x - 1;
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
      const int yn = (y + 1 == ny) ? (wall ? y : 0) : y + 1;
      const int ys = (y == 0) ? (wall ? 0 : ny - 1) : y - 1;
      Nv[q] = Bq[o * plane + yn * nx + x];
      Sv[q] = Bq[o * plane + ys * nx + x];
    }
    if (DIMS >= 2) {
      // outer neighbours: local, the neighbouring CTA's first/last
      // plane, or (at a wall) the cell itself
      T vp, vm;
      if (o + 1 < nloc) vp = Bq[c + plane];
      else if (wall && rank == CS - 1) vp = Cv[q];
      else vp = BN[q * ncell + ii];
      if (o > 0) vm = Bq[c - plane];
      else if (wall && rank == 0) vm = Cv[q];
      else vm = BP[q * ncell + (nloc - 1) * plane + ii];
      if (DIMS == 2) { Nv[q] = vp; Sv[q] = vm; } else { Uv[q] = vp; Dv[q] = vm; }
    }
  }
  if constexpr (KP == KP_SWE) {
    // reflecting walls: the cell across a wall is this cell with its
    // momentum normal to the wall negated
    if (wall) {
      if (x + 1 == nx) Ev[1] = -Ev[1];
      if (x == 0) Wv[1] = -Wv[1];
      if (o + 1 == nloc && rank == CS - 1) Nv[2] = -Nv[2];
      if (o == 0 && rank == 0) Sv[2] = -Sv[2];
    }
  }
  rhs_point<KP, T, EX>(Cv, Ev, Wv, Nv, Sv, Uv, Dv, kk, k);
  if constexpr (KP == KP_SWE) {
    // bottom term -g h grad b
    if (P.coef.bath) {
      using A = Ar<T, EX>;
      const long long gi = (long long)rank * ncell + c;
      k[1] = A::sub(k[1], A::mul(Cv[0], T(P.coef.bath[gi])));
      k[2] = A::sub(k[2], A::mul(Cv[0], T(P.coef.bath[P.n + gi])));
    }
  }
}

template <int KP, typename T, bool EX, int R>
__global__ void __launch_bounds__(512, 1) k_stencil_fused(const FusedParams P) {
  constexpr int NC = KT<KP>::NC;
  using A = Ar<T, EX>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CS = P.cluster;
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int item = blockIdx.x / CS;
  if (item >= P.it.n) return;                // uniform over the cluster
  if (P.it.gate && !P.it.gate[item]) return; // uniform over the cluster
  const int nloc = P.outer / CS;
  const int ncell = nloc * P.plane;
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
        T k[NC];
        fused_cell_rhs<KP, T, EX>(P, B, BP, BN, c, ncell, nloc, rank, CS, kk, k);
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

// FP64 eighth-order fine solver (the eleven-stage explicit method of Cooper
// & Verner, SIAM J. Numer. Anal. 9, 1972; the paper's F is RK8, Sec. 5.1-5.2).
// Same residency and neighbour exchange as k_stencil_fused; the ten stage
// derivatives k_0..k_9 of a step stay in registers (R <= 2 cells per
// thread).  Stage s is evaluated at u + dt (a_{s,0} k_0 + ... + a_{s,s-1}
// k_{s-1}), summed left to right, and the step adds dt (b_0 k_0 + ... +
// b_10 k_10); every operation is explicitly rounded, so the result is
// bit-identical to a plain serial evaluation of the same sums.
template <int KP, int R>
__global__ void __launch_bounds__(512, 1) k_stencil_fused_rk8(const FusedParams P) {
  using T = double;
  using A = Ar<double, true>;
  constexpr int NC = KT<KP>::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CS = P.cluster;
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int item = blockIdx.x / CS;
  if (item >= P.it.n) return;                // uniform over the cluster
  if (P.it.gate && !P.it.gate[item]) return; // uniform over the cluster
  const int nloc = P.outer / CS;
  const int ncell = nloc * P.plane;
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
  for (int i = 0; i < 12; ++i) kk[i] = P.coef.k[i];
  const T dt = P.dt;
  const long long base = (long long)rank * ncell;
  const double* in = P.in + item_off(P.it.src_off, P.it.src_base, P.it.src_stride, item) + base;
  const int tid = threadIdx.x, TT = blockDim.x;

  T u[R][NC], ks[10][R][NC];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int c = tid + j * TT;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      T v = T(0);
      if (c < ncell) {
        v = in[q * P.n + c];
        buf0[q * ncell + c] = v;
      }
      u[j][q] = v;
    }
  }
  if (CS > 1) cg::this_cluster().sync(); else __syncthreads();

  int cur = 0;
  for (int step = 0; step < P.steps; ++step) {
#pragma unroll
    for (int s = 0; s < 11; ++s) {
      const T* B = cur ? buf1 : buf0;
      T* Bn = cur ? buf0 : buf1;
      const T* BP = cur ? rp1 : rp0;
      const T* BN = cur ? rn1 : rn0;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int c = tid + j * TT;
        if (c >= ncell) continue;
        T k[NC];
        fused_cell_rhs<KP, T, true>(P, B, BP, BN, c, ncell, nloc, rank, CS, kk, k);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          T w;
          if (s < 10) {
            // input of stage s + 1
            const double* an = P.rk + (s + 1) * s / 2;
            ks[s][j][q] = k[q];
            T acc = A::mul(an[0], ks[0][j][q]);
#pragma unroll
            for (int i = 1; i <= s; ++i) acc = A::add(acc, A::mul(an[i], ks[i][j][q]));
            w = A::add(u[j][q], A::mul(dt, acc));
          } else {
            const double* bw = P.rk + 55;
            T acc = A::mul(bw[0], ks[0][j][q]);
#pragma unroll
            for (int i = 1; i < 10; ++i) acc = A::add(acc, A::mul(bw[i], ks[i][j][q]));
            acc = A::add(acc, A::mul(bw[10], k[q]));
            u[j][q] = A::add(u[j][q], A::mul(dt, acc));
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
      out[q * P.n + c] = u[j][q];
      if (out2) out2[q * P.n + c] = u[j][q];
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
  int bc;             // 0 periodic, 1 no-flux walls
  double* Kst;        // RK8: stage derivatives k_0..k_9, [10][nitems * d]
  double rk[66];      // RK8 tableau, laid out as in FusedParams::rk
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
    // neighbours: periodic wrap, or the cell itself across a no-flux wall
    const bool wall = P.bc != 0;
    const int xe = x + 1 < nx ? x + 1 : (wall ? x : 0);
    const int xw = x > 0 ? x - 1 : (wall ? x : nx - 1);
    const int yn = y + 1 < ny ? y + 1 : (wall ? y : 0);
    const int ys = y > 0 ? y - 1 : (wall ? y : ny - 1);
    const int zu = z + 1 < nz ? z + 1 : (wall ? z : 0);
    const int zd = z > 0 ? z - 1 : (wall ? z : nz - 1);
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
    if constexpr (KP == KP_SWE) {
      // reflecting walls: the normal momentum of the mirrored cell is negated
      if (wall) {
        if (x + 1 == nx) Ev[1] = -Ev[1];
        if (x == 0) Wv[1] = -Wv[1];
        if (y + 1 == ny) Nv[2] = -Nv[2];
        if (y == 0) Sv[2] = -Sv[2];
      }
    }
    double k[NC];
    rhs_point<KP, double, true>(Cv, Ev, Wv, Nv, Sv, Uv, Dv, P.coef.k, k);
    if constexpr (KP == KP_SWE) {
      if (P.coef.bath) {   // bottom term -g h grad b
        k[1] = A::sub(k[1], A::mul(Cv[0], P.coef.bath[cell]));
        k[2] = A::sub(k[2], A::mul(Cv[0], P.coef.bath[P.n + cell]));
      }
    }
    for (int q = 0; q < NC; ++q) {
      const long long e = (long long)item * P.d + q * P.n + cell;
      double w;
      const double u = P.U[e];
      if (P.scheme == SCHEME_RK8) {
        // stage s: keep k_s, then form the input of stage s + 1 (or the step)
        const long long tot = (long long)P.nitems * P.d;
        const int s = P.stage;
        const double* cf = s < 10 ? P.rk + (s + 1) * s / 2 : P.rk + 55;
        double acc = A::mul(cf[0], s == 0 ? k[q] : P.Kst[e]);
        for (int i = 1; i <= s; ++i)
          acc = A::add(acc, A::mul(cf[i], i == s ? k[q] : P.Kst[i * tot + e]));
        if (s < 10) P.Kst[s * tot + e] = k[q];
        w = A::add(u, A::mul(P.dt, acc));
        if (s == 10) P.U[e] = w;
      } else if (P.scheme == SCHEME_EULER) {
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
// Same residency as k_stencil_fused (one slice per cluster, split along the
// outer axis, stage values double-buffered in shared memory), with these
// differences:
//  * the step state is an unevaluated sum u = uh + ul of two FP32 numbers;
//    each step's increment is added with Fast2Sum (Dekker), so the
//    state keeps ~48 bits over thousands of steps while every right-hand
//    side is evaluated in FP32 (uh in registers, ul in shared memory);
//  * thread t owns PX adjacent x-points (vector shared-memory accesses) over
//    RS consecutive outer rows: the outer-axis neighbours come from a rolling
//    window of registers, only the x neighbours (and y in 3D) are loaded;
//  * the four Runge-Kutta stages are unrolled at compile time;
//  * for the two-species reaction-diffusion operators (diffusion-reaction,
//    Brusselator) pairs of x-points share packed FP32 instructions
//    (fadd2 / fmul2 / ffma2), halving the arithmetic instructions;
//  * no CTA reads another CTA's stage buffer.  The threads that own a CTA's
//    first or last outer row push that row's new stage values into the
//    neighbouring CTA's halo rows (st.async into distributed shared memory,
//    completing bytes on that CTA's mbarrier), so a stage ends with a CTA
//    barrier instead of a cluster barrier.  Halos and mbarriers are
//    double-buffered by stage parity.  The group owning the last row walks
//    its rows downwards, so both edge rows are computed (and pushed) first
//    in a stage and their halos are read a whole stage after they were sent.
//    Every mbarrier wait is bounded: on timeout the kernel sets *err, all
//    CTAs leave the step loop at the next stage boundary and meet at one
//    final cluster barrier.
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

// (uh, ul) += x, keeping the rounding error of the sum: Dekker's Fast2Sum
// (exact when |uh| >= |x|, i.e. whenever the step increment is smaller than
// the state; where the state crosses zero the error term is approximate, to
// within an ulp of the increment), then renormalise.
__device__ __forceinline__ void two_sum_acc(float& uh, float& ul, float x) {
  const float s = __fadd_rn(uh, x);
  const float err = __fsub_rn(x, __fsub_rn(s, uh));
  const float l = __fadd_rn(ul, err);
  const float h = __fadd_rn(s, l);
  ul = __fsub_rn(l, __fsub_rn(h, s));
  uh = h;
}

// Packed FP32 (two lanes per instruction, sm_100 and later): the two
// x-points of a PX = 2 tile share each arithmetic instruction.  a - b is
// fma(b, -1, a): b * -1 is exact, so the result is a - b rounded once.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk1(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// two_sum_acc on both lanes
__device__ __forceinline__ void two_sum_acc2(float2& uh, float2& ul, float2 x) {
  const float2 s = add2(uh, x);
  const float2 err = sub2(x, sub2(s, uh));
  const float2 l = add2(ul, err);
  const float2 h = add2(s, l);
  ul = sub2(l, sub2(h, s));
  uh = h;
}

// --- distributed-shared-memory halo exchange ------------------------------
// Bound of a halo wait: kPolls polls (each may suspend the thread for the
// hardware's own short time limit; a suspend-time hint would cost the
// register-tight stencil a spill).
static constexpr unsigned kPolls = 2u << 20;


__device__ __forceinline__ uint32_t cta_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_map_u32(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// PX FP32 values to another CTA's shared memory; completes PX*4 bytes on
// that CTA's mbarrier.
template <int PX>
__device__ __forceinline__ void st_async_vec(uint32_t addr, const float* v, uint32_t mbar) {
  if constexpr (PX == 2)
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
        ::"r"(addr), "f"(v[0]), "f"(v[1]), "r"(mbar) : "memory");
  else if constexpr (PX == 4)
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
        ::"r"(addr), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "r"(mbar) : "memory");
  else
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];"
                 ::"r"(addr), "f"(v[0]), "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase of the given parity; acquire at cluster scope
// (the bytes were written by other CTAs of the cluster).
// Polls until the phase completes, at most kPolls times; false when the
// wait gave up.
__device__ __forceinline__ bool halo_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned it = 0; it < kPolls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Whether the phase of the given parity has completed (no wait).
__device__ __forceinline__ bool mbar_done(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
// Counts bytes that will never arrive as received, so that the phase can
// complete on the bytes that were sent.
__device__ __forceinline__ void mbar_complete(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// Where a stage sends its edge rows: outer row 0 to the previous rank's
// ghost row nloc, outer row nloc - 1 to the next rank's ghost row -1, both
// in the buffer of the next stage's parity (with no-flux walls the first and
// last ranks keep their wall rows: row 0 to their own ghost row -1, row
// nloc - 1 to their own ghost row nloc).  Addresses are 32-bit
// shared-window addresses: the neighbours' windows (mapa) for a cluster of
// several CTAs, this CTA's own window for a one-CTA cluster (periodic wrap
// onto itself, written with plain shared stores).  The four targets are the
// same for every thread of a CTA and sit in shared memory (tab: row-0
// target, row-(nloc-1) target, previous / next rank's mbarrier 0), so the
// register tile does not carry them.
struct HaloOut {
  bool on;               // false on the last stage of the launch
  bool self;             // one-CTA cluster
  bool first, last, edge;  // this thread owns outer row 0 / nloc - 1 / either
  const uint4* tab;      // the CTA's target table
  uint32_t boff;         // byte offset of buffer `parity` from buffer 0
  uint32_t moff;         // byte offset of mbarrier `parity` from mbarrier 0
};

template <int PX>
__device__ __forceinline__ void st_shared_vec(uint32_t addr, const float* v) {
  if constexpr (PX == 2)
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v[0]), "f"(v[1]) : "memory");
  else if constexpr (PX == 4)
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3]) : "memory");
  else
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v[0]) : "memory");
}

// Sends PX values (element `elem` of the row, counted in floats from the
// start of the buffer) of outer row 0 (to_prev) or nloc - 1; t is the
// CTA's target table (*h.tab), read once by the caller for all its pushes.
template <int PX>
__device__ __forceinline__ void push_edge(const HaloOut& h, const uint4& t, bool to_prev,
                                          uint32_t elem, const float* v) {
  const uint32_t a = (to_prev ? t.x : t.y) + h.boff + 4u * elem;
  const uint32_t mb = to_prev ? t.z : t.w;  // 0: a local target (wall)
  if (h.self || mb == 0) st_shared_vec<PX>(a, v);
  else st_async_vec<PX>(a, v, mb + h.moff);
}

// push_edge for component q; a shallow-water wall ghost row (a local target
// when WALL) mirrors the row with its normal momentum hv negated
template <int KP, int PX, bool WALL>
__device__ __forceinline__ void push_edge_q(const HaloOut& h, const uint4& t, bool to_prev,
                                            uint32_t elem, const float* v, int q) {
  if constexpr (WALL && KP == KP_SWE) {
    if (q == 2) {
      if (h.self || (to_prev ? t.z : t.w) == 0) {
        float nv[PX];
#pragma unroll
        for (int p = 0; p < PX; ++p) nv[p] = -v[p];
        push_edge<PX>(h, t, to_prev, elem, nv);
        return;
      }
    }
  }
  push_edge<PX>(h, t, to_prev, elem, v);
}

// --- tensor memory as per-thread storage -------------------------------
// The wide 3D kernel keeps each thread's step state uh and Runge-Kutta
// accumulator in tensor memory (TMEM, 256 KB per SM, otherwise unused by
// the stencil) instead of registers: warp w reaches TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31 (its lane quadrant), thread i of the warp
// lane 32 (w % 4) + i, and the warps sharing a quadrant use disjoint column
// ranges.  tcgen05.ld / tcgen05.st move N consecutive 32-bit columns of the
// thread's own lane; both are warp-collective and asynchronous
// (tcgen05.wait::ld before the loaded registers are used, tcgen05.wait::st
// before the columns are read again).  Only N = 4 and 8 are used.
template <int N>
__device__ __forceinline__ void tm_ld(uint32_t taddr, float* v) {
  uint32_t r[N];
  if constexpr (N == 4)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
  else
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}
template <int N>
__device__ __forceinline__ void tm_st(uint32_t taddr, const float* v) {
  if constexpr (N == 4)
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                 "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 : "memory");
  else
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                     taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                 "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                 "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
// Waits for this thread's TMEM loads; the registers pass through the asm so
// that no use of them is scheduled before the wait.
template <int N>
__device__ __forceinline__ void tm_wait_ld(float* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+f"(v[i]));
}
// The same register fence for more loaded registers after a tm_wait_ld (one
// wait covers every earlier load of the thread).
template <int N>
__device__ __forceinline__ void tm_fence_ld(float* v) {
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+f"(v[i]));
}
__device__ __forceinline__ void tm_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int KP, int PX, int RS, int STAGE, bool XS, bool WALL, bool TM, bool ISO>
__device__ __forceinline__ void mixed_stage(const FusedParams& P, const float* __restrict__ B,
                                            float* __restrict__ Bn, float* ulo,
                                            float (&uh)[RS][KT<KP>::NC][PX],
                                            float (&acc)[RS][KT<KP>::NC][PX], uint32_t tm,
                                            int ncell, int plane, int nloc, int ofirst, int dir,
                                            int rowoff, int dW, int dE, int dN, int dS,
                                            bool euler, const HaloOut& ho, unsigned xmask,
                                            int xw, int xwest, int xeast, bool xlo, bool xhi,
                                            const float* __restrict__ bth) {
  const float* kk = P.kf;
  const float dt = P.fdt, h2 = P.fh2, h6 = P.fh6;
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  const int ncl = P.mcl;  // component stride of the low words (no ghost rows)
  // two-species reaction-diffusion with an even number of x-points per
  // thread: packed FP32 on pairs of points; kk[kLx..] = 1/hx^2, 1/hy^2, 1/hz^2
  constexpr bool kPacked =
      PX % 2 == 0 && (KP == KP_DIFFREACT || KP == KP_BRUSS2 || KP == KP_BRUSS3);
  constexpr int kLx = KP == KP_DIFFREACT ? 3 : 5;
  // ISO (equal spacing h on every axis): the Laplacian is the neighbour sum
  // minus 2 DIMS times the centre, and the diffusion coefficients come
  // premultiplied by 1/h^2: kk[kIsoD], kk[kIsoD + 1] = D_u / h^2, D_v / h^2
  constexpr int kIsoD = KP == KP_DIFFREACT ? 5 : 8;
  // Only the shallow-water fluxes tell the two outer neighbours apart; the
  // other right-hand sides take their sum.
  constexpr bool kOrdered = KP == KP_SWE;
  const int rstep = dir * plane;
  // rolling window along the walking direction: `back` is the row behind
  // the one being updated, `ahead` the row in front of it (ghost rows -1
  // and nloc hold the neighbours' edge rows)
  float back[NC][PX], cur[NC][PX], ahead[NC][PX];
  // this row's first cell in the read buffer, the write buffer, the low
  // words and the bottom factors (species 0); advanced by rstep per row.
  // The neighbours sit at fixed offsets from it: dW / dE the first cells of
  // the west / east tiles, dN / dS the y neighbours (3D), rstep the next row.
  const int c0 = ofirst * plane + rowoff;
  const float* pB = B + c0;
  float* pBn = Bn + c0;
  float* pL = TM ? nullptr : ulo + c0;
  const float* pT = bth ? bth + c0 : nullptr;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    ld_vec<PX>(pB + q * ncell, cur[q]);
    if (DIMS >= 2) ld_vec<PX>(pB + q * ncell - rstep, back[q]);
  }
  // (TM: the rows' state is addressed in tensor memory, so the row loop can
  // stay partly rolled, which keeps two rows' values live at a time:
  // unrolled by 2 it measured 4 % faster than rolled and 6 % faster than
  // fully unrolled on the 3D Brusselator)
#pragma unroll (TM ? 2 : RS)
  for (int r = 0; r < RS; ++r) {
    // this row's step state and accumulator: the register tile's row, or
    // (TM) a copy loaded from tensor memory (columns r NC PX .. of the
    // thread's uh block, then of its accumulator block RS NC PX further)
    // (TM: the low words of the compensated state too, at 2 RS NC PX, read
    // and written in Euler steps and the last RK stage)
    float ur[NC][PX], ar[NC][PX], lr[NC][PX];
    if constexpr (TM) {
      // the row's loads in flight together, then one wait
      tm_ld<NC * PX>(tm + (uint32_t)(r * NC * PX), &ur[0][0]);
      if (!euler && STAGE > 0)
        tm_ld<NC * PX>(tm + (uint32_t)((RS + r) * NC * PX), &ar[0][0]);
      if (euler || STAGE == 3)
        tm_ld<NC * PX>(tm + (uint32_t)((2 * RS + r) * NC * PX), &lr[0][0]);
      tm_wait_ld<NC * PX>(&ur[0][0]);
      if (!euler && STAGE > 0) tm_fence_ld<NC * PX>(&ar[0][0]);
      if (euler || STAGE == 3) tm_fence_ld<NC * PX>(&lr[0][0]);
    }
    float (&U_)[NC][PX] = TM ? ur : uh[r];
    float (&A_)[NC][PX] = TM ? ar : acc[r];
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if (DIMS >= 2) ld_vec<PX>(pB + q * ncell + rstep, ahead[q]);
    float ew[NC], ee[NC];
    float yn[NC][PX], ys[NC][PX];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const float* Bq = pB + q * ncell;   // this tile's first cell, species q
      if constexpr (XS) {
        // x neighbours from the adjacent lanes: an x-row spans xw lanes, so
        // a width-xw shuffle wraps periodically in x
        ew[q] = __shfl_sync(xmask, cur[q][PX - 1], xwest, xw);
        ee[q] = __shfl_sync(xmask, cur[q][0], xeast, xw);
      } else if constexpr (kPacked) {
        // x neighbours: the adjacent tiles' edge values, loaded as scalars
        // into one register pair for the packed arithmetic
        if constexpr (PX == 4) {
          // the last pair of the west tile and the first pair of the east
          // tile: 8-byte loads halve the bank conflicts of the strided
          // 4-byte loads
          ew[q] = reinterpret_cast<const float2*>(Bq + dW + PX - 2)->y;
          ee[q] = reinterpret_cast<const float2*>(Bq + dE)->x;
        } else {
          ew[q] = Bq[dW + PX - 1];
          ee[q] = Bq[dE];
        }
      } else {
        // x neighbours: aligned vector loads of the adjacent tiles (lanes
        // read consecutive vectors, so there is no bank conflict); keep the edge
        float vw[PX], ve[PX];
        ld_vec<PX>(Bq + dW, vw);
        ld_vec<PX>(Bq + dE, ve);
        ew[q] = vw[PX - 1];
        ee[q] = ve[0];
      }
      if constexpr (WALL) {
        // no-flux walls: the neighbour across the wall is the cell itself
        // (shallow water: with its normal momentum hu negated)
        constexpr bool kFlip = KP == KP_SWE;
        if (xlo) ew[q] = (kFlip && q == 1) ? -cur[q][0] : cur[q][0];
        if (xhi) ee[q] = (kFlip && q == 1) ? -cur[q][PX - 1] : cur[q][PX - 1];
      }
      if (DIMS == 3) {
        ld_vec<PX>(Bq + dN, yn[q]);
        ld_vec<PX>(Bq + dS, ys[q]);
      }
    }
    // shallow water: the bottom term's per-cell factors of this tile row
    float bx[PX], by[PX];
    if constexpr (KP == KP_SWE) {
      if (bth) {
        ld_vec<PX>(pT, bx);
        ld_vec<PX>(pT + P.n, by);
      }
    }
    float wout[NC][PX];
    if constexpr (kPacked) {
      // pairs of x-points (2i, 2i + 1) in packed FP32: the outer neighbours
      // pair up as loaded; in x, point 2i's east neighbour is point 2i + 1
      // and point 2i + 1's west neighbour point 2i, the other two are the
      // tile's or the adjacent tiles' values
#pragma unroll
      for (int pp = 0; pp < PX / 2; ++pp) {
        const int p0 = 2 * pp, p1 = 2 * pp + 1;
        float2 kq[NC], Cq[NC], lq[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          const float w0 = p0 > 0 ? cur[q][p0 - 1] : ew[q];
          const float e1 = p1 + 1 < PX ? cur[q][p1 + 1] : ee[q];
          const float2 C = pk(cur[q][p0], cur[q][p1]);
          // E + W of both points, as two scalar adds that write the pair
          const float2 EW = pk(cur[q][p1] + w0, e1 + cur[q][p0]);
          const float2 hi = pk(ahead[q][p0], ahead[q][p1]);
          const float2 lo = pk(back[q][p0], back[q][p1]);
          float2 l;
          if constexpr (ISO) {
            // unscaled: (sum of the 2 DIMS neighbours) - 2 DIMS C
            float2 sum = add2(EW, add2(hi, lo));
            if constexpr (DIMS == 3)
              sum = add2(sum, add2(pk(yn[q][p0], yn[q][p1]), pk(ys[q][p0], ys[q][p1])));
            l = fma2(pk1(-2.f * DIMS), C, sum);
          } else if constexpr (DIMS == 2) {
            const float2 lx = mul2(fma2(pk1(-2.f), C, EW), pk1(kk[kLx]));
            l = fma2(fma2(pk1(-2.f), C, add2(hi, lo)), pk1(kk[kLx + 1]), lx);
          } else {
            const float2 NS = add2(pk(yn[q][p0], yn[q][p1]), pk(ys[q][p0], ys[q][p1]));
            const float2 lx = mul2(fma2(pk1(-2.f), C, EW), pk1(kk[kLx]));
            const float2 ly = fma2(fma2(pk1(-2.f), C, NS), pk1(kk[kLx + 1]), lx);
            l = fma2(fma2(pk1(-2.f), C, add2(hi, lo)), pk1(kk[kLx + 2]), ly);
          }
          lq[q] = l;
          Cq[q] = C;
        }
        const float2 a = Cq[0], b = Cq[1];
        if constexpr (KP == KP_DIFFREACT) {
          // Du lap u + (u - u^3 - c - v);  Dv lap v + (u - v), the first
          // reaction term factored as -c - (u (u^2 - 1) + v)
          constexpr int iD = ISO ? kIsoD : 0;
          const float2 w = fma2(a, fma2(a, a, pk1(-1.f)), b);
          kq[0] = fma2(pk1(kk[iD]), lq[0], sub2(pk1(-kk[2]), w));
          kq[1] = fma2(pk1(kk[iD + 1]), lq[1], sub2(a, b));
        } else {
          // D0 lap u + (a - (1 + b) u + v u^2);  D1 lap v + (b u - v u^2),
          // factored: a + u (v u - (1 + b)) and u (b - v u), where
          // b - v u = (b - (1 + b)) - (v u - (1 + b))
          constexpr int iD = ISO ? kIsoD : 2;
          const float2 s0 = fma2(b, a, pk1(-kk[4]));
          kq[0] = fma2(pk1(kk[iD]), lq[0], fma2(a, s0, pk1(kk[0])));
          kq[1] = fma2(pk1(kk[iD + 1]), lq[1], mul2(a, sub2(pk1(kk[1] - kk[4]), s0)));
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          float2 U = pk(U_[q][p0], U_[q][p1]);
          float2 w;
          if (euler) {
            float2 l = TM ? pk(lr[q][p0], lr[q][p1]) : *reinterpret_cast<const float2*>(pL + q * ncl + p0);
            two_sum_acc2(U, l, mul2(pk1(dt), kq[q]));
            if constexpr (TM) { lr[q][p0] = l.x; lr[q][p1] = l.y; } else *reinterpret_cast<float2*>(pL + q * ncl + p0) = l;
            w = U;
          } else if (STAGE == 0) {
            A_[q][p0] = kq[q].x; A_[q][p1] = kq[q].y;
            w = fma2(pk1(h2), kq[q], U);
          } else if (STAGE == 1 || STAGE == 2) {
            const float2 A2 = fma2(pk1(2.f), kq[q], pk(A_[q][p0], A_[q][p1]));
            A_[q][p0] = A2.x; A_[q][p1] = A2.y;
            w = fma2(pk1(STAGE == 1 ? h2 : dt), kq[q], U);
          } else {
            const float2 A2 = add2(pk(A_[q][p0], A_[q][p1]), kq[q]);
            float2 l = TM ? pk(lr[q][p0], lr[q][p1]) : *reinterpret_cast<const float2*>(pL + q * ncl + p0);
            two_sum_acc2(U, l, mul2(pk1(h6), A2));
            if constexpr (TM) { lr[q][p0] = l.x; lr[q][p1] = l.y; } else *reinterpret_cast<float2*>(pL + q * ncl + p0) = l;
            w = U;
          }
          U_[q][p0] = U.x; U_[q][p1] = U.y;
          wout[q][p0] = w.x; wout[q][p1] = w.y;
        }
      }
    } else {
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        float Cv[NC], Ev[NC], Wv[NC], Nv[NC], Sv[NC], Uv[NC], Dv[NC], k[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          // outer neighbours o + 1 and o - 1
          const float hi = kOrdered ? (dir > 0 ? ahead[q][p] : back[q][p]) : ahead[q][p];
          const float lo = kOrdered ? (dir > 0 ? back[q][p] : ahead[q][p]) : back[q][p];
          Cv[q] = cur[q][p];
          Ev[q] = (p + 1 < PX) ? cur[q][p + 1] : ee[q];
          Wv[q] = (p > 0) ? cur[q][p - 1] : ew[q];
          if (DIMS == 2) { Nv[q] = hi; Sv[q] = lo; Uv[q] = Dv[q] = 0.f; }
          else if (DIMS == 3) { Nv[q] = yn[q][p]; Sv[q] = ys[q][p]; Uv[q] = hi; Dv[q] = lo; }
          else { Nv[q] = Sv[q] = Uv[q] = Dv[q] = 0.f; }
        }
        rhs_point<KP, float, false>(Cv, Ev, Wv, Nv, Sv, Uv, Dv, kk, k);
        if constexpr (KP == KP_SWE) {
          if (bth) {
            k[1] = k[1] - Cv[0] * bx[p];
            k[2] = k[2] - Cv[0] * by[p];
          }
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          float w;
          if (euler) {
            float l = TM ? lr[q][p] : pL[q * ncl + p];
            two_sum_acc(U_[q][p], l, __fmul_rn(dt, k[q]));
            if constexpr (TM) lr[q][p] = l; else pL[q * ncl + p] = l;
            w = U_[q][p];
          } else if (STAGE == 0) {
            A_[q][p] = k[q];
            w = U_[q][p] + h2 * k[q];
          } else if (STAGE == 1) {
            A_[q][p] = A_[q][p] + 2.f * k[q];
            w = U_[q][p] + h2 * k[q];
          } else if (STAGE == 2) {
            A_[q][p] = A_[q][p] + 2.f * k[q];
            w = U_[q][p] + dt * k[q];
          } else {
            const float a = A_[q][p] + k[q];
            float l = TM ? lr[q][p] : pL[q * ncl + p];
            two_sum_acc(U_[q][p], l, __fmul_rn(h6, a));
            if constexpr (TM) lr[q][p] = l; else pL[q * ncl + p] = l;
            w = U_[q][p];
          }
          wout[q][p] = w;
        }
      }
    }
    if constexpr (TM) {
      // the state changes in Euler steps and the last RK stage, the
      // accumulator in the first three RK stages
      if (euler || STAGE == 3) {
        tm_st<NC * PX>(tm + (uint32_t)(r * NC * PX), &ur[0][0]);
        tm_st<NC * PX>(tm + (uint32_t)((2 * RS + r) * NC * PX), &lr[0][0]);
      } else {
        tm_st<NC * PX>(tm + (uint32_t)((RS + r) * NC * PX), &ar[0][0]);
      }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) st_vec<PX>(pBn + q * ncell, wout[q]);
    if (DIMS >= 2) {
      // edge rows are visited first: row 0 (walking up) or nloc - 1 (down);
      // a CTA with a single row group also sends its last row at r = RS - 1
      // (one test per row for all components)
      const bool e0 = r == 0 && ho.on && ho.edge;
      const bool e1 = r == RS - 1 && ho.on && ho.first && ho.last;
      if (e0 || e1) {
        const uint4 t = *ho.tab;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          if (e0) push_edge_q<KP, PX, WALL>(ho, t, ho.first, q * ncell + rowoff, wout[q], q);
          if (e1) push_edge_q<KP, PX, WALL>(ho, t, false, q * ncell + rowoff, wout[q], q);
        }
      }
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int p = 0; p < PX; ++p) { back[q][p] = cur[q][p]; cur[q][p] = ahead[q][p]; }
    }
    pB += rstep;
    pBn += rstep;
    if constexpr (!TM) pL += rstep;
    if (pT) pT += rstep;
  }
  if constexpr (TM) tm_wait_st();
}

// RK: the fine solver's RK4 (true) or the coarse forward Euler (false), one
// instantiation each, so the RK4 kernel carries no Euler code (registers).
// The body is shared by two kernels: k_stencil_mixed (up to 512 threads,
// 128 registers each) and k_stencil_mixed_wide (up to 800 threads capped at
// 80 registers, for slices whose CTA share leaves one CTA per SM: there the
// wider block holds twice the warps and a smaller register tile per thread).
template <int KP, int PX, int RS, bool XS, bool WALL, bool RK, bool TM, bool ISO>
__device__ __forceinline__ void mixed_body(const FusedParams& P) {
  constexpr int NC = KT<KP>::NC, DIMS = KT<KP>::DIMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CS = P.cluster;
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int item = blockIdx.x / CS;
  if (item >= P.it.n) return;                // uniform over the cluster
  if (P.it.gate && !P.it.gate[item]) return; // uniform over the cluster
  const int plane = P.plane, nx = P.nx, ny = P.ny;
  const int nloc = P.nloc;
  // shared memory: stage buffers 0/1, each [NC][nloc + 2][plane] (outer
  // rows -1 .. nloc; rows -1 and nloc are the ghost rows), the low words
  // [NC][nloc][plane], two mbarriers, the halo target table, abort flags
  const int ncell = P.mcell;   // (nloc + 2) * plane
  const int ncl = P.mcl;       // nloc * plane
  float* const buf0 = reinterpret_cast<float*>(smem_raw) + plane;   // row 0 of buffer 0
  float* const buf1 = buf0 + NC * ncell;
  // the low words (not with TM: they live in tensor memory)
  float* const ulo = TM ? nullptr : reinterpret_cast<float*>(smem_raw) + 2 * NC * ncell;
  // (P.moff = the 16-byte aligned end of the buffers: 4 (2 NC ncell + NC ncl);
  // after it 64 bytes: mbarriers, target table, flags, stop stages, TMEM base)
  uint64_t* const mbar = reinterpret_cast<uint64_t*>(smem_raw + P.moff);
  const bool remote = DIMS >= 2 && CS > 1;
  const uint32_t sbase = cta_smem_u32(smem_raw);
  const uint32_t mb0 = cta_smem_u32(mbar);
  if (remote && threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
  // y neighbours inside a 3D plane: periodic, or the row itself at a wall
  const int yn_row = yrow + 1 == ny ? (WALL ? yrow : 0) : yrow + 1;
  const int ys_row = yrow == 0 ? (WALL ? 0 : ny - 1) : yrow - 1;
  // offsets of the y neighbours from the tile's first cell (3D)
  const int dN = DIMS == 3 ? (yn_row - yrow) * nx : 0;
  const int dS = DIMS == 3 ? (ys_row - yrow) * nx : 0;
  // first cells of the tiles west and east of this one (periodic in x; at a
  // wall the value is replaced by the cell's own)
  const int dW = (xw + 1 - PX) - x0, dE = xe - x0;
  const bool xlo = WALL && x0 == 0, xhi = WALL && x0 + PX == nx;
  const bool first = o0 == 0, last = o0 + RS == nloc;
  const bool edge = DIMS >= 2 && (first || last);
  // the group owning the last row (unless it also owns the first) walks
  // downwards; register tile row r is outer row ofirst + dir * r
  const int dir = (last && !first) ? -1 : 1;
  const int ofirst = dir > 0 ? o0 : o0 + RS - 1;
  // x-neighbour shuffles: an x-row is xsw = nx / PX consecutive lanes
  const int xsw = nx / PX;
  const int xl = (int)(threadIdx.x & 31) & (xsw - 1);
  const int xwest = (xl + xsw - 1) & (xsw - 1), xeast = (xl + 1) & (xsw - 1);
  // lanes present in this warp (the last warp of a block whose size is not
  // a multiple of 32 is partial; it still holds whole x-rows)
  const int wl = min(32, (int)blockDim.x - (int)(threadIdx.x & ~31u));
  const unsigned xmask = wl >= 32 ? 0xffffffffu : ((1u << wl) - 1u);

  // halo targets: my first row is the previous rank's ghost row nloc, my
  // last row the next rank's ghost row -1 (buffer 0; +boff for buffer 1)
  uint4* const tab = reinterpret_cast<uint4*>(mbar + 2);
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(tab + 1);  // [2]
  // the stop stages of the previous and the next rank (written by them);
  // after them 16 bytes for the tensor-memory base (wide kernel)
  volatile int* const stop_in = abort_flag + 2;  // [2]
  // With no-flux walls the first rank's row 0 fills its own S ghost row and
  // the last rank's last row its own N ghost row (local stores, no mbarrier:
  // a zero mbarrier address in the table marks a local target).
  const bool wall_lo = WALL && rank == 0, wall_hi = WALL && rank == CS - 1;
  if (threadIdx.x == 0) {
    abort_flag[0] = abort_flag[1] = 0;
    uint32_t rb_prev = sbase, rb_next = sbase;
    if (remote) {
      rb_prev = cluster_map_u32(sbase, (rank + CS - 1) % CS);
      rb_next = cluster_map_u32(sbase, (rank + 1) % CS);
    }
    const uint32_t ghostN = (uint32_t)((nloc + 1) * plane) * 4u, mboff = mb0 - sbase;
    uint4 t = make_uint4(rb_prev + ghostN, rb_next, rb_prev + mboff, rb_next + mboff);
    if (wall_lo) { t.x = sbase; t.z = 0; }
    if (wall_hi) { t.y = sbase + ghostN; t.w = 0; }
    *tab = t;
  }
  auto halo_out = [&](int par, bool on) {
    HaloOut h;
    h.on = on;
    h.self = !remote;
    h.first = first; h.last = last; h.edge = edge;
    h.tab = tab;
    h.boff = (uint32_t)(par * NC * ncell) * 4u;
    h.moff = 8u * par;
    return h;
  };
  // ghost rows that arrive from other CTAs each stage
  const int n_remote = remote ? (wall_lo ? 0 : 1) + (wall_hi ? 0 : 1) : 0;
  const uint32_t tx_bytes = (uint32_t)(n_remote * NC * plane * 4);

  const long long base = (long long)rank * nloc * plane;
  const double* in = P.in + item_off(P.it.src_off, P.it.src_base, P.it.src_stride, item) + base;
  // shallow water over a bottom b: this CTA's rows of the bottom term
  const float* const bth =
      (KP == KP_SWE && P.coef.bath32) ? P.coef.bath32 + base : nullptr;
  float uh[RS][NC][PX], acc[RS][NC][PX];
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        const int o = ofirst + dir * r;
        const double v = in[q * P.n + o * plane + rowoff + p];
        const float h = (float)v;
        uh[r][q][p] = h;
        acc[r][q][p] = 0.f;
        buf0[q * ncell + o * plane + rowoff + p] = h;
        if constexpr (TM) acc[r][q][p] = (float)(v - (double)h);   // staged for TMEM
        else ulo[q * ncl + o * plane + rowoff + p] = (float)(v - (double)h);
      }
  // TM: P.tmcols TMEM columns for the CTA (a power of two of at least
  // 3 RS NC PX columns per warp times the warps sharing a lane quadrant:
  // step state, accumulator, low words), allocated by warp 0; the
  // allocation writes the base address to tm_base.  The host sizes the
  // columns so that the CTAs that can share an SM never ask for more than
  // its 512 (an allocation that had to wait could deadlock two clusters).
  volatile uint32_t* const tm_base = reinterpret_cast<volatile uint32_t*>(stop_in + 2);
  if constexpr (TM) {
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       cta_smem_u32(const_cast<uint32_t*>(tm_base))),
                   "r"((uint32_t)P.tmcols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // every CTA's mbarriers and target table are initialised before anyone
  // pushes
  if (CS > 1) cg::this_cluster().sync(); else __syncthreads();
  // this thread's TMEM columns: lane quadrant of its warp, column block of
  // its warp among those sharing the quadrant
  uint32_t tm = 0;
  if constexpr (TM) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t w = threadIdx.x >> 5;
    tm = *tm_base + ((32u * (w & 3u)) << 16) + (w >> 2) * (uint32_t)(3 * RS * NC * PX);
#pragma unroll
    for (int r = 0; r < RS; ++r) {
      tm_st<NC * PX>(tm + (uint32_t)(r * NC * PX), &uh[r][0][0]);
      tm_st<NC * PX>(tm + (uint32_t)((2 * RS + r) * NC * PX), &acc[r][0][0]);  // low words
    }
    tm_wait_st();
  }
  // stage 0's halo: the initial edge rows
  if (DIMS >= 2) {
    const HaloOut h0 = halo_out(0, true);
    const uint4 t0 = *h0.tab;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      // outer rows 0 and nloc - 1 sit in register rows 0 / RS - 1 or, walking
      // downwards, RS - 1 / 0
      float v0[PX], v1[PX];
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        v0[p] = dir > 0 ? uh[0][q][p] : uh[RS - 1][q][p];
        v1[p] = dir > 0 ? uh[RS - 1][q][p] : uh[0][q][p];
      }
      if (first) push_edge_q<KP, PX, WALL>(h0, t0, true, q * ncell + rowoff, v0, q);
      if (last) push_edge_q<KP, PX, WALL>(h0, t0, false, q * ncell + rowoff, v1, q);
    }
  }

  // Stage s reads buffer s & 1 (with its ghost rows) and writes buffer
  // (s + 1) & 1 and the neighbours' ghost rows of that buffer.  The ghost
  // rows of stage s are pushed by the neighbours during their stage s - 1
  // (stage 0's before the loop) and complete bytes on mbarrier s & 1, in
  // its phase of parity (s >> 1) & 1.  Thread 0 arms that phase one stage
  // ahead, at the start of stage s - 1 (the mbarrier's previous phase, stage
  // s - 2, completed before stage s - 2 began), and thread 0 waits for it
  // at the end of stage s - 1, with cluster-scope acquire, before the CTA
  // barrier that closes the stage (the barrier then orders the ghost rows
  // before every thread's reads of them: one cluster-scope acquire per CTA
  // and stage instead of one per thread that owns an edge row).  A CTA
  // whose wait gave up therefore stops before computing
  // stage s and pushes no further rows.  Since a CTA computes stage s only
  // after both neighbours' stage-s rows arrived, i.e. after both neighbours
  // computed stage s - 1, the stop stages of adjacent CTAs differ by at most
  // one, which bounds what can still be in flight (the drain below).
  const int nst = RK ? 4 * P.steps : P.steps;
  auto arm = [&](int s) {
    if (remote && s < nst && threadIdx.x == 0) mbar_expect(mb0 + 8u * (s & 1), tx_bytes);
  };
  auto wait_rows = [&](int s) {
    if (remote && s < nst && threadIdx.x == 0 &&
        !halo_wait(mb0 + 8u * (s & 1), (uint32_t)((s >> 1) & 1))) {
      abort_flag[s & 1] = 1;
      if (P.err) atomicExch(P.err, 1);
    }
  };
  // CTA barrier before stage s; true when a wait for the ghost rows of
  // stage s gave up.  The flag of stage s is written before this barrier
  // and read after it; the next write to it (stage s + 2) comes after the
  // barrier before stage s + 1, so every thread reads the same value and
  // stops at the same stage.
  auto gate = [&](int s) {
    __syncthreads();
    return abort_flag[s & 1] != 0;
  };
#define RNP_MIXED_STAGE(STG, BIN, BOUT, PAR, ON, EUL)                                          \
  mixed_stage<KP, PX, RS, STG, XS, WALL, TM, ISO>(P, BIN, BOUT, ulo, uh, acc, tm, ncell, plane, \
                                                  nloc,                                       \
                                         ofirst, dir, rowoff, dW, dE, dN, dS,                \
                                         EUL, halo_out((PAR) ^ 1, ON), xmask, xsw, xwest,    \
                                         xeast, xlo, xhi, bth)

  // first stage this CTA did not compute (nst: it computed them all)
  int stop = nst;
  arm(0);
  __syncthreads();
  wait_rows(0);
  if (gate(0)) stop = 0;
  for (int step = 0; step < P.steps && stop == nst; ++step) {
    if constexpr (RK) {
      const int s0 = 4 * step;
      arm(s0 + 1);
      RNP_MIXED_STAGE(0, buf0, buf1, 0, true, false);
      wait_rows(s0 + 1);
      if (gate(s0 + 1)) { stop = s0 + 1; break; }
      arm(s0 + 2);
      RNP_MIXED_STAGE(1, buf1, buf0, 1, true, false);
      wait_rows(s0 + 2);
      if (gate(s0 + 2)) { stop = s0 + 2; break; }
      arm(s0 + 3);
      RNP_MIXED_STAGE(2, buf0, buf1, 0, true, false);
      wait_rows(s0 + 3);
      if (gate(s0 + 3)) { stop = s0 + 3; break; }
      arm(s0 + 4);
      RNP_MIXED_STAGE(3, buf1, buf0, 1, s0 + 4 < nst, false);
      wait_rows(s0 + 4);
      if (gate(s0 + 4)) { stop = s0 + 4; break; }
    } else {
      // forward Euler: buffers alternate every step
      arm(step + 1);
      if ((step & 1) == 0)
        RNP_MIXED_STAGE(0, buf0, buf1, 0, step + 1 < nst, true);
      else
        RNP_MIXED_STAGE(0, buf1, buf0, 1, step + 1 < nst, true);
      wait_rows(step + 1);
      if (gate(step + 1)) { stop = step + 1; break; }
    }
  }
#undef RNP_MIXED_STAGE
  // Drain: no CTA leaves while a ghost-row store aimed at it may be in
  // flight.  Every CTA publishes its stop stage to both neighbours; after
  // the cluster barrier nobody pushes any more.  A neighbour with stop
  // stage sn sent the rows of every stage t <= sn (t < nst).  Pending at
  // this CTA are at most the armed phase of stage `stop` (bytes of a
  // neighbour that stopped earlier never come: they are counted as received)
  // and the unarmed phase of stage stop + 1 (armed now for the bytes of the
  // neighbours that computed stage `stop`); nothing of a later stage can
  // have been sent.  Thread 0 waits (bounded) for both, then the cluster
  // barrier below lets every CTA leave.  With no timeout anywhere every
  // stop stage is nst and nothing is pending.
  if (remote) {
    if (threadIdx.x == 0) {
      cg::cluster_group cl = cg::this_cluster();
      volatile int* to_prev = cl.map_shared_rank(const_cast<int*>(stop_in) + 1, (rank + CS - 1) % CS);
      volatile int* to_next = cl.map_shared_rank(const_cast<int*>(stop_in), (rank + 1) % CS);
      *to_prev = stop;
      *to_next = stop;
    }
    cg::this_cluster().sync();
    if (threadIdx.x == 0) {
      const int sp = wall_lo ? nst : stop_in[0];
      const int sn = wall_hi ? nst : stop_in[1];
      const uint32_t row = (uint32_t)(NC * plane * 4);
      bool ok = true;
      if (stop < nst) {
        const uint32_t mb = mb0 + 8u * (stop & 1), par = (uint32_t)((stop >> 1) & 1);
        if (!mbar_done(mb, par)) {
          const uint32_t missing = (!wall_lo && sp < stop ? row : 0u) +
                                   (!wall_hi && sn < stop ? row : 0u);
          if (missing) mbar_complete(mb, missing);
          ok = halo_wait(mb, par);
        }
      }
      if (stop + 1 < nst) {
        const uint32_t sent = (!wall_lo && sp > stop ? row : 0u) +
                              (!wall_hi && sn > stop ? row : 0u);
        if (sent) {
          const uint32_t mb = mb0 + 8u * ((stop + 1) & 1);
          mbar_expect(mb, sent);
          ok = halo_wait(mb, (uint32_t)(((stop + 1) >> 1) & 1)) && ok;
        }
      }
      if (!ok && P.err) atomicExch(P.err, 1);
    }
  }
  if (CS > 1) cg::this_cluster().sync();
  if constexpr (TM) {
    // the final state back from tensor memory, then the columns released
#pragma unroll
    for (int r = 0; r < RS; ++r) {
      tm_ld<NC * PX>(tm + (uint32_t)(r * NC * PX), &uh[r][0][0]);
      tm_ld<NC * PX>(tm + (uint32_t)((2 * RS + r) * NC * PX), &acc[r][0][0]);  // low words
      tm_wait_ld<NC * PX>(&uh[r][0][0]);
      tm_fence_ld<NC * PX>(&acc[r][0][0]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tm_base),
                   "r"((uint32_t)P.tmcols)
                   : "memory");
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
        const int o = ofirst + dir * r;
        const double v = (double)uh[r][q][p] +
                         (double)(TM ? acc[r][q][p] : ulo[q * ncl + o * plane + rowoff + p]);
        out[q * P.n + o * plane + rowoff + p] = v;
        if (out2) out2[q * P.n + o * plane + rowoff + p] = v;
      }
}

template <int KP, int PX, int RS, bool XS, bool WALL, bool RK>
__global__ void __launch_bounds__(512, 1) k_stencil_mixed(const __grid_constant__ FusedParams P) {
  mixed_body<KP, PX, RS, XS, WALL, RK, false, false>(P);
}

// Registers per thread of the wide kernel.  The register file is split
// evenly over the SM's four schedulers (16384 each) and a block's warps are
// dealt out among them, so 25 warps put 7 on one scheduler: 7 x 32 x 72 =
// 16128 registers fit, 80 would not.  Blocks of 128 to 800 threads launch
// (above 512 threads one block per SM; at 256 threads three).
static constexpr int kWideRegs = 72;
static constexpr int kWideThreads = 800;
static constexpr int kWideMinThreads = 128;

// The wide kernel keeps the step state, the accumulator and the low words in
// tensor memory (TM), which leaves the registers to the stencil's working
// rows, and requires equal grid spacing on every axis (ISO: a cheaper
// Laplacian with fewer constants); the host falls back to the other kernel
// otherwise.
template <int KP, int PX, int RS, bool XS, bool WALL, bool RK>
__global__ void __maxnreg__(kWideRegs) k_stencil_mixed_wide(const __grid_constant__ FusedParams P) {
  mixed_body<KP, PX, RS, XS, WALL, RK, true, true>(P);
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

template <int KP>
inline FusedFn fused_rk8_for_R(int R) {
  switch (R) {
    case 1: return k_stencil_fused_rk8<KP, 1>;
    case 2: return k_stencil_fused_rk8<KP, 2>;
    default: return nullptr;
  }
}

// Register tiles of more than kMaxTileValues state values per thread spill
// beyond use and are not instantiated (the host picker never asks for them).
static constexpr int kMaxTileValues = 40;

template <int KP, int PX, int RS, bool XS, bool WALL, bool RK>
inline FusedFn mixed_if_fits() {
  if constexpr (RS * KT<KP>::NC * PX <= kMaxTileValues)
    return k_stencil_mixed<KP, PX, RS, XS, WALL, RK>;
  else
    return nullptr;
}

template <int KP, int PX, bool XS, bool WALL, bool RK>
inline FusedFn mixed_for_RS(int RS) {
  switch (RS) {
    case 1: return mixed_if_fits<KP, PX, 1, XS, WALL, RK>();
    case 2: return mixed_if_fits<KP, PX, 2, XS, WALL, RK>();
    case 4: return mixed_if_fits<KP, PX, 4, XS, WALL, RK>();
    case 5: return mixed_if_fits<KP, PX, 5, XS, WALL, RK>();
    case 8: return mixed_if_fits<KP, PX, 8, XS, WALL, RK>();
    default: return nullptr;
  }
}

template <int KP, int PX, bool WALL, bool RK>
inline FusedFn mixed_for_xs(int RS, bool XS) {
  return XS ? mixed_for_RS<KP, PX, true, WALL, RK>(RS) : mixed_for_RS<KP, PX, false, WALL, RK>(RS);
}

template <int KP, int PX, bool RK>
inline FusedFn mixed_for_wall(int RS, bool XS, bool WALL) {
  return WALL ? mixed_for_xs<KP, PX, true, RK>(RS, XS) : mixed_for_xs<KP, PX, false, RK>(RS, XS);
}

template <int KP>
inline FusedFn mixed_for(int PX, int RS, bool XS, bool WALL, bool RK) {
  if (PX == 2) return RK ? mixed_for_wall<KP, 2, true>(RS, XS, WALL) : mixed_for_wall<KP, 2, false>(RS, XS, WALL);
  if (PX == 4) return RK ? mixed_for_wall<KP, 4, true>(RS, XS, WALL) : mixed_for_wall<KP, 4, false>(RS, XS, WALL);
  return nullptr;
}

// The wide kernel's instantiations: tiles of at most 20 state values per
// thread (3 x 20 TMEM columns per warp, at most 7 warps per lane quadrant:
// 420 of the 512 columns), periodic, x neighbours from shared memory (the
// configurations a wide block is picked for: a slice whose CTA share fills
// the shared memory).
template <int KP, bool RK>
inline FusedFn mixed_wide_for(int PX, int RS) {
  if (PX == 2 && RS == 1) return k_stencil_mixed_wide<KP, 2, 1, false, false, RK>;
  if (PX == 2 && RS == 2) return k_stencil_mixed_wide<KP, 2, 2, false, false, RK>;
  if (PX == 2 && RS == 4) return k_stencil_mixed_wide<KP, 2, 4, false, false, RK>;
  if (PX == 2 && RS == 5) return k_stencil_mixed_wide<KP, 2, 5, false, false, RK>;
  if (PX == 4 && RS == 1) return k_stencil_mixed_wide<KP, 4, 1, false, false, RK>;
  if (PX == 4 && RS == 2) return k_stencil_mixed_wide<KP, 4, 2, false, false, RK>;
  return nullptr;
}
// defined in stencil_wide.cu: the wide kernels of the reaction-diffusion
// operators on grids of equal spacing (nullptr for other operators, tiles
// and grids)
FusedFn mixed_wide_fn(int kp, int PX, int RS, bool XS, bool WALL, bool RK, bool iso);

// Per-PDE entry points, defined in stencil_<pde>.cu.
#define RNP_STENCIL_DECL(NAME)                 \
  FusedFn fused_fn_##NAME(int R);              \
  FusedFn fused_rk8_fn_##NAME(int R);          \
  FusedFn mixed_fn_##NAME(int PX, int RS, bool XS, bool WALL, bool RK); \
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

template <int KP, bool WALL>
inline FusedFn mixed_for_w(int PX, int RS, bool XS, bool RK) {
  if (PX == 2) return RK ? mixed_for_xs<KP, 2, WALL, true>(RS, XS) : mixed_for_xs<KP, 2, WALL, false>(RS, XS);
  if (PX == 4) return RK ? mixed_for_xs<KP, 4, WALL, true>(RS, XS) : mixed_for_xs<KP, 4, WALL, false>(RS, XS);
  return nullptr;
}

// Shallow water compiles its wall instantiations of the mixed kernel in a
// translation unit of their own (stencil_swe_wall.cu) so the two halves
// build in parallel.
FusedFn mixed_fn_swe_wall(int PX, int RS, bool XS, bool RK);

#define RNP_STENCIL_DEFINE_SPLIT(KPV, NAME)                                          \
  FusedFn fused_fn_##NAME(int R) { return fused_for_R<KPV, double, true>(R); }       \
  FusedFn fused_rk8_fn_##NAME(int R) { return fused_rk8_for_R<KPV>(R); }             \
  FusedFn mixed_fn_##NAME(int PX, int RS, bool XS, bool WALL, bool RK) {             \
    return WALL ? mixed_fn_##NAME##_wall(PX, RS, XS, RK)                             \
                : mixed_for_w<KPV, false>(PX, RS, XS, RK);                           \
  }                                                                                  \
  PlainFn plain_fn_##NAME() { return k_stage_plain<KPV>; }

#define RNP_STENCIL_DEFINE_WALL(KPV, NAME)                                           \
  FusedFn mixed_fn_##NAME##_wall(int PX, int RS, bool XS, bool RK) {                 \
    return mixed_for_w<KPV, true>(PX, RS, XS, RK);                                   \
  }

#define RNP_STENCIL_DEFINE(KPV, NAME)                                                \
  FusedFn fused_fn_##NAME(int R) { return fused_for_R<KPV, double, true>(R); }       \
  FusedFn fused_rk8_fn_##NAME(int R) { return fused_rk8_for_R<KPV>(R); }             \
  FusedFn mixed_fn_##NAME(int PX, int RS, bool XS, bool WALL, bool RK) {             \
    return mixed_for<KPV>(PX, RS, XS, WALL, RK);                                     \
  }                                                                                  \
  PlainFn plain_fn_##NAME() { return k_stage_plain<KPV>; }

}  // namespace rnp
