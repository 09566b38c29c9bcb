// stencil.cu -- fine (F, classic RK4 or eighth-order RK8) and coarse (G,
// forward Euler or RK4)
// propagators of Sec. 2 over the periodic finite-difference right-hand sides
// h(u) of Eq. 1 (Sec. 5.1 Burgers, Sec. 5.2 diffusion-reaction, App. E
// Brusselator, Sec. 5.3 shallow water, plus heat and advection operators).
//
// Fused path: one launch advances every work item (a slice start, or a
// batch member in the coarse sweep) through all of its steps.  Each item is
// owned by a thread-block cluster; the state is split along the outermost
// axis, each CTA keeps its block of the Runge-Kutta stage input in shared
// memory (double-buffered) and the step state u and stage accumulator in
// registers.  Neighbour planes across a CTA boundary are read straight from
// the neighbouring CTA's shared memory (distributed shared memory); one
// cluster barrier separates consecutive stages.  HBM is touched only to
// load the start state and store the end state.
//
// Plain path: one launch per Runge-Kutta stage over global memory.
//
// RK8 is the eleven-stage explicit eighth-order method of Cooper & Verner
// (SIAM J. Numer. Anal. 9, 1972), in FP64 only.
//
// FP64 variants evaluate every expression with explicitly rounded
// operations (no contraction), in the same order as the plain serial
// formulas, so F and G are bit-identical to a serial FP64 evaluation.  FP32
// variants let the compiler contract multiply-adds.
#include <cmath>
#include <cstdio>
#include <cstdarg>
#include <cstring>

#include "stencil_impl.cuh"

namespace rnp {

__global__ void k_plain_load(const double* in, const Items it, long long d, double* U,
                             double* W) {
  const long long tot = (long long)it.n * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int item = (int)(t / d);
    if (it.gate && !it.gate[item]) continue;
    const double v = in[item_off(it.src_off, it.src_base, it.src_stride, item) +
                        (t - (long long)item * d)];
    U[t] = v;
    W[t] = v;
  }
}

__global__ void k_plain_store(const double* U, const Items it, long long d, double* out,
                              double* out2) {
  const long long tot = (long long)it.n * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int item = (int)(t / d);
    if (it.gate && !it.gate[item]) continue;
    const long long e = t - (long long)item * d;
    out[item_off(it.dst_off, it.dst_base, it.dst_stride, item) + e] = U[t];
    if (out2) out2[item_off(it.dst2_off, it.dst2_base, it.dst2_stride, item) + e] = U[t];
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
Geom make_geom(const rnp_problem& p) {
  Geom g;
  g.nx = p.nx; g.ny = p.ny; g.nz = p.nz;
  g.n = (long long)p.nx * p.ny * p.nz;
  switch (p.pde) {
    case RNP_BURGERS1D: g.kp = KP_BURGERS; g.ncomp = 1; g.dims = 1; break;
    case RNP_ADVECT1D: g.kp = KP_ADVECT; g.ncomp = 1; g.dims = 1; break;
    case RNP_HEAT:
      g.ncomp = 1;
      g.dims = p.nz > 1 ? 3 : (p.ny > 1 ? 2 : 1);
      g.kp = g.dims == 1 ? KP_HEAT1 : (g.dims == 2 ? KP_HEAT2 : KP_HEAT3);
      break;
    case RNP_DIFFREACT2D: g.kp = KP_DIFFREACT; g.ncomp = 2; g.dims = 2; break;
    case RNP_BRUSS2D: g.kp = KP_BRUSS2; g.ncomp = 2; g.dims = 2; break;
    case RNP_BRUSS3D: g.kp = KP_BRUSS3; g.ncomp = 2; g.dims = 3; break;
    case RNP_SWE2D: g.kp = KP_SWE; g.ncomp = 3; g.dims = 2; break;
    default: g.kp = -1; g.ncomp = 1; g.dims = 1;
  }
  g.d = g.n * g.ncomp;
  g.iso = false;
  if (g.dims == 1) { g.outer = 1; g.plane = p.nx; }
  else if (g.dims == 2) { g.outer = p.ny; g.plane = p.nx; }
  else { g.outer = p.nz; g.plane = (long long)p.nx * p.ny; }
  g.bc = p.bc;
  // equal spacing on every axis of a reaction-diffusion operator (1/h^2
  // compared exactly as the kernels receive it)
  const Coef c = make_coef(p, g);
  if (g.kp == KP_BRUSS2 || g.kp == KP_BRUSS3)
    g.iso = c.k[5] == c.k[6] && (g.dims < 3 || c.k[6] == c.k[7]);
  else if (g.kp == KP_DIFFREACT)
    g.iso = c.k[3] == c.k[4];
  return g;
}

Coef make_coef(const rnp_problem& p, const Geom& g) {
  Coef c;
  memset(&c, 0, sizeof(c));
  const double hx = p.lx / p.nx, hy = p.ly / p.ny, hz = p.lz / p.nz;
  const double ix2 = 1.0 / (hx * hx), iy2 = 1.0 / (hy * hy), iz2 = 1.0 / (hz * hz);
  const double* P = p.param;
  switch (g.kp) {
    case KP_BURGERS: c.k[0] = P[0]; c.k[1] = ix2; c.k[2] = 0.5 / hx; break;
    case KP_ADVECT: c.k[0] = P[0]; c.k[1] = 0.5 / hx; break;
    case KP_HEAT1: case KP_HEAT2: case KP_HEAT3:
      c.k[0] = P[0]; c.k[1] = ix2; c.k[2] = iy2; c.k[3] = iz2; break;
    case KP_DIFFREACT:
      c.k[0] = P[0]; c.k[1] = P[1]; c.k[2] = P[2]; c.k[3] = ix2; c.k[4] = iy2;
      // diffusion coefficients over h^2 (equal spacing; mixed kernel only)
      c.k[5] = P[0] * ix2; c.k[6] = P[1] * ix2; break;
    case KP_BRUSS2: case KP_BRUSS3:
      c.k[0] = P[0]; c.k[1] = P[1]; c.k[2] = P[2]; c.k[3] = P[3];
      c.k[4] = 1.0 + P[1]; c.k[5] = ix2; c.k[6] = iy2; c.k[7] = iz2;
      c.k[8] = P[2] * ix2; c.k[9] = P[3] * ix2; break;
    case KP_SWE:
      c.k[0] = P[0]; c.k[1] = 0.5 * P[0]; c.k[2] = 1.0 / hx; c.k[3] = 1.0 / hy; break;
  }
  return c;
}

// The Cooper-Verner RK8 tableau from its published closed forms (rational
// numbers and rational combinations of sqrt(21)): a_{s,j} at
// rk[s*(s-1)/2 + j] for s = 1..10, j < s; b_0..b_10 at rk[55..65].
static void rk8_tableau(double* rk) {
  const double q = sqrt(21.0);
  double a[11][11] = {};
  a[1][0] = 1.0 / 2.0;
  a[2][0] = 1.0 / 4.0;  a[2][1] = 1.0 / 4.0;
  a[3][0] = 1.0 / 7.0;  a[3][1] = (-7.0 - 3.0 * q) / 98.0;  a[3][2] = (21.0 + 5.0 * q) / 49.0;
  a[4][0] = (11.0 + q) / 84.0;  a[4][2] = (18.0 + 4.0 * q) / 63.0;
  a[4][3] = (21.0 - q) / 252.0;
  a[5][0] = (5.0 + q) / 48.0;  a[5][2] = (9.0 + q) / 36.0;
  a[5][3] = (-231.0 + 14.0 * q) / 360.0;  a[5][4] = (63.0 - 7.0 * q) / 80.0;
  a[6][0] = (10.0 - q) / 42.0;  a[6][2] = (-432.0 + 92.0 * q) / 315.0;
  a[6][3] = (633.0 - 145.0 * q) / 90.0;  a[6][4] = (-504.0 + 115.0 * q) / 70.0;
  a[6][5] = (63.0 - 13.0 * q) / 35.0;
  a[7][0] = 1.0 / 14.0;  a[7][4] = (14.0 - 3.0 * q) / 126.0;
  a[7][5] = (13.0 - 3.0 * q) / 63.0;  a[7][6] = 1.0 / 9.0;
  a[8][0] = 1.0 / 32.0;  a[8][4] = (91.0 - 21.0 * q) / 576.0;  a[8][5] = 11.0 / 72.0;
  a[8][6] = (-385.0 - 75.0 * q) / 1152.0;  a[8][7] = (63.0 + 13.0 * q) / 128.0;
  a[9][0] = 1.0 / 14.0;  a[9][4] = 1.0 / 9.0;  a[9][5] = (-733.0 - 147.0 * q) / 2205.0;
  a[9][6] = (515.0 + 111.0 * q) / 504.0;  a[9][7] = (-51.0 - 11.0 * q) / 56.0;
  a[9][8] = (132.0 + 28.0 * q) / 245.0;
  a[10][4] = (-42.0 + 7.0 * q) / 18.0;  a[10][5] = (-18.0 + 28.0 * q) / 45.0;
  a[10][6] = (-273.0 - 53.0 * q) / 72.0;  a[10][7] = (301.0 + 53.0 * q) / 72.0;
  a[10][8] = (28.0 - 28.0 * q) / 45.0;  a[10][9] = (49.0 - 7.0 * q) / 18.0;
  for (int s = 1; s <= 10; ++s)
    for (int j = 0; j < s; ++j) rk[s * (s - 1) / 2 + j] = a[s][j];
  double* b = rk + 55;
  for (int j = 0; j < 11; ++j) b[j] = 0.0;
  b[0] = 1.0 / 20.0;
  b[7] = 49.0 / 180.0;
  b[8] = 16.0 / 45.0;
  b[9] = 49.0 / 180.0;
  b[10] = 1.0 / 20.0;
}

static FusedFn fused_rk8_fn(int kp, int R) {
  switch (kp) {
    case KP_BURGERS: return fused_rk8_fn_burgers(R);
    case KP_ADVECT: return fused_rk8_fn_advect(R);
    case KP_HEAT1: return fused_rk8_fn_heat1(R);
    case KP_HEAT2: return fused_rk8_fn_heat2(R);
    case KP_HEAT3: return fused_rk8_fn_heat3(R);
    case KP_DIFFREACT: return fused_rk8_fn_diffreact(R);
    case KP_BRUSS2: return fused_rk8_fn_bruss2(R);
    case KP_BRUSS3: return fused_rk8_fn_bruss3(R);
    case KP_SWE: return fused_rk8_fn_swe(R);
  }
  return nullptr;
}

// The FP64 fused kernel (every operation explicitly rounded).
static FusedFn fused_fn(int kp, int R) {
  switch (kp) {
    case KP_BURGERS: return fused_fn_burgers(R);
    case KP_ADVECT: return fused_fn_advect(R);
    case KP_HEAT1: return fused_fn_heat1(R);
    case KP_HEAT2: return fused_fn_heat2(R);
    case KP_HEAT3: return fused_fn_heat3(R);
    case KP_DIFFREACT: return fused_fn_diffreact(R);
    case KP_BRUSS2: return fused_fn_bruss2(R);
    case KP_BRUSS3: return fused_fn_bruss3(R);
    case KP_SWE: return fused_fn_swe(R);
  }
  return nullptr;
}

// x-neighbours by warp shuffles when an x-row of PX-point tiles spans a
// power-of-two number of lanes that divides the warp
static bool x_shuffles(const Geom& g, int PX) {
  const int w = g.nx / PX;
  return w >= 1 && w <= 32 && (32 % w) == 0;
}

static FusedFn mixed_fn_narrow(int kp, int PX, int RS, bool XS, bool WALL, bool RK) {
  switch (kp) {
    case KP_BURGERS: return mixed_fn_burgers(PX, RS, XS, WALL, RK);
    case KP_ADVECT: return mixed_fn_advect(PX, RS, XS, WALL, RK);
    case KP_HEAT1: return mixed_fn_heat1(PX, RS, XS, WALL, RK);
    case KP_HEAT2: return mixed_fn_heat2(PX, RS, XS, WALL, RK);
    case KP_HEAT3: return mixed_fn_heat3(PX, RS, XS, WALL, RK);
    case KP_DIFFREACT: return mixed_fn_diffreact(PX, RS, XS, WALL, RK);
    case KP_BRUSS2: return mixed_fn_bruss2(PX, RS, XS, WALL, RK);
    case KP_BRUSS3: return mixed_fn_bruss3(PX, RS, XS, WALL, RK);
    case KP_SWE: return mixed_fn_swe(PX, RS, XS, WALL, RK);
  }
  return nullptr;
}

// The mixed kernel: tm selects the wide instantiation (72 registers per
// thread, state in tensor memory, equal grid spacing only, 128..800
// threads), otherwise the 512-thread one.
static FusedFn mixed_fn(const Geom& g, int PX, int RS, bool XS, bool WALL, bool RK,
                        int threads, bool tm) {
  if (tm)
    return threads >= kWideMinThreads && threads <= kWideThreads && threads % 32 == 0
               ? mixed_wide_fn(g.kp, PX, RS, XS, WALL, RK, g.iso)
               : nullptr;
  return threads <= 512 ? mixed_fn_narrow(g.kp, PX, RS, XS, WALL, RK) : nullptr;
}

// Tensor-memory columns of a wide-kernel CTA: a power of two (>= 32) of at
// least 3 RS ncomp PX columns (step state, accumulator, low words) per warp
// times the warps that share a lane quadrant; 0 when the CTA may not take
// them.  tcgen05.alloc waits while the SM's 512 columns are taken, and a
// CTA waiting there inside a cluster can deadlock against another cluster
// holding columns, so co-resident CTAs must never ask for more than 512.
// Wide CTAs (72 registers per thread) claim at most their share of the
// register file in columns (512 x threads x 72 / 65536), so any set of
// them that fits an SM's registers fits its tensor memory; a CTA above 512
// threads may take all 512 columns, because the registers it leaves
// cannot hold another wide CTA (of at least 128 threads).  (The feature
// map's 128 columns ride on its own 195-register threads: a feature CTA and
// wide CTAs fitting one SM's registers stay within 512 columns too.)
static int tm_columns(const Geom& g, int PX, int RS, int threads) {
  const int nwq = ((threads / 32) + 3) / 4;
  const int need = 3 * RS * g.ncomp * PX * nwq;
  int cols = 32;
  while (cols < need) cols *= 2;
  if (cols > 512) return 0;
  const bool alone = 65536 - threads * kWideRegs < kWideMinThreads * kWideRegs;
  if (!alone && (long long)cols * 65536 > 512LL * threads * kWideRegs) return 0;
  return cols;
}

static const int kRs[] = {1, 2, 4, 8, 16};
static const int kMaxSmem = 220 * 1024;

static int round_R(long long cells_per_thread) {
  for (int R : kRs)
    if (R >= cells_per_thread) return R;
  return -1;
}

// Byte offset of the mixed kernel's mbarriers: the 16-byte aligned end of
// its two stage buffers (with two ghost rows each) and, unless the low words
// live in tensor memory (the wide kernel, tm), the low words.
static size_t mixed_tail_offset(const Geom& g, int CS, bool tm) {
  const long long ncell = (long long)(g.outer / CS) * g.plane;
  const size_t f = (2 * (size_t)g.ncomp * (ncell + 2 * g.plane) +
                    (tm ? 0 : (size_t)g.ncomp * ncell)) * 4;
  return (f + 15) & ~(size_t)15;
}

static size_t smem_bytes(const Geom& g, bool fp32, int CS, bool tm = false) {
  const long long ncell = (long long)(g.outer / CS) * g.plane;
  // FP64 kernel: two stage buffers; mixed kernel: the buffers above, then
  // two mbarriers, the 16-byte halo target table, two abort flags, the
  // neighbours' two stop stages and the tensor-memory base (64 bytes)
  if (!fp32) return 2 * (size_t)g.ncomp * ncell * 8;
  return mixed_tail_offset(g, CS, tm) + 64;
}

// Why the configurations tried were not launchable (for error messages):
// the first reasons of the current pick, appended.
static thread_local char g_unlaunchable[384] = "";
static void note_unlaunchable(const char* fmt, ...) __attribute__((format(printf, 1, 2)));
static void note_unlaunchable(const char* fmt, ...) {
  const size_t n = strlen(g_unlaunchable);
  if (n + 8 >= sizeof(g_unlaunchable)) return;
  char* p = g_unlaunchable + n;
  size_t left = sizeof(g_unlaunchable) - n;
  if (n) { snprintf(p, left, "; "); p += 2; left -= 2; }
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(p, left, fmt, ap);
  va_end(ap);
}

static bool launchable(FusedFn fn, int CS, int threads, size_t smem, int nitems) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    note_unlaunchable("no current device");
    cudaGetLastError();
    return false;
  }
  // the kernel's static shared memory (the wide kernel's tensor-memory base)
  // comes out of the same per-block limit as the dynamic part
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)fn) != cudaSuccess) {
    cudaGetLastError();
    note_unlaunchable("no attributes for the kernel");
    return false;
  }
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if ((long long)smem > dyn_max) {
    note_unlaunchable("%zu B of shared memory > %d", smem, dyn_max);
    return false;
  }
  if (threads > fa.maxThreadsPerBlock) {
    note_unlaunchable("%d threads > %d per block for this kernel (%d registers)", threads,
                      fa.maxThreadsPerBlock, fa.numRegs);
    return false;
  }
  // The limit is a per-function attribute shared by every configuration that
  // maps to this instantiation, so it is raised to the device maximum once
  // rather than set to this configuration's size.
  cudaError_t e = cudaFuncSetAttribute((const void*)fn,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e != cudaSuccess) {
    note_unlaunchable("shared-memory attribute: %s",
             cudaGetErrorString(e));
    cudaGetLastError();
    return false;
  }
  if (CS > 8 &&
      (e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                1)) != cudaSuccess) {
    note_unlaunchable("cluster-size attribute: %s",
             cudaGetErrorString(e));
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.gridDim = dim3(CS * (nitems > 0 ? nitems : 1));
  lc.blockDim = dim3(threads);
  lc.dynamicSmemBytes = smem;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  int nclusters = 0;
  if ((e = cudaOccupancyMaxActiveClusters(&nclusters, (const void*)fn, &lc)) != cudaSuccess) {
    note_unlaunchable("occupancy query: %s",
             cudaGetErrorString(e));
    cudaGetLastError();
    return false;
  }
  if (nclusters < 1)
    note_unlaunchable("no cluster of %d CTAs x %d threads with %zu B of shared memory fits", CS,
             threads, smem);
  return nclusters >= 1;
}

static thread_local int g_tile_relax = 0;  // 1: allow register tiles that spill a little

static bool try_cfg(const Geom& g, bool fp32, int CS, int threads, int nitems,
                    StencilCfg* out, int want_px = 0, int want_rs = 0, bool rk8 = false,
                    int want_tm = -1) {
  if (g.outer % CS) return false;
  if (g.dims == 1 && CS != 1) return false;
  const long long nloc = g.outer / CS;
  const long long ncell = nloc * g.plane;
  const size_t smem_n = smem_bytes(g, fp32, CS), smem_t = smem_bytes(g, fp32, CS, true);
  if (fp32 && smem_t <= (size_t)kMaxSmem) {
    // mixed kernel: PX x-points by RS rows per thread; the most threads
    // (up to 512) whose register tile fits, or exactly `threads` if given
    const int pxs[] = {2, 4};
    const int rss[] = {1, 2, 4, 5, 8};
    for (int PX : pxs) {
      if (g.nx % PX || (want_px && PX != want_px)) continue;
      const long long tiles = g.plane / PX;
      for (int RS : rss) {
        if (nloc % RS || (want_rs && RS != want_rs)) continue;
        // register tile measured spill-free with ptxas at 512 threads (the
        // relaxed pass accepts tiles that spill a little: still far faster
        // than the FP64 kernel on GB300's FP64 units)
        int budget = (g.dims <= 2 && g.ncomp <= 2) ? 16 : 8;
        if (g_tile_relax == 1) budget = 24;
        if (g_tile_relax == 2) budget = 40;
        if (RS * g.ncomp * PX > budget) continue;
        const long long t = tiles * (nloc / RS);
        if (t > kWideThreads || t < 1) continue;
        if (threads > 0 && t != threads) continue;
        // up to 512 threads the 512-thread kernel first (on the 2D
        // workloads the autotuner measured it faster), then the wide kernel
        // (state in tensor memory); above 512 threads only the wide kernel.
        // The wide kernel's tensor-memory accesses are warp-collective
        // (whole warps only) and its low words live in tensor memory (less
        // shared memory)
        for (int k = 0; k < 2; ++k) {
          const int tm = t > 512 ? 1 - k : k;
          if (want_tm >= 0 && tm != want_tm) continue;
          const int cols = tm ? tm_columns(g, PX, RS, (int)t) : 0;
          if (tm && cols == 0) continue;
          const size_t smem = tm ? smem_t : smem_n;
          if (smem > (size_t)kMaxSmem) continue;
          // the RK4 and the Euler instantiation of this tile (the RK4 one
          // is the larger: it decides launchability)
          FusedFn fn = mixed_fn(g, PX, RS, x_shuffles(g, PX), g.bc != 0, true, (int)t, tm);
          FusedFn fe = mixed_fn(g, PX, RS, x_shuffles(g, PX), g.bc != 0, false, (int)t, tm);
          if (!fn || !fe || !launchable(fn, CS, (int)t, smem, nitems) ||
              !launchable(fe, CS, (int)t, smem, nitems))
            continue;
          out->cluster = CS;
          out->threads = (int)t;
          out->R = 0;
          out->px = PX;
          out->rs = RS;
          out->tm = tm;
          return true;
        }
      }
    }
    return false;
  }
  if (fp32) return false;
  if (smem_bytes(g, false, CS) > (size_t)kMaxSmem) return false;
  if (rk8) {
    // RK8 kernel: the ten stage derivatives of each cell live in registers,
    // so a thread owns at most two cells
    if (threads <= 0) {
      long long t = (ncell + 1) / 2;
      t = ((t + 31) / 32) * 32;
      if (t < 32) t = 32;
      threads = (int)t;
    }
    if (threads > 512) return false;
    const long long per = (ncell + threads - 1) / threads;
    const int R = per <= 1 ? 1 : (per <= 2 ? 2 : -1);
    if (R < 0) return false;
    FusedFn fn = fused_rk8_fn(g.kp, R);
    if (!fn || !launchable(fn, CS, threads, smem_bytes(g, false, CS), nitems)) return false;
    out->cluster = CS;
    out->threads = threads;
    out->R = R;
    out->px = out->rs = 0;
    out->tm = 0;
    return true;
  }
  if (threads <= 0) {
    // enough threads that every thread owns <= 4 points
    long long t = (ncell + 3) / 4;
    t = ((t + 31) / 32) * 32;
    if (t < 64) t = 64;
    if (t > 512) t = 512;
    threads = (int)t;
  }
  const int R = round_R((ncell + threads - 1) / threads);
  if (R < 0) return false;
  FusedFn fn = fused_fn(g.kp, R);
  if (!fn || !launchable(fn, CS, threads, smem_bytes(g, false, CS), nitems)) return false;
  out->cluster = CS;
  out->threads = threads;
  out->R = R;
  out->px = out->rs = 0;
  out->tm = 0;
  return true;
}

static bool pick_one(const Geom& g, bool fp32, int nitems, bool latency, int want_cluster,
                     int want_threads, StencilCfg* out, char* why, int why_len, bool rk8);

bool pick_stencil(const Geom& g, bool fp32, int nitems, bool latency, int want_cluster,
                  int want_threads, StencilCfg* out, char* why, int why_len, bool rk8) {
  g_unlaunchable[0] = 0;
  if (rk8) return pick_one(g, false, nitems, latency, want_cluster, want_threads, out, why,
                           why_len, true);
  // a mixed-precision context prefers an FP32 tile at any cluster size and
  // falls back to the FP64 kernel only when no FP32 tile fits
  if (fp32) {
    g_tile_relax = 0;
    if (pick_one(g, true, nitems, latency, want_cluster, want_threads, out, why, why_len, false))
      return true;
    for (int level = 1; level <= 2; ++level) {
      g_tile_relax = level;
      const bool ok = pick_one(g, true, nitems, latency, want_cluster, want_threads, out, why,
                               why_len, false);
      g_tile_relax = 0;
      if (ok) return true;
    }
  }
  return pick_one(g, false, nitems, latency, want_cluster, want_threads, out, why, why_len,
                  false);
}

static bool pick_one(const Geom& g, bool fp32, int nitems, bool latency, int want_cluster,
                     int want_threads, StencilCfg* out, char* why, int why_len, bool rk8) {
  if (want_cluster > 0) {
    if (try_cfg(g, fp32, want_cluster, want_threads, nitems, out, 0, 0, rk8)) return true;
    snprintf(why, why_len, "stencil configuration cluster=%d threads=%d is not launchable (%s)",
             want_cluster, want_threads, g_unlaunchable[0] ? g_unlaunchable : "no tile of that size");
    return false;
  }
  // every cluster size up to 16 that divides the split axis; the smallest
  // that fits, or for latency the largest up to 8 (16 when nothing smaller fits)
  int cands[16], nc = 0;
  for (int CS = 1; CS <= 16; ++CS)
    if (g.outer % CS == 0) cands[nc++] = CS;
  int best = -1;
  for (int ci = 0; ci < nc; ++ci) {
    const int CS = cands[ci];
    StencilCfg c;
    if (!try_cfg(g, fp32, CS, want_threads, nitems, &c, 0, 0, rk8)) continue;
    if (best < 0) { *out = c; best = CS; if (!latency) break; }
    else if (latency && CS <= 8) { *out = c; best = CS; }
  }
  if (best < 0) {
    if (rk8)
      snprintf(why, why_len,
               "the fused RK8 kernel holds at most 2 x 512 cells per CTA of a 16-CTA cluster "
               "(state of %lld unknowns); use the plain execution",
               (long long)g.d);
    else
      snprintf(why, why_len,
               "state of %lld unknowns does not fit the shared memory of a 16-CTA cluster",
               (long long)g.d);
    return false;
  }
  // throughput: grow the cluster while the grid is below one CTA per SM
  if (!latency) {
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int ci = 0; ci < nc; ++ci) {
      const int CS = cands[ci];
      if (CS <= out->cluster || CS > 8 || (long long)nitems * CS > sms) continue;
      StencilCfg c;
      if (try_cfg(g, fp32, CS, want_threads, nitems, &c, 0, 0, rk8)) *out = c;
    }
  }
  return true;
}

int list_stencil_cfgs(const Geom& g, bool fp32, int nitems, StencilCfg* out, int maxn,
                      bool rk8) {
  int n = 0;
  // FP32: the spill-free tiles; where fewer than three exist (slices whose
  // CTA share leaves little room), also the wide and the register-tight
  // tiles, level by level, so that the timing decides between them
  for (int level = 0; level <= (fp32 ? 2 : 0); ++level) {
    g_tile_relax = level;
    n = 0;
    for (int CS = 1; CS <= 16 && n < maxn; ++CS) {
      if (g.outer % CS) continue;
      if (fp32) {
        const int pxs[] = {2, 4};
        const int rss[] = {1, 2, 4, 5, 8};
        for (int PX : pxs)
          for (int RS : rss) {
            if (n >= maxn) break;
            if (g.nx % PX || (g.outer / CS) % RS) continue;
            const long long t = (g.plane / PX) * ((g.outer / CS) / RS);
            for (int tm = 1; tm >= 0 && n < maxn; --tm) {
              StencilCfg c;
              if (t >= 32 && t <= kWideThreads &&
                  try_cfg(g, true, CS, (int)t, nitems, &c, PX, RS, false, tm))
                out[n++] = c;
            }
          }
      } else {
        StencilCfg c;
        if (try_cfg(g, false, CS, 0, nitems, &c, 0, 0, rk8)) out[n++] = c;
      }
    }
    if (n >= 3) break;
  }
  g_tile_relax = 0;
  return n;
}

cudaError_t launch_stencil_fused(const Geom& g, const Coef& c, bool fp32, int scheme,
                                 int steps, double dt, const double* in, double* out,
                                 double* out2, const Items& it, const StencilCfg& cfg,
                                 cudaStream_t st, int* err) {
  if (it.n <= 0 || steps <= 0) return cudaSuccess;
  // a mixed-precision context uses the FP64 kernel where no FP32 tile fits
  const bool use_mixed = fp32 && cfg.px > 0;
  const bool tm = use_mixed && cfg.tm;
  if (scheme == SCHEME_RK8 && use_mixed) return cudaErrorInvalidValue;  // FP64 only
  FusedFn fn = use_mixed ? mixed_fn(g, cfg.px, cfg.rs, x_shuffles(g, cfg.px), g.bc != 0,
                                    scheme == SCHEME_RK4, cfg.threads, tm)
               : scheme == SCHEME_RK8 ? fused_rk8_fn(g.kp, cfg.R)
                                      : fused_fn(g.kp, cfg.R);
  if (!fn) return cudaErrorInvalidValue;
  FusedParams P;
  P.in = in; P.out = out; P.out2 = out2;
  P.it = it;
  P.nx = g.nx; P.ny = g.ny; P.n = g.n; P.outer = g.outer; P.plane = (int)g.plane;
  P.cluster = cfg.cluster; P.steps = steps; P.scheme = scheme;
  P.dt = dt; P.h2 = dt / 2.0; P.h6 = dt / 6.0;
  P.coef = c;
  for (int i = 0; i < 12; ++i) P.kf[i] = (float)c.k[i];
  P.fdt = (float)P.dt; P.fh2 = (float)P.h2; P.fh6 = (float)P.h6;
  P.err = err;
  P.bc = g.bc;
  P.nloc = g.outer / cfg.cluster;
  P.mcell = (P.nloc + 2) * (int)g.plane;
  P.mcl = P.nloc * (int)g.plane;
  P.moff = use_mixed ? (int)mixed_tail_offset(g, cfg.cluster, tm) : 0;
  P.tmcols = tm ? tm_columns(g, cfg.px, cfg.rs, cfg.threads) : 0;
  if (tm && P.tmcols == 0) return cudaErrorInvalidValue;
  if (scheme == SCHEME_RK8) rk8_tableau(P.rk);
  else memset(P.rk, 0, sizeof(P.rk));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.gridDim = dim3(cfg.cluster * it.n);
  lc.blockDim = dim3(cfg.threads);
  lc.dynamicSmemBytes = smem_bytes(g, use_mixed, cfg.cluster, tm);
  lc.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cfg.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  count_launches(1);
  return cudaLaunchKernelEx(&lc, fn, P);
}

static PlainFn plain_fn(int kp) {
  switch (kp) {
    case KP_BURGERS: return plain_fn_burgers();
    case KP_ADVECT: return plain_fn_advect();
    case KP_HEAT1: return plain_fn_heat1();
    case KP_HEAT2: return plain_fn_heat2();
    case KP_HEAT3: return plain_fn_heat3();
    case KP_DIFFREACT: return plain_fn_diffreact();
    case KP_BRUSS2: return plain_fn_bruss2();
    case KP_BRUSS3: return plain_fn_bruss3();
    case KP_SWE: return plain_fn_swe();
  }
  return nullptr;
}

static int grid_for(long long tot, int threads) {
  long long b = (tot + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

long long plain_work_doubles(int scheme, long long items_d) {
  return (scheme == SCHEME_RK8 ? 14 : 4) * items_d;
}

cudaError_t launch_stencil_plain(const Geom& g, const Coef& c, int scheme, int steps,
                                 double dt, const double* in, double* out, double* out2,
                                 const Items& it, double* work, cudaStream_t st) {
  if (it.n <= 0 || steps <= 0) return cudaSuccess;
  PlainFn fn = plain_fn(g.kp);
  if (!fn) return cudaErrorInvalidValue;
  const long long tot = (long long)it.n * g.d;
  double* U = work;
  double* Acc = work + tot;
  double* Wb[2] = {work + 2 * tot, work + 3 * tot};
  count_launches(1);
  k_plain_load<<<grid_for(tot, 256), 256, 0, st>>>(in, it, g.d, U, Wb[0]);
  PlainParams P;
  P.U = U; P.Acc = Acc; P.gate = it.gate; P.nitems = it.n;
  P.nx = g.nx; P.ny = g.ny; P.nz = g.nz; P.n = g.n; P.d = g.d;
  P.scheme = scheme; P.dt = dt; P.h2 = dt / 2.0; P.h6 = dt / 6.0; P.coef = c;
  P.bc = g.bc;
  P.Kst = work + 4 * tot;   // RK8 only: ten more state-sized arrays
  if (scheme == SCHEME_RK8) rk8_tableau(P.rk);
  else memset(P.rk, 0, sizeof(P.rk));
  const int S = scheme == SCHEME_RK8 ? 11 : (scheme == SCHEME_RK4 ? 4 : 1);
  const long long cells = (long long)it.n * g.n;
  int cur = 0;
  for (int step = 0; step < steps; ++step)
    for (int s = 0; s < S; ++s) {
      P.Wc = Wb[cur];
      P.Wn = Wb[cur ^ 1];
      P.stage = s;
      count_launches(1);
      fn<<<grid_for(cells, 256), 256, 0, st>>>(P);
      cur ^= 1;
    }
  count_launches(1);
  k_plain_store<<<grid_for(tot, 256), 256, 0, st>>>(U, it, g.d, out, out2);
  return cudaGetLastError();
}

}  // namespace rnp
