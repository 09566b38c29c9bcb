/*
 * rnp_oracle.c -- FP64 CPU oracle for RandNet-Parareal.  TEST
 * INFRASTRUCTURE ONLY (see rnp_oracle.h).  Plain loops, evaluated in the
 * order written; build with -O2 -ffp-contract=off.
 */
#include "rnp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int orc_ncomp(const orc_problem* p) {
  switch (p->pde) {
    case ORC_DIFFREACT2D: case ORC_BRUSS2D: case ORC_BRUSS3D: return 2;
    case ORC_SWE2D: return 3;
    default: return 1;
  }
}

long orc_dim(const orc_problem* p) {
  return (long)orc_ncomp(p) * p->nx * p->ny * p->nz;
}

/* ------------------------------------------------------------------ */
/* Right-hand sides h(u) of Eq. 1 (periodic finite differences).       */
/* Layout: component-major, then z, then y, then x (x fastest).        */
/* ------------------------------------------------------------------ */

/* Second difference along each axis, summed x + y + z:
 *   ((f[+1] - 2 f) + f[-1]) * (1 / h^2) per axis. */
/* Index of the neighbour of cell i (0 <= i < n) in direction dir (+1/-1):
 * periodic wrap, or -- no-flux wall -- the cell itself. */
static int nbr(int i, int dir, int n, int bc) {
  int j = i + dir;
  if (j >= 0 && j < n) return j;
  if (bc == ORC_BC_NEUMANN) return i;
  return j < 0 ? j + n : j - n;
}

static double lap(const double* f, int x, int y, int z, int nx, int ny,
                  int nz, int dims, double ix2, double iy2, double iz2, int bc) {
  long row = ((long)z * ny + y) * nx;
  double c = f[row + x];
  double fe = f[row + nbr(x, 1, nx, bc)], fw = f[row + nbr(x, -1, nx, bc)];
  double s = ((fe - 2.0 * c) + fw) * ix2;
  if (dims >= 2) {
    double fn = f[((long)z * ny + nbr(y, 1, ny, bc)) * nx + x];
    double fs = f[((long)z * ny + nbr(y, -1, ny, bc)) * nx + x];
    s = s + ((fn - 2.0 * c) + fs) * iy2;
  }
  if (dims >= 3) {
    double fu = f[((long)nbr(z, 1, nz, bc) * ny + y) * nx + x];
    double fd = f[((long)nbr(z, -1, nz, bc) * ny + y) * nx + x];
    s = s + ((fu - 2.0 * c) + fd) * iz2;
  }
  return s;
}

/* Rusanov (local Lax-Friedrichs) numerical flux of the shallow-water
 * system across one face, direction dir (0: x, 1: y).  L and R are the
 * conserved states (h, hu, hv) on either side. */
static void swe_flux(double g, int dir, const double* L, const double* R,
                     double* F) {
  double hg = 0.5 * g;
  double uL = L[1] / L[0], vL = L[2] / L[0];
  double uR = R[1] / R[0], vR = R[2] / R[0];
  double FL[3], FR[3], sL, sR;
  if (dir == 0) {
    FL[0] = L[1]; FL[1] = L[1] * uL + (hg * L[0]) * L[0]; FL[2] = L[2] * uL;
    FR[0] = R[1]; FR[1] = R[1] * uR + (hg * R[0]) * R[0]; FR[2] = R[2] * uR;
    sL = fabs(uL) + sqrt(g * L[0]);
    sR = fabs(uR) + sqrt(g * R[0]);
  } else {
    FL[0] = L[2]; FL[1] = L[1] * vL; FL[2] = L[2] * vL + (hg * L[0]) * L[0];
    FR[0] = R[2]; FR[1] = R[1] * vR; FR[2] = R[2] * vR + (hg * R[0]) * R[0];
    sL = fabs(vL) + sqrt(g * L[0]);
    sR = fabs(vR) + sqrt(g * R[0]);
  }
  double a = sL > sR ? sL : sR;
  for (int q = 0; q < 3; ++q)
    F[q] = 0.5 * (FL[q] + FR[q]) - (0.5 * a) * (R[q] - L[q]);
}

void orc_rhs(const orc_problem* p, const double* u, double* out) {
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const long n = (long)nx * ny * nz;
  const double hx = p->lx / nx, hy = p->ly / ny, hz = p->lz / nz;
  const double ix2 = 1.0 / (hx * hx), iy2 = 1.0 / (hy * hy),
               iz2 = 1.0 / (hz * hz);
  const double* P = p->param;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long i = ((long)z * ny + y) * nx + x;
        switch (p->pde) {
          case ORC_BURGERS1D: {
            /* nu * v_xx - v * v_x, central differences (Sec. 5.1). */
            double i2h = 0.5 / hx;
            double v = u[i], ve = u[nbr(x, 1, nx, p->bc)], vw = u[nbr(x, -1, nx, p->bc)];
            double diff = P[0] * lap(u, x, 0, 0, nx, 1, 1, 1, ix2, 0, 0, p->bc);
            out[i] = diff - v * ((ve - vw) * i2h);
          } break;
          case ORC_ADVECT1D: {
            double i2h = 0.5 / hx;
            double ve = u[nbr(x, 1, nx, p->bc)], vw = u[nbr(x, -1, nx, p->bc)];
            out[i] = -(P[0] * ((ve - vw) * i2h));
          } break;
          case ORC_HEAT: {
            int dims = nz > 1 ? 3 : (ny > 1 ? 2 : 1);
            out[i] = P[0] * lap(u, x, y, z, nx, ny, nz, dims, ix2, iy2, iz2, p->bc);
          } break;
          case ORC_DIFFREACT2D: {
            /* Du lap u + (u - u^3 - c - v);  Dv lap v + (u - v)  (Sec. 5.2) */
            const double* uu = u; const double* vv = u + n;
            double a = uu[i], b = vv[i];
            double lu = lap(uu, x, y, 0, nx, ny, 1, 2, ix2, iy2, 0, p->bc);
            double lv = lap(vv, x, y, 0, nx, ny, 1, 2, ix2, iy2, 0, p->bc);
            out[i] = P[0] * lu + (((a - (a * a) * a) - P[2]) - b);
            out[n + i] = P[1] * lv + (a - b);
          } break;
          case ORC_BRUSS2D: case ORC_BRUSS3D: {
            /* D0 lap u + a - (1+b) u + v u^2;  D1 lap v + b u - v u^2  (App. E) */
            int dims = p->pde == ORC_BRUSS3D ? 3 : 2;
            const double* uu = u; const double* vv = u + n;
            double a = uu[i], b = vv[i];
            double lu = lap(uu, x, y, z, nx, ny, nz, dims, ix2, iy2, iz2, p->bc);
            double lv = lap(vv, x, y, z, nx, ny, nz, dims, ix2, iy2, iz2, p->bc);
            double a2 = a * a;
            double opb = 1.0 + P[1];
            out[i] = P[2] * lu + ((P[0] - opb * a) + b * a2);
            out[n + i] = P[3] * lv + (P[1] * a - b * a2);
          } break;
          case ORC_SWE2D: {
            /* dU/dt = -(F_{x+1/2} - F_{x-1/2})/hx - (G_{y+1/2} - G_{y-1/2})/hy
             *         + (0, -g h b_x, -g h b_y)   (Sec. 5.3) */
            double g = P[0];
            int wall = p->bc == ORC_BC_NEUMANN;
            long ie = ((long)y) * nx + nbr(x, 1, nx, p->bc);
            long iw = ((long)y) * nx + nbr(x, -1, nx, p->bc);
            long in_ = ((long)nbr(y, 1, ny, p->bc)) * nx + x;
            long is = ((long)nbr(y, -1, ny, p->bc)) * nx + x;
            double C[3], E[3], W[3], Nn[3], S[3];
            for (int q = 0; q < 3; ++q) {
              C[q] = u[q * n + i]; E[q] = u[q * n + ie]; W[q] = u[q * n + iw];
              Nn[q] = u[q * n + in_]; S[q] = u[q * n + is];
            }
            /* reflecting walls: the cell across the wall is this cell with
             * its normal momentum negated */
            if (wall && x == nx - 1) E[1] = -E[1];
            if (wall && x == 0) W[1] = -W[1];
            if (wall && y == ny - 1) Nn[2] = -Nn[2];
            if (wall && y == 0) S[2] = -S[2];
            double Fe[3], Fw[3], Gn[3], Gs[3];
            swe_flux(g, 0, C, E, Fe);
            swe_flux(g, 0, W, C, Fw);
            swe_flux(g, 1, C, Nn, Gn);
            swe_flux(g, 1, S, C, Gs);
            double ihx = 1.0 / hx, ihy = 1.0 / hy;
            for (int q = 0; q < 3; ++q)
              out[q * n + i] = (Fw[q] - Fe[q]) * ihx + (Gs[q] - Gn[q]) * ihy;
            if (p->bathy) {
              /* -g h grad b by central differences of b (across a wall the
               * bottom's value is the cell's own) */
              const double* b = p->bathy;
              double bx = g * ((b[ie] - b[iw]) * (0.5 / hx));
              double by = g * ((b[in_] - b[is]) * (0.5 / hy));
              out[n + i] = out[n + i] - C[0] * bx;
              out[2 * n + i] = out[2 * n + i] - C[0] * by;
            }
          } break;
          default: out[i] = 0.0;
        }
      }
}

/* ------------------------------------------------------------------ */
/* Time integrators (Sec. 2: F accurate, G cheap).                     */
/* ------------------------------------------------------------------ */

/* Classic RK4: k1 = h(u), k2 = h(u + dt/2 k1), k3 = h(u + dt/2 k2),
 * k4 = h(u + dt k3), u += dt/6 (((k1 + 2 k2) + 2 k3) + k4). */
void orc_rk4(const orc_problem* p, double* u, double dt, int nsteps) {
  long d = orc_dim(p);
  double* w = (double*)malloc(sizeof(double) * d);
  double* k = (double*)malloc(sizeof(double) * d);
  double* acc = (double*)malloc(sizeof(double) * d);
  double h2 = dt / 2.0, h6 = dt / 6.0;
  for (int s = 0; s < nsteps; ++s) {
    orc_rhs(p, u, k);                               /* k1 */
    for (long j = 0; j < d; ++j) { acc[j] = k[j]; w[j] = u[j] + h2 * k[j]; }
    orc_rhs(p, w, k);                               /* k2 */
    for (long j = 0; j < d; ++j) { acc[j] = acc[j] + 2.0 * k[j]; w[j] = u[j] + h2 * k[j]; }
    orc_rhs(p, w, k);                               /* k3 */
    for (long j = 0; j < d; ++j) { acc[j] = acc[j] + 2.0 * k[j]; w[j] = u[j] + dt * k[j]; }
    orc_rhs(p, w, k);                               /* k4 */
    for (long j = 0; j < d; ++j) { acc[j] = acc[j] + k[j]; u[j] = u[j] + h6 * acc[j]; }
  }
  free(w); free(k); free(acc);
}

/* Cooper & Verner's eighth-order explicit Runge-Kutta method with eleven
 * stages (SIAM J. Numer. Anal. 9, 1972), written out from its published
 * tableau; every entry is a rational number or a rational combination of
 * sqrt(21).  Rows s = 1..10 of the strictly lower-triangular A are stored
 * contiguously: a_{s,j} at a[s*(s-1)/2 + j]. */
void orc_rk8_tableau(double* a, double* b, double* c) {
  const double r = sqrt(21.0);
  double A[11][11];
  memset(A, 0, sizeof(A));
  A[1][0] = 1.0 / 2.0;
  A[2][0] = 1.0 / 4.0;
  A[2][1] = 1.0 / 4.0;
  A[3][0] = 1.0 / 7.0;
  A[3][1] = (-7.0 - 3.0 * r) / 98.0;
  A[3][2] = (21.0 + 5.0 * r) / 49.0;
  A[4][0] = (11.0 + r) / 84.0;
  A[4][2] = (18.0 + 4.0 * r) / 63.0;
  A[4][3] = (21.0 - r) / 252.0;
  A[5][0] = (5.0 + r) / 48.0;
  A[5][2] = (9.0 + r) / 36.0;
  A[5][3] = (-231.0 + 14.0 * r) / 360.0;
  A[5][4] = (63.0 - 7.0 * r) / 80.0;
  A[6][0] = (10.0 - r) / 42.0;
  A[6][2] = (-432.0 + 92.0 * r) / 315.0;
  A[6][3] = (633.0 - 145.0 * r) / 90.0;
  A[6][4] = (-504.0 + 115.0 * r) / 70.0;
  A[6][5] = (63.0 - 13.0 * r) / 35.0;
  A[7][0] = 1.0 / 14.0;
  A[7][4] = (14.0 - 3.0 * r) / 126.0;
  A[7][5] = (13.0 - 3.0 * r) / 63.0;
  A[7][6] = 1.0 / 9.0;
  A[8][0] = 1.0 / 32.0;
  A[8][4] = (91.0 - 21.0 * r) / 576.0;
  A[8][5] = 11.0 / 72.0;
  A[8][6] = (-385.0 - 75.0 * r) / 1152.0;
  A[8][7] = (63.0 + 13.0 * r) / 128.0;
  A[9][0] = 1.0 / 14.0;
  A[9][4] = 1.0 / 9.0;
  A[9][5] = (-733.0 - 147.0 * r) / 2205.0;
  A[9][6] = (515.0 + 111.0 * r) / 504.0;
  A[9][7] = (-51.0 - 11.0 * r) / 56.0;
  A[9][8] = (132.0 + 28.0 * r) / 245.0;
  A[10][4] = (-42.0 + 7.0 * r) / 18.0;
  A[10][5] = (-18.0 + 28.0 * r) / 45.0;
  A[10][6] = (-273.0 - 53.0 * r) / 72.0;
  A[10][7] = (301.0 + 53.0 * r) / 72.0;
  A[10][8] = (28.0 - 28.0 * r) / 45.0;
  A[10][9] = (49.0 - 7.0 * r) / 18.0;
  for (int s = 1; s < 11; ++s)
    for (int j = 0; j < s; ++j) a[s * (s - 1) / 2 + j] = A[s][j];
  for (int j = 0; j < 11; ++j) b[j] = 0.0;
  b[0] = 1.0 / 20.0;
  b[7] = 49.0 / 180.0;
  b[8] = 16.0 / 45.0;
  b[9] = 49.0 / 180.0;
  b[10] = 1.0 / 20.0;
  c[0] = 0.0;
  c[1] = c[2] = c[5] = c[8] = 0.5;
  c[3] = c[4] = c[9] = (7.0 + r) / 14.0;
  c[6] = c[7] = (7.0 - r) / 14.0;
  c[10] = 1.0;
}

void orc_rk8(const orc_problem* p, double* u, double dt, int nsteps) {
  long d = orc_dim(p);
  double a[55], b[11], c[11];
  orc_rk8_tableau(a, b, c);
  double* k = (double*)malloc(sizeof(double) * 11 * d);
  double* w = (double*)malloc(sizeof(double) * d);
  for (int n = 0; n < nsteps; ++n) {
    orc_rhs(p, u, k);                                         /* k_0 = h(u) */
    for (int s = 1; s < 11; ++s) {
      const double* as = a + s * (s - 1) / 2;
      for (long j = 0; j < d; ++j) {
        double acc = as[0] * k[j];
        for (int i = 1; i < s; ++i) acc = acc + as[i] * k[(long)i * d + j];
        w[j] = u[j] + dt * acc;
      }
      orc_rhs(p, w, k + (long)s * d);                         /* k_s */
    }
    for (long j = 0; j < d; ++j) {
      double acc = b[0] * k[j];
      for (int i = 1; i < 11; ++i) acc = acc + b[i] * k[(long)i * d + j];
      u[j] = u[j] + dt * acc;
    }
  }
  free(k); free(w);
}

/* Forward Euler (RK1): u += dt h(u). */
void orc_euler(const orc_problem* p, double* u, double dt, int nsteps) {
  long d = orc_dim(p);
  double* k = (double*)malloc(sizeof(double) * d);
  for (int s = 0; s < nsteps; ++s) {
    orc_rhs(p, u, k);
    for (long j = 0; j < d; ++j) u[j] = u[j] + dt * k[j];
  }
  free(k);
}

static double slice_len(const orc_problem* p) { return (p->tN - p->t0) / p->N; }

void orc_fine(const orc_problem* p, const double* in, double* out) {
  long d = orc_dim(p);
  if (out != in) memcpy(out, in, sizeof(double) * d);
  if (p->fscheme == ORC_F_RK8)
    orc_rk8(p, out, slice_len(p) / p->nF, p->nF);
  else
    orc_rk4(p, out, slice_len(p) / p->nF, p->nF);
}

void orc_coarse(const orc_problem* p, const double* in, double* out) {
  long d = orc_dim(p);
  if (out != in) memcpy(out, in, sizeof(double) * d);
  if (p->gscheme == 1)
    orc_rk4(p, out, slice_len(p) / p->nG, p->nG);
  else
    orc_euler(p, out, slice_len(p) / p->nG, p->nG);
}

void orc_serial_fine(const orc_problem* p, const double* u0, double* U) {
  long d = orc_dim(p);
  memcpy(U, u0, sizeof(double) * d);
  for (int i = 1; i <= p->N; ++i) orc_fine(p, U + (long)(i - 1) * d, U + (long)i * d);
}

/* ------------------------------------------------------------------ */
/* Seeded weights (Alg. 3: A_wj, zeta_w ~ Uniform(-1,1), kept fixed).  */
/* ------------------------------------------------------------------ */

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

uint64_t orc_splitmix64_next(uint64_t* state) {
  *state += 0x9e3779b97f4a7c15ULL;
  return mix64(*state);
}

double orc_uniform(uint64_t seed, uint32_t stream, uint64_t idx) {
  uint64_t n = ((uint64_t)stream << 40) + idx + 1;
  uint64_t z = mix64(seed + n * 0x9e3779b97f4a7c15ULL);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

void orc_weights(const orc_problem* p, double* A, double* zeta) {
  long d = orc_dim(p);
  for (long w = 0; w < p->M; ++w) {
    for (long j = 0; j < d; ++j)
      A[w * d + j] = 2.0 * orc_uniform(p->seed, 0, (uint64_t)(w * d + j)) - 1.0;
    zeta[w] = 2.0 * orc_uniform(p->seed, 1, (uint64_t)w) - 1.0;
  }
}

/* ------------------------------------------------------------------ */
/* Rescaling to [-1,1] (Alg. 1 initialisation, Alg. 3), per species.   */
/* ------------------------------------------------------------------ */

void orc_scaling(const orc_problem* p, const double* U, int nstates,
                 double* c, double* r) {
  int nc = orc_ncomp(p);
  long n = (long)p->nx * p->ny * p->nz, d = orc_dim(p);
  for (int q = 0; q < nc; ++q) {
    if (p->scale_mode == ORC_SCALE_NONE) { c[q] = 0.0; r[q] = 1.0; continue; }
    double mn = U[q * n], mx = U[q * n];
    for (int s = 0; s < nstates; ++s)
      for (long j = 0; j < n; ++j) {
        double v = U[(long)s * d + q * n + j];
        if (v < mn) mn = v;
        if (v > mx) mx = v;
      }
    c[q] = 0.5 * (mx + mn);
    r[q] = 0.5 * (mx - mn);
    if (r[q] == 0.0) r[q] = 1.0;
  }
}

void orc_scale(const orc_problem* p, const double* c, const double* r,
               const double* u, double* s) {
  int nc = orc_ncomp(p);
  long n = (long)p->nx * p->ny * p->nz;
  for (int q = 0; q < nc; ++q)
    for (long j = 0; j < n; ++j) s[q * n + j] = (u[q * n + j] - c[q]) / r[q];
}

/* ------------------------------------------------------------------ */
/* RandNet pieces (Eq. HA, Eq. ridgeless, App. B).                     */
/* ------------------------------------------------------------------ */

void orc_features(const double* A, const double* zeta, int M, long d,
                  const double* s, double* phi) {
  for (int w = 0; w < M; ++w) {
    double acc = 0.0;
    for (long j = 0; j < d; ++j) acc = acc + A[(long)w * d + j] * s[j];
    double v = acc + zeta[w];
    phi[w] = v > 0.0 ? v : 0.0;
  }
}

int orc_nn(const double* S, long P, long d, const double* q, int m,
           long* idx, double* dist) {
  int me = (long)m < P ? m : (int)P;
  double* del = (double*)malloc(sizeof(double) * (P > 0 ? P : 1));
  char* used = (char*)calloc(P > 0 ? P : 1, 1);
  for (long p = 0; p < P; ++p) {
    double acc = 0.0;
    for (long j = 0; j < d; ++j) {
      double t = q[j] - S[p * d + j];
      acc = acc + t * t;
    }
    del[p] = acc;
  }
  for (int l = 0; l < me; ++l) {
    long best = -1;
    for (long p = 0; p < P; ++p) {
      if (used[p]) continue;
      if (best < 0 || del[p] < del[best]) best = p;   /* ties keep lower p */
    }
    used[best] = 1;
    idx[l] = best;
    if (dist) dist[l] = del[best];
  }
  free(del); free(used);
  return me;
}

int orc_cholesky_solve(const double* K, int n, const double* b, double* x) {
  double* L = (double*)calloc((size_t)n * n, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * n);
  int rc = 0;
  for (int j = 0; j < n && rc == 0; ++j) {
    double s = K[j * n + j];
    for (int k = 0; k < j; ++k) s = s - L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) { rc = -1; break; }
    double ljj = sqrt(s);
    L[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = K[i * n + j];
      for (int k = 0; k < j; ++k) t = t - L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / ljj;
    }
  }
  if (rc == 0) {
    for (int i = 0; i < n; ++i) {
      double t = b[i];
      for (int k = 0; k < i; ++k) t = t - L[i * n + k] * y[k];
      y[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t = t - L[k * n + i] * x[k];
      x[i] = t / L[i * n + i];
    }
  }
  free(L); free(y);
  return rc;
}

int orc_ridge_dual(const double* X, int m, int M, const double* phiq,
                   double lambda, double* alpha) {
  double* K = (double*)malloc(sizeof(double) * m * m);
  double* b = (double*)malloc(sizeof(double) * m);
  for (int i = 0; i < m; ++i) {
    double acc = 0.0;
    for (int w = 0; w < M; ++w) acc = acc + X[i * M + w] * phiq[w];
    b[i] = acc;
  }
  int esc = -1;
  double lam = lambda;
  for (int tries = 0; tries <= 4; ++tries) {
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= i; ++j) {
        double acc = 0.0;
        for (int w = 0; w < M; ++w) acc = acc + X[i * M + w] * X[j * M + w];
        if (i == j) acc = acc + lam;
        K[i * m + j] = acc;
        K[j * m + i] = acc;
      }
    if (orc_cholesky_solve(K, m, b, alpha) == 0) { esc = tries; break; }
    lam = lam * 10.0;
  }
  free(K); free(b);
  return esc;
}

int orc_ridge_primal(const double* X, const double* Y, int m, int M, long d,
                     const double* phiq, double lambda, double* pred) {
  /* Solve (X^T X + lambda I_M) z = phiq, then pred = Y^T X z
   * (= W^T phiq with W = (X^T X + lambda I)^{-1} X^T Y). */
  double* G = (double*)malloc(sizeof(double) * M * M);
  double* z = (double*)malloc(sizeof(double) * M);
  double* t = (double*)malloc(sizeof(double) * m);
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      double acc = 0.0;
      for (int l = 0; l < m; ++l) acc = acc + X[l * M + a] * X[l * M + b];
      if (a == b) acc = acc + lambda;
      G[a * M + b] = acc;
    }
  int rc = orc_cholesky_solve(G, M, phiq, z);
  if (rc == 0) {
    for (int l = 0; l < m; ++l) {
      double acc = 0.0;
      for (int a = 0; a < M; ++a) acc = acc + X[l * M + a] * z[a];
      t[l] = acc;
    }
    for (long j = 0; j < d; ++j) {
      double acc = 0.0;
      for (int l = 0; l < m; ++l) acc = acc + t[l] * Y[(long)l * d + j];
      pred[j] = acc;
    }
  }
  free(G); free(z); free(t);
  return rc;
}

/* Gather the m nearest rows, solve the dual ridge system, combine the
 * targets: out = sum_l alpha_l Y[p_l] (l ascending). */
static int predict_scaled(int M, int m, double lambda, long d,
                          const double* S, const double* Y, const double* Phi,
                          long P, const double* s, const double* phiq,
                          double* out, long* nn_out) {
  for (long j = 0; j < d; ++j) out[j] = 0.0;
  if (P == 0) return 0;
  long idx[64];
  int me = orc_nn(S, P, d, s, m, idx, NULL);
  double* X = (double*)malloc(sizeof(double) * me * M);
  double alpha[64];
  for (int l = 0; l < me; ++l)
    memcpy(X + (long)l * M, Phi + idx[l] * M, sizeof(double) * M);
  int esc = orc_ridge_dual(X, me, M, phiq, lambda, alpha);
  free(X);
  if (esc < 0) return -1;
  for (long j = 0; j < d; ++j) {
    double acc = 0.0;
    for (int l = 0; l < me; ++l) acc = acc + alpha[l] * Y[idx[l] * d + j];
    out[j] = acc;
  }
  if (nn_out) for (int l = 0; l < me; ++l) nn_out[l] = idx[l];
  return esc;
}

int orc_predict(const orc_problem* p, const double* S, const double* Y,
                const double* Phi, long P, const double* A,
                const double* zeta, const double* c, const double* r,
                const double* u, double* out, long* nn_out) {
  long d = orc_dim(p);
  double* s = (double*)malloc(sizeof(double) * d);
  double* phiq = (double*)malloc(sizeof(double) * p->M);
  orc_scale(p, c, r, u, s);
  orc_features(A, zeta, p->M, d, s, phiq);
  int rc = predict_scaled(p->M, p->m, p->lambda, d, S, Y, Phi, P, s, phiq,
                          out, nn_out);
  free(s); free(phiq);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Alg. 1 (generic Parareal) with Eq. 3 and Eq. randnet / Eq. 4.        */
/* ------------------------------------------------------------------ */

static int all_finite(const double* v, long n) {
  for (long j = 0; j < n; ++j) if (!isfinite(v[j])) return 0;
  return 1;
}

int orc_solve(const orc_problem* p, const double* u0, double* U,
              orc_stats* st, orc_trace* tr) {
  const int N = p->N, M = p->M;
  const long d = orc_dim(p);
  if (N < 1 || p->nF < 1 || p->nG < 1 || p->m < 1 || p->m > 64 || M < 1 ||
      p->max_iters < 1 || p->bc < 0 || p->bc > 1 ||
      (p->bathy && p->pde != ORC_SWE2D))
    return ORC_EINVAL;
  const int K_max = p->max_iters < N ? p->max_iters : N;
  /* At most N - k + 1 pairs are appended at iteration k (L >= k - 1). */
  long cap = 0;
  for (int k = 1; k <= K_max; ++k) cap += N - k + 1;

  double* Uold = (double*)malloc(sizeof(double) * (N + 1) * d);
  double* Fv = (double*)malloc(sizeof(double) * N * d);
  double* Gc = (double*)malloc(sizeof(double) * N * d);     /* G(U_j) */
  double* Yv = (double*)malloc(sizeof(double) * N * d);     /* (F-G)(U_j) */
  double* S = (double*)malloc(sizeof(double) * cap * d);
  double* Y = (double*)malloc(sizeof(double) * cap * d);
  double* Phi = (double*)malloc(sizeof(double) * cap * M);
  double* A = (double*)malloc(sizeof(double) * M * d);
  double* zeta = (double*)malloc(sizeof(double) * M);
  double* sq = (double*)malloc(sizeof(double) * d);
  double* phiq = (double*)malloc(sizeof(double) * M);
  double* corr = (double*)malloc(sizeof(double) * d);
  double c[3], r[3];
  int status = ORC_OK;
  if (!Uold || !Fv || !Gc || !Yv || !S || !Y || !Phi || !A || !zeta || !sq ||
      !phiq || !corr) {
    status = ORC_ENOMEM;
    goto done;
  }
  memset(st, 0, sizeof(*st));

  /* k = 0: U_i^0 = G(U_{i-1}^0), sequentially (Alg. 1 initialisation). */
  memcpy(U, u0, sizeof(double) * d);
  for (int i = 1; i <= N; ++i) {
    orc_coarse(p, U + (long)(i - 1) * d, U + (long)i * d);
    memcpy(Gc + (long)(i - 1) * d, U + (long)i * d, sizeof(double) * d);
  }
  if (!all_finite(U, (long)(N + 1) * d)) { status = ORC_ENONFINITE; goto done; }
  orc_scaling(p, U, N + 1, c, r);
  if (p->corr == ORC_CORR_RANDNET) orc_weights(p, A, zeta);

  int L = 0;
  long P = 0;
  for (int k = 1; k <= K_max; ++k) {
    /* F on every start not yet converged, all slices "in parallel". */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
#endif
    for (int j = L; j < N; ++j) orc_fine(p, U + (long)j * d, Fv + (long)j * d);
    st->fine_cell_updates += (long long)(N - L) * p->nF * d;

    /* Dataset D_k (Eq. 6): pairs (U_j^{k-1}, (F - G)(U_j^{k-1})). */
    for (int j = L; j < N; ++j) {
      for (long t = 0; t < d; ++t)
        Yv[(long)j * d + t] = Fv[(long)j * d + t] - Gc[(long)j * d + t];
      if (p->corr == ORC_CORR_RANDNET) {
        orc_scale(p, c, r, U + (long)j * d, S + P * d);
        memcpy(Y + P * d, Yv + (long)j * d, sizeof(double) * d);
        orc_features(A, zeta, M, d, S + P * d, Phi + P * M);
        ++P;
      }
    }

    memcpy(Uold, U, sizeof(double) * (N + 1) * d);
    /* The leftmost start is converged, so its fine value is exact. */
    memcpy(U + (long)(L + 1) * d, Fv + (long)L * d, sizeof(double) * d);

    /* Sequential predictor-corrector sweep, Eq. 3. */
    for (int i = L + 2; i <= N; ++i) {
      const double* prev = U + (long)(i - 1) * d;
      double* g = Gc + (long)(i - 1) * d;
      orc_coarse(p, prev, g);
      if (p->corr == ORC_CORR_RANDNET) {
        long nn[64];
        orc_scale(p, c, r, prev, sq);
        orc_features(A, zeta, M, d, sq, phiq);
        int esc = predict_scaled(M, p->m, p->lambda, d, S, Y, Phi, P, sq, phiq,
                                 corr, nn);
        if (esc < 0) { status = ORC_ENONFINITE; goto done; }
        st->lambda_escalations += esc;
        if (tr && tr->nn_idx) {
          int me = (long)p->m < P ? p->m : (int)P;
          for (int l = 0; l < p->m; ++l)
            tr->nn_idx[((long)(k - 1) * (N + 1) + i) * p->m + l] =
                l < me ? nn[l] : -1;
        }
      } else {
        memcpy(corr, Yv + (long)(i - 1) * d, sizeof(double) * d);
      }
      double* ui = U + (long)i * d;
      for (long t = 0; t < d; ++t) ui[t] = g[t] + corr[t];
    }
    if (!all_finite(U, (long)(N + 1) * d)) { status = ORC_ENONFINITE; goto done; }

    /* Convergence (Eq. 5): U_{L+1} is exact; then advance while
     * ||U_i^k - U_i^{k-1}||_inf < tol, in order. */
    int Lnew = L + 1;
    for (int i = L + 2; i <= N; ++i) {
      double e = 0.0;
      for (long t = 0; t < d; ++t) {
        double a = fabs(U[(long)i * d + t] - Uold[(long)i * d + t]);
        if (a > e) e = a;
      }
      if (e < p->tol) Lnew = i; else break;
    }
    L = Lnew;
    st->K = k;
    if (tr && tr->L_hist) tr->L_hist[k - 1] = L;
    if (L == N) break;
  }
  st->L = L;
  st->converged = (L == N);
  st->pairs = P;
  if (!st->converged) status = ORC_ENOTCONV;

done:
  free(Uold); free(Fv); free(Gc); free(Yv); free(S); free(Y); free(Phi);
  free(A); free(zeta); free(sq); free(phiq); free(corr);
  return status;
}
