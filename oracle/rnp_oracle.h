/*
 * rnp_oracle.h -- plain, slow, single-precision-free (FP64) CPU oracle for
 * RandNet-Parareal (Gattiglio, Grigoryeva, Tamborrino, NeurIPS 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this code: only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library; both sides are written from the
 * paper independently.
 *
 * What it computes (paper sections in brackets):
 *   - the semi-discretised right-hand sides h(u) of Eq. 1 for the five PDE
 *     families of Sec. 5 and App. E (Burgers, diffusion-reaction, 2D/3D
 *     Brusselator, shallow water) plus two linear test operators;
 *   - the fine solver F (classic RK4, or the eighth-order RK8 the paper
 *     uses for Burgers and diffusion-reaction, Sec. 5.1-5.2) and the coarse
 *     solver G (forward Euler) over one time slice [Sec. 2, Tables 4-7];
 *   - the RandNet of Eq. HA with seeded U(-1,1) weights (Alg. 3), the
 *     m-nearest-neighbour restriction of App. B (eq. fhat_mnn) and the
 *     ridge(less) readout of Eq. ridgeless in its dual (m x m) form;
 *   - the generic Parareal iteration of Alg. 1 with the update rule of
 *     Eq. 3, the RandNet correction of Eq. randnet or the classic
 *     correction of Eq. 4, and the stopping rule of Eq. 5.
 *
 * Every floating-point expression is evaluated in the order written in
 * the source, compiled with -ffp-contract=off (no fused multiply-add).
 *
 * Pins (tests/test_oracle_*.py): every function is checked against closed
 * forms, invariants, brute force, library routines or published vectors.
 * orc_solve's iterates for tol > 0 have no value printed in the paper:
 * beyond K <= N, eps = 0 (K = N, bitwise the serial fine solution), G = F
 * (K = 1) and the converged error near tol, they are "parity unpinned".
 */
#ifndef RNP_ORACLE_H
#define RNP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_BURGERS1D = 0,  /* v_t = nu v_xx - v v_x                      (Sec. 5.1) */
  ORC_DIFFREACT2D = 1,/* FitzHugh-Nagumo diffusion-reaction           (Sec. 5.2) */
  ORC_BRUSS2D = 2,    /* Brusselator, 2 space dims                     (App. E)   */
  ORC_BRUSS3D = 3,    /* Brusselator, 3 space dims                     (App. E)   */
  ORC_SWE2D = 4,      /* shallow water, conserved (h, hu, hv)          (Sec. 5.3) */
  ORC_HEAT = 5,       /* u_t = D lap u, 1/2/3 dims (test operator)                 */
  ORC_ADVECT1D = 6    /* u_t = -c u_x (test operator)                              */
};

enum { ORC_CORR_RANDNET = 0, ORC_CORR_PARAREAL = 1 };
/* Boundary: periodic, or no-flux (homogeneous Neumann) on a cell-centred
 * finite-volume grid -- the flux through a wall face is zero, i.e. the
 * neighbour across the wall is the cell itself (Sec. 5.2: no-flow
 * Neumann boundary, finite-volume discretisation).  Shallow water
 * (Sec. 5.3: a box whose walls the water rebounds from): the cell across a
 * wall mirrors the cell with its momentum normal to the wall negated (a
 * reflecting wall: zero normal gradient of h and of the tangential
 * momentum, no mass through the wall). */
enum { ORC_BC_PERIODIC = 0, ORC_BC_NEUMANN = 1 };
enum { ORC_SCALE_MINMAX = 0, ORC_SCALE_NONE = 1 };
/* Fine integrator: classic RK4, or RK8 = the explicit eleven-stage
 * eighth-order method of Cooper & Verner (SIAM J. Numer. Anal. 9, 1972). */
enum { ORC_F_RK4 = 0, ORC_F_RK8 = 1 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENONFINITE = 4,
       ORC_ENOTCONV = 5 };

typedef struct {
  int pde;
  int nx, ny, nz;           /* grid points per axis (ny = nz = 1 in 1D)   */
  double lx, ly, lz;        /* domain lengths (cell size lx / nx, ...)     */
  double param[8];          /* PDE coefficients, see orc_rhs               */
  double t0, tN;            /* time interval of Eq. 1                      */
  int N;                    /* number of time slices                       */
  int nF, nG;               /* steps of F and of G per slice               */
  int M, m;                 /* hidden neurons, nearest neighbours          */
  double lambda;            /* ridge penalty                               */
  uint64_t seed;            /* weight seed                                 */
  double tol;               /* epsilon of Eq. 5                            */
  int max_iters;            /* <= N                                        */
  int corr;                 /* ORC_CORR_*                                  */
  int scale_mode;           /* ORC_SCALE_*                                 */
  int gscheme;              /* G integrator: 0 forward Euler (RK1), 1 RK4  */
  int bc;                   /* ORC_BC_* (shallow water: periodic only)     */
  int fscheme;              /* ORC_F_*: F integrator                       */
  const double* bathy;      /* shallow water: bottom b at the nx*ny cell
                               centres (row-major, x fastest), or NULL for a
                               flat bottom; adds -g h grad b (Sec. 5.3)     */
} orc_problem;

typedef struct {
  int K;                    /* iterations performed                        */
  int L;                    /* last converged state index at exit          */
  int converged;            /* L == N                                      */
  long pairs;               /* dataset size at exit                        */
  long long fine_cell_updates; /* sum over F runs of nF * d               */
  int lambda_escalations;   /* ridge retries with a larger lambda          */
} orc_stats;

/* Optional per-iteration record (any pointer may be NULL).
 *   L_hist[k-1]                 : L after iteration k
 *   nn_idx[((k-1)*(N+1)+i)*m+l] : l-th neighbour used for state i at
 *                                 iteration k (-1 where no prediction)   */
typedef struct {
  int* L_hist;
  long* nn_idx;
} orc_trace;

int  orc_ncomp(const orc_problem* p);
long orc_dim(const orc_problem* p);
void orc_set_threads(int n);        /* slice-parallel F (results unchanged) */

/* h(u) of Eq. 1 for one state vector of length orc_dim(p). */
void orc_rhs(const orc_problem* p, const double* u, double* out);
/* nsteps classic RK4 / forward-Euler steps of size dt, in place. */
void orc_rk4(const orc_problem* p, double* u, double dt, int nsteps);
void orc_euler(const orc_problem* p, double* u, double dt, int nsteps);
/* The Cooper-Verner RK8 tableau: a[s*(s-1)/2 + j] = a_{s,j} (0 <= j < s,
 * stages s = 1..10, 0-based), b[0..10], c[0..10]. */
void orc_rk8_tableau(double* a, double* b, double* c);
/* nsteps RK8 steps of size dt, in place.  Stage s is evaluated at
 * u + dt (a_{s,0} k_0 + a_{s,1} k_1 + ... + a_{s,s-1} k_{s-1}) (sum left to
 * right) and the step adds dt (b_0 k_0 + ... + b_10 k_10). */
void orc_rk8(const orc_problem* p, double* u, double dt, int nsteps);
/* F and G over one slice of length (tN - t0) / N. */
void orc_fine(const orc_problem* p, const double* in, double* out);
void orc_coarse(const orc_problem* p, const double* in, double* out);
/* Serial fine solution: U[0] = u0, U[i] = F(U[i-1]), i = 1..N. */
void orc_serial_fine(const orc_problem* p, const double* u0, double* U);

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): next output of a
 * sequential generator whose state is *state. */
uint64_t orc_splitmix64_next(uint64_t* state);
/* Counter form: output number (stream * 2^40 + idx + 1) of the generator
 * seeded with seed, mapped to [0,1) with 53 bits. */
double orc_uniform(uint64_t seed, uint32_t stream, uint64_t idx);
/* A[w*d + j], zeta[w] ~ U(-1,1) (Alg. 3): streams 0 and 1. */
void orc_weights(const orc_problem* p, double* A, double* zeta);

/* Per-species affine map to [-1,1] from nstates state vectors. */
void orc_scaling(const orc_problem* p, const double* U, int nstates,
                 double* c, double* r);
void orc_scale(const orc_problem* p, const double* c, const double* r,
               const double* u, double* s);
/* phi = ReLU(A s + zeta), Eq. HA. */
void orc_features(const double* A, const double* zeta, int M, long d,
                  const double* s, double* phi);
/* m smallest squared Euclidean distances, ties broken by index (App. B). */
int  orc_nn(const double* S, long P, long d, const double* q, int m,
            long* idx, double* dist);
/* Cholesky factorisation and solve of an n x n SPD system (row-major).
 * Returns 0, or -1 when a pivot is not positive. */
int  orc_cholesky_solve(const double* K, int n, const double* b, double* x);
/* Dual ridge coefficients alpha = (X X^T + lambda I_m)^{-1} X phiq.
 * Returns the number of lambda escalations (x10 each, at most 4) or -1. */
int  orc_ridge_dual(const double* X, int m, int M, const double* phiq,
                    double lambda, double* alpha);
/* Primal form W = (X^T X + lambda I_M)^{-1} X^T Y, pred = W^T phiq
 * (Eq. ridgeless).  Used only to pin the dual form.  0 or -1. */
int  orc_ridge_primal(const double* X, const double* Y, int m, int M, long d,
                      const double* phiq, double lambda, double* pred);
/* RandNet correction for one query u (Eq. randnet with the m-nn dataset):
 * out = sum_l alpha_l Y[p_l].  S, Y: P x d, Phi: P x M.  Returns the
 * number of lambda escalations or -1. */
int  orc_predict(const orc_problem* p, const double* S, const double* Y,
                 const double* Phi, long P, const double* A,
                 const double* zeta, const double* c, const double* r,
                 const double* u, double* out, long* nn_out);

/* Alg. 1.  U: (N+1) x d output (U_0 .. U_N).  Returns ORC_OK,
 * ORC_ENOTCONV (U filled with the last iterate) or another status. */
int  orc_solve(const orc_problem* p, const double* u0, double* U,
               orc_stats* st, orc_trace* tr);

#ifdef __cplusplus
}
#endif
#endif
