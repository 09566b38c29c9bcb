/*
 * rnp.h -- C ABI of librnp, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of RandNet-Parareal (Gattiglio, Grigoryeva,
 * Tamborrino, "RandNet-Parareal: a time-parallel PDE solver using Random
 * Neural Networks", NeurIPS 2024).
 *
 * The library solves the initial value problem of Eq. 1,
 *     du/dt = h(u),  t in [t0, tN],  u(t0) = u0,  u in R^d,
 * split into N time slices (Sec. 2), with a cheap coarse propagator G
 * (forward Euler or RK4), an accurate fine propagator F (classic RK4, or
 * the eighth-order RK8 the paper uses in Sec. 5.1-5.2) and the RandNet
 * correction of Eq. randnet: a fixed random hidden layer
 * (Eq. HA, weights and biases U(-1,1), ReLU) whose linear readout is a
 * ridge fit (Eq. ridgeless) on the m nearest stored pairs (App. B), inside
 * the predictor-corrector sweep of Eq. 3 and the loop of Alg. 1.
 *
 * Conventions shared by every call
 *   - Array arguments are caller-owned DEVICE pointers to contiguous FP64
 *     data on the device that was current at rnp_create, except where a
 *     call or field says "host".  The library never frees them and never
 *     keeps them past the call.
 *   - d = ncomp * nx * ny * nz unknowns per state, component-major, then z,
 *     then y, then x (x fastest).  ncomp: Burgers/heat/advection 1,
 *     diffusion-reaction and Brusselator 2 (u then v), shallow water 3
 *     (h, hu, hv).
 *   - B = problem.batch independent initial conditions share the grid,
 *     N, F, G and the random weights; each has its own dataset, scaling and
 *     convergence state.  Batched arrays put the member index outermost.
 *   - Calls enqueue work on the stream given to rnp_create and return
 *     without waiting, except rnp_solve (which returns statistics) and
 *     rnp_coarse_sweep / rnp_randnet_predict (which read the dataset size on
 *     the host).  Inputs must be ready on that stream.
 *   - A context is not thread-safe; use one per concurrent solve.
 *   - No call throws.  Every call returns an rnp_status; on failure
 *     rnp_last_error(ctx) holds a message until the next call on ctx.
 *   - A context owns its device memory (slice states, the dataset arena of
 *     scaled inputs, targets and features, the random weights, workspace),
 *     allocated at rnp_create and released by rnp_destroy.
 */
#ifndef RNP_H
#define RNP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rnp_ctx rnp_ctx;

typedef enum {
  RNP_OK = 0,
  RNP_EINVAL = 1,      /* bad argument or unsupported configuration        */
  RNP_ENOMEM = 2,      /* device allocation failed or dataset arena full   */
  RNP_ECUDA = 3,       /* a CUDA runtime call failed                        */
  RNP_ENONFINITE = 4,  /* a state became NaN/Inf, or the ridge solve failed */
  RNP_ENOTCONV = 5,    /* max_iters reached before Eq. 5 held for all i     */
  RNP_ETIMEOUT = 6,    /* a bounded device wait gave up                     */
  RNP_EBUSY = 7        /* the server has no free slot                       */
} rnp_status;

/* h(u) of Eq. 1: finite-difference semi-discretisations (periodic, or with
 * no-flux walls, see rnp_bc) of the paper's test systems (Sec. 5.1 Burgers,
 * Sec. 5.2 diffusion-reaction, App. E Brusselator, Sec. 5.3 shallow water)
 * and two linear operators. */
typedef enum {
  RNP_BURGERS1D = 0,   /* param: nu                                        */
  RNP_DIFFREACT2D = 1, /* param: Du, Dv, c   (FitzHugh-Nagumo kinetics)   */
  RNP_BRUSS2D = 2,     /* param: a, b, D0, D1                              */
  RNP_BRUSS3D = 3,     /* param: a, b, D0, D1                              */
  RNP_SWE2D = 4,       /* param: g  (Rusanov flux; bottom: bathymetry)     */
  RNP_HEAT = 5,        /* param: D  (1, 2 or 3 dimensions)                 */
  RNP_ADVECT1D = 6     /* param: c                                         */
} rnp_pde;

typedef enum { RNP_FP64 = 0, RNP_MIXED = 1, RNP_MIXED_BF16 = 2 } rnp_precision;
/* FP64: every step in double precision; F and G are bit-identical to a
 *       plain serial FP64 evaluation of the same formulas.
 * MIXED: F and G stencils in FP32 arithmetic on a compensated (two-word)
 *       FP32 state; random features and neighbour distances in FP32; ridge
 *       solve, correction and norm in FP64.
 * MIXED_BF16: as MIXED, but the random features use BF16 operands (weights
 *       and scaled inputs rounded to BF16) with FP32 accumulation: batched
 *       rows on the tensor cores (tcgen05), single queries on CUDA cores.  */

typedef enum { RNP_EXEC_FUSED = 0, RNP_EXEC_PLAIN = 1 } rnp_exec;
/* FUSED: one launch advances every active slice through all of its steps,
 *        each slice resident in the shared memory of a thread-block cluster.
 * PLAIN: one launch per Runge-Kutta stage over global memory (baseline). */

typedef enum { RNP_CORR_RANDNET = 0, RNP_CORR_PARAREAL = 1 } rnp_corr;
/* RANDNET: f_hat of Eq. randnet.  PARAREAL: f_hat of Eq. 4. */

typedef enum { RNP_SCALE_MINMAX = 0, RNP_SCALE_NONE = 1 } rnp_scale;
/* MINMAX: the RandNet input is rescaled per species to [-1,1] from the
 * k = 0 coarse trajectory (Alg. 1 initialisation, Alg. 3).  NONE: identity. */

typedef enum { RNP_G_EULER = 0, RNP_G_RK4 = 1 } rnp_gscheme;

typedef enum { RNP_F_RK4 = 0, RNP_F_RK8 = 1 } rnp_fscheme;
/* F's integrator.  RK4: classic fourth order.  RK8: the eleven-stage
 * explicit eighth-order method of Cooper & Verner (SIAM J. Numer. Anal. 9,
 * 1972), the paper's RK8 fine solver (Sec. 5.1, 5.2) with a fixed step;
 * requires precision RNP_FP64 (RNP_EINVAL otherwise).  In the fused
 * execution a thread keeps the ten stage derivatives of at most two cells
 * in registers, so a slice must fit 2 x 512 cells per CTA of a 16-CTA
 * cluster (RNP_EINVAL otherwise; the plain execution has no such limit). */

typedef enum { RNP_BC_PERIODIC = 0, RNP_BC_NEUMANN = 1 } rnp_bc;
/* PERIODIC: every axis wraps.  NEUMANN: no-flux walls on a cell-centred
 * finite-volume grid (Sec. 5.2's no-flow Neumann boundary): the flux through
 * a wall face is zero, i.e. the neighbour across the wall is the cell
 * itself.  Shallow water (Sec. 5.3: a box whose walls the water rebounds
 * from): reflecting walls, the cell across a wall mirrors the cell with its
 * momentum normal to the wall negated (zero normal gradient of h and of the
 * tangential momentum, no mass through a wall). */

#define RNP_MAX_BATCH 64
#define RNP_MAX_M 32   /* largest number of nearest neighbours m */

typedef struct {
  int pde;                /* rnp_pde                                        */
  int nx, ny, nz;         /* grid points per axis (1 for unused axes)       */
  double lx, ly, lz;      /* periodic domain lengths                        */
  double param[8];        /* PDE coefficients (see rnp_pde)                 */
  double t0, tN;          /* time interval of Eq. 1                         */
  int N;                  /* time slices (Sec. 2)                           */
  int nF, nG;             /* steps of F (RK4 or RK8) and G per slice        */
  int M, m;               /* hidden neurons (Eq. HA), neighbours (App. B)   */
  double lambda;          /* ridge penalty of Eq. ridgeless (> 0)           */
  uint64_t seed;          /* seed of A and zeta (Alg. 3)                    */
  double tol;             /* epsilon of Eq. 5                               */
  int max_iters;          /* iteration cap, 1 <= max_iters <= N             */
  int corr;               /* rnp_corr                                       */
  int scale_mode;         /* rnp_scale                                      */
  int gscheme;            /* rnp_gscheme                                    */
  int precision;          /* rnp_precision                                  */
  int exec;               /* rnp_exec                                       */
  int batch;              /* independent initial conditions, 1..64          */
  int cluster;            /* fused stencil: CTAs per slice (0 = auto)       */
  int threads;            /* fused stencil: threads per CTA, 0..800 (0 = auto) */
  long long max_pairs;    /* dataset rows per member (0 = enough for
                             max_iters iterations)                          */
  int autotune;           /* 1: rnp_create times every launchable stencil
                             tiling on the context's buffers and keeps the
                             fastest (ignored when cluster/threads are set) */
  int bc;                 /* rnp_bc                                        */
  int fscheme;            /* rnp_fscheme                                   */
  const double* bathymetry; /* shallow water only: HOST array of the bottom
                             b at the nx*ny cell centres (x fastest), read
                             during rnp_create only (the caller keeps
                             ownership); adds -g h grad b to the momentum
                             equations (Sec. 5.3) by central differences
                             of b (across a wall b's neighbour is the cell
                             itself).  NULL: flat bottom.  Non-NULL for
                             another PDE: RNP_EINVAL.                       */
} rnp_problem;

typedef struct {
  int K;                  /* iterations performed (max over the batch)      */
  int L;                  /* min over the batch of the last converged index */
  int converged;          /* every member reached L = N                     */
  long long pairs;        /* dataset rows over the batch                    */
  long long fine_cell_updates; /* sum over F runs of nF * d                */
  int lambda_escalations; /* ridge retries with lambda x 10                 */
  double t_fine_ms;       /* device time in F (events on the ctx stream)    */
  double t_sweep_ms;      /* device time in the sequential sweeps           */
  double t_fit_ms;        /* device time appending pairs and features       */
  double t_total_ms;      /* wall time of the call                          */
  long long kernel_launches; /* kernels this call launched                   */
  int K_each[RNP_MAX_BATCH];  /* per-member iterations                      */
} rnp_stats;

/* Create a context for one problem.  cuda_stream is a cudaStream_t (NULL
 * for the legacy default stream).  Allocates every device buffer the solve
 * needs (dataset arena sized for max_iters iterations: at most
 * N - k + 1 pairs are added at iteration k, Alg. 1 with Eq. 6).
 * Errors: RNP_EINVAL (bad sizes or parameters), RNP_ENOMEM, RNP_ECUDA.   */
rnp_status rnp_create(const rnp_problem* prob, void* cuda_stream, rnp_ctx** out);

/* Release every resource of ctx (NULL is allowed).  Waits for the stream. */
rnp_status rnp_destroy(rnp_ctx* ctx);

/* Fine propagator F on n slice starts per member (Sec. 2: F run "in
 * parallel" across slices; Alg. 1, parallel step).
 *   U_in  : device [B][n][d]  slice start states
 *   U_out : device [B][n][d]  F(U_in); may not alias U_in
 * 1 <= n <= N.  Enqueues one launch.                                      */
rnp_status rnp_fine_batch(rnp_ctx* ctx, const double* U_in, int n, double* U_out);

/* Sequential predictor-corrector sweep, Eq. 3 with the context's f_hat:
 *   U[b][first] = U_first[b];
 *   U[b][i] = G(U[b][i-1]) + f_hat(U[b][i-1]),  i = first+1 .. N.
 *   U_first : device [B][d];  U : device [B][N+1][d].
 * With an empty dataset f_hat = 0 (the k = 0 coarse sweep of Alg. 1); such
 * a sweep from first = 0 also sets the scaling of Alg. 1 from U[b][0..N]
 * when scale_mode is MINMAX.  0 <= first <= N.                            */
rnp_status rnp_coarse_sweep(rnp_ctx* ctx, int first, const double* U_first,
                            double* U);

/* Append P training pairs per member to the dataset D_k of Eq. 6: inputs
 * Uin (unscaled) and targets Y = (F - G)(Uin).  The context stores the
 * scaled input, the target and its random features phi = ReLU(A s + zeta)
 * (Eq. HA); the readout itself is refit per query, on the m nearest pairs,
 * inside rnp_randnet_predict (Alg. 3).
 *   Uin, Y : device [B][P][d].  Errors: RNP_ENOMEM when the arena is full.*/
rnp_status rnp_randnet_fit(rnp_ctx* ctx, const double* Uin, const double* Y, int P);

/* RandNet correction of Eq. randnet for one query per member:
 * out[b] = W_hat^T ReLU(A s(q[b]) + zeta), W_hat the ridge readout of
 * Eq. ridgeless fit on the m nearest stored pairs of q[b] (App. B), solved
 * in its dual m x m form.  A member with no stored pair gets 0.
 *   q, out : device [B][d].                                               */
rnp_status rnp_randnet_predict(rnp_ctx* ctx, const double* q, double* out);

/* Full RandNet-Parareal solve (Alg. 1 with Eq. 3, Eq. 5, Eq. randnet or
 * Eq. 4).  Resets the dataset and scaling, then iterates until every state
 * passed Eq. 5 or max_iters.
 *   u0 : [B][d];  U : [B][N+1][d] receives U_0 .. U_N.  Each of u0 and U
 *        may be device memory or HOST memory (pinned or pageable; told
 *        apart with cudaPointerGetAttributes).  With U in host memory the
 *        states U_0 .. U_L of a member, final once Eq. 5 has set L, are
 *        copied out after every iteration on a copy stream of the context,
 *        overlapping the next iteration; the remaining states at the end
 *        (into pinned memory by a copy kernel through its device address).
 *   stats : host, may be NULL.
 * Returns RNP_OK, or RNP_ENOTCONV with U holding the last iterate.
 * Blocks until the result is in U (also on an error: no copy into U is
 * still in flight when the call returns).                                 */
rnp_status rnp_solve(rnp_ctx* ctx, const double* u0, double* U, rnp_stats* stats);

/* Message of the last failed call on ctx ("" if none).  ctx may be NULL
 * for errors raised by rnp_create and rnp_randnet_predict_noalloc: that
 * message is kept per calling thread. */
const char* rnp_last_error(const rnp_ctx* ctx);

/* --- Alg. 1 one iteration at a time (continuous batching) --------------- */
/* The B members of a context are slots: a member can start while others
 * are iterating, every rnp_iterate advances all active members by one
 * iteration of Alg. 1 (their fine steps share one launch), and a finished
 * member's slot is reused after its result is read.  rnp_solve is these
 * calls for all members at once.                                          */
enum { RNP_MEMBER_FREE = 0, RNP_MEMBER_ACTIVE = 1, RNP_MEMBER_CONVERGED = 2,
       RNP_MEMBER_NOTCONV = 3 };
/* Start a member from u0 (device [d]): the k = 0 coarse sweep of Alg. 1
 * and the member's scaling; empties its dataset.  RNP_EBUSY if the member
 * is active.  Returns after the sweep. */
rnp_status rnp_member_start(rnp_ctx* ctx, int member, const double* u0);
/* One iteration for every active member; *active receives how many are
 * still iterating (host, may be NULL).  Returns after the iteration.     */
rnp_status rnp_iterate(rnp_ctx* ctx, int* active);
/* Host out: rnp_member_state state, iterations done, last converged index. */
rnp_status rnp_member_status(const rnp_ctx* ctx, int member, int* state, int* K, int* L);
/* Copy a finished member's U_0..U_N (device [N+1][d]) and free the slot.
 * RNP_OK (converged) or RNP_ENOTCONV (max_iters reached).                 */
rnp_status rnp_member_result(rnp_ctx* ctx, int member, double* U);

/* --- inspection helpers (not steps of the method) ----------------------- */

/* Copy the random weights of Alg. 3 to device buffers A [M][d], zeta [M]. */
rnp_status rnp_get_weights(rnp_ctx* ctx, double* A, double* zeta);
/* Set (host in) or read (host out) the per-member affine scaling:
 * c, r : host [B][3]; s(u) = (u - c[species]) / r[species].               */
rnp_status rnp_set_scaling(rnp_ctx* ctx, const double* c, const double* r);
rnp_status rnp_get_scaling(rnp_ctx* ctx, double* c, double* r);
/* Drop every stored pair and the scaling. */
rnp_status rnp_reset(rnp_ctx* ctx);
/* Host out: pairs [B] currently stored. */
rnp_status rnp_get_pairs(rnp_ctx* ctx, long long* pairs);
/* Unknowns per state. */
long long rnp_dim(const rnp_problem* prob);
/* Random features phi = ReLU(A s(u) + zeta) (Eq. HA) of R states with the
 * context's scaling, weights and precision (MIXED_BF16: tensor cores).
 * U : device [R][d] (unscaled), phi : device [R][M].  1 <= R <= B N.  Uses
 * the context's fine-step buffer as scratch: not during rnp_iterate.      */
rnp_status rnp_features(rnp_ctx* ctx, const double* U, int R, double* phi);
/* Stencil launch configuration in use: which = 0 fine step, 1 coarse step.
 * out (host, 6 ints): out[0] cluster size, out[1] threads per CTA, out[2]
 * x-points per thread (0 for the FP64 kernel), out[3] rows per thread,
 * out[4] 1 if chosen by timing, out[5] 1 if the step state lives in tensor
 * memory (the wide FP32 kernel). */
rnp_status rnp_stencil_config(const rnp_ctx* ctx, int which, int* out);

/* --- allocation-free prediction (no counterpart in the paper) ----------- */

/* rnp_randnet_predict for callers that cannot allocate device memory when
 * they need a prediction: creating a context allocates, and some callers run
 * where an allocation is not allowed or would synchronise the device (a
 * real-time loop with a fixed memory plan, a host callback on a stream, an
 * application that only hands out pre-allocated buffers).  This call makes
 * the same prediction for one query without a context and calls no
 * allocating routine: the caller passes every input and the output, and the
 * intermediates (scaled query, features, distance partials, ridge weights)
 * live in one fixed file-scope device array of about 5.3 MB (660,518
 * doubles for the limits below, plus 38 ints) that every GPU loading the
 * library keeps until the process exits.
 *   prob       : only pde, grid, M, m and lambda are read.
 *   A, zeta    : device [M][d], [M]  random weights (e.g. rnp_get_weights).
 *   S, Y, Phi  : device [P][d], [P][d], [P][M]  scaled inputs
 *                ((u - c) / r per species), targets F - G, and features
 *                ReLU(A s + zeta) of the stored pairs.
 *   c, r       : host [3]  per-species scaling of the query.
 *   q, out     : device [d]  query (unscaled) and prediction.
 *   status     : device int, may be NULL; receives RNP_OK, or
 *                RNP_ENONFINITE when the ridge system failed or the output
 *                is not finite (out is then 0 or not finite).
 * Limits: d <= 262144, P <= 4096, M <= 1024; larger sizes return RNP_EINVAL
 * before any work (message in rnp_last_error(NULL)).  Work is enqueued on
 * cuda_stream and the call returns without waiting.  Each call looks up the
 * array's device address on the current device; the first call on a device
 * also loads the library's device code there, so make that first call
 * before any stream capture.  Every call on
 * a device shares the one array: calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller.     */
rnp_status rnp_randnet_predict_noalloc(const rnp_problem* prob, const double* A,
                                       const double* zeta, const double* S,
                                       const double* Y, const double* Phi, int P,
                                       const double* c, const double* r,
                                       const double* q, double* out, int* status,
                                       void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
