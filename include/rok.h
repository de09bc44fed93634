/*
 * rok.h -- C ABI of librok.so: matrix-free Rosenbrock-Krylov (ROK) time
 * stepping of semi-discrete compressible flow on one GB300 GPU (sm_103a).
 *
 * The library integrates the autonomous IVP y' = f(y), y in R^N (Sec. 2,
 * Eq. ode), where f is the cell-centred finite-volume residual of the 2-D
 * compressible Euler / Navier-Stokes equations (Sec. 3.2, Eq. Nav_Stokes)
 * or the Lorenz-96 system (appendix).
 *
 * Conventions shared by every entry point
 *   - State vectors are contiguous float64 arrays of N entries in DEVICE
 *     memory, structure of arrays y[var][j][i] with var = (rho, rho u,
 *     rho v, E), i fastest; N = 4 nx ny (Lorenz-96: N = nx).  The caller
 *     owns every pointer it passes; the library owns all workspace, which
 *     it allocates in rok_init (sized for desc.krylov_max) and frees in
 *     rok_destroy -- no step allocates.
 *   - All work is enqueued on the stream given to rok_init (or
 *     rok_set_stream) and is asynchronous unless stated otherwise.
 *   - Calls never abort or trap.  Argument errors are returned at once.
 *     Errors found on the device (non-finite residuals, a singular stage
 *     matrix, Newton non-convergence) are latched in the context; they are
 *     returned by the step call itself when its `info` is non-NULL (that
 *     call then synchronises the stream), otherwise by the next rok_sync.
 *     A step that latches an error leaves y unmodified.
 */
#ifndef ROK_H
#define ROK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rok_ctx rok_ctx; /* opaque, library-owned */

typedef enum {
    ROK_OK = 0,
    ROK_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum or option        */
    ROK_ERR_CUDA = 2,          /* a CUDA runtime call failed               */
    ROK_ERR_NONFINITE = 3,     /* NaN/Inf in a residual or stage solve     */
    ROK_ERR_NOT_CONVERGED = 4, /* ESDIRK Newton iteration did not converge */
    ROK_ERR_TIMEOUT = 5,       /* a bounded device wait expired            */
    ROK_ERR_UNSUPPORTED = 6,   /* valid request this build does not do     */
    ROK_ERR_NOMEM = 7          /* workspace allocation failed              */
} rok_status;

enum { ROK_EULER2D = 0, ROK_NS2D = 1, ROK_LORENZ96 = 2 };
enum { ROK_BC_PERIODIC = 0, ROK_BC_WALL = 1, ROK_BC_FARFIELD = 2 };
enum { ROK_JVP_FD = 0, ROK_JVP_EXACT = 1 };
/* ROK_ROUND_STRICT compiles the stencil without multiply-add contraction, so
 * f(y) is the IEEE result of the written-out formulas (bitwise reproducible
 * against a plain CPU evaluation in the same order); ROK_ROUND_FAST lets the
 * compiler contract into FMA (fewer FP64 instructions, last-bit differences). */
enum { ROK_ROUND_FAST = 0, ROK_ROUND_STRICT = 1 };
/* Krylov basis of the ROK step: binary64, or binary32 storage with binary32
 * Gram-Schmidt (the mixed-precision form; the state, the finite-difference
 * quotient and its eps, the flux accumulation, the Hessenberg / stage solves,
 * the projections phi and the stage vectors stay binary64). */
enum { ROK_BASIS_FP64 = 0, ROK_BASIS_FP32 = 1 };

/* Problem description, copied by rok_init (pointers are not retained). */
typedef struct {
    int kind;            /* ROK_EULER2D | ROK_NS2D | ROK_LORENZ96                     */
    int nx, ny;          /* cells (i fastest); Lorenz-96: nx = N, ny = 1              */
    const double *xv;    /* HOST vertex x, (ny+1)*(nx+1), index j*(nx+1)+i, or NULL    */
    const double *yv;    /* HOST vertex y; NULL together with xv = uniform box         */
    double lx, ly;       /* box size when xv == NULL                                  */
    int bc[4];           /* i-low, i-high, j-low, j-high: ROK_BC_*                    */
    double gamma;        /* ratio of specific heats                                   */
    double prandtl;      /* Prandtl number (Navier-Stokes)                            */
    double mu;           /* viscosity at t_ref (constant when sutherland_s <= 0)      */
    double t_ref;        /* Sutherland reference temperature (T = p/rho, R = 1)        */
    double sutherland_s; /* Sutherland S / t_ref; <= 0: constant viscosity            */
    double q_inf[4];     /* free stream (conservative), far-field ghost state         */
    double muscl_kappa;  /* kappa of the unlimited MUSCL reconstruction               */
    double entropy_fix;  /* Harten coefficient: delta = c (|q_n| + a) on acoustic waves */
    double lorenz_f;     /* Lorenz-96 forcing F                                       */
    int krylov_max;      /* largest Krylov dimension M / GMRES restart length used    */
    int rounding;        /* ROK_ROUND_FAST | ROK_ROUND_STRICT                         */
    int basis;           /* ROK_BASIS_FP64 | ROK_BASIS_FP32 (rok_step / rok_arnoldi)   */
    int jvp;             /* Jacobian-vector products inside rok_step, rok_arnoldi and
                            esdirk_step: ROK_JVP_FD (Eq. matvecFD) or ROK_JVP_EXACT
                            (forward-mode dual numbers, J v to rounding)              */
} rok_problem_desc;

typedef struct {
    int status;          /* rok_status of the step                                     */
    int m_eff;           /* Krylov dimension actually built (Arnoldi breakdown lowers it) */
    int residual_evals;  /* f evaluations, JVPs included                               */
    int jvps;            /* Jacobian-vector products                                   */
    int newton_iters;    /* ESDIRK: Newton iterations, all stages                      */
    int gmres_iters;     /* ESDIRK, ROS4/ROW: GMRES iterations of the step             */
    double eps;          /* finite-difference increment used (Eq. matvecFD)            */
} rok_step_info;

typedef struct {
    int gmres_m;         /* restart length (<= krylov_max)                             */
    double gmres_tol;    /* relative residual tolerance of each linear solve           */
    int gmres_restarts;  /* restarts after the first cycle                             */
    double newton_tol;   /* stop when h g ||dk|| <= newton_tol ||stage state||          */
    int newton_max;      /* Newton iterations per stage                                */
} esdirk_opts;

/* Create a context for one problem on the current CUDA device.  `cuda_stream`
 * is a cudaStream_t (NULL = legacy default stream).  Allocates the Krylov
 * basis ((krylov_max+1) x N float64), stage vectors (8 N) and, for
 * curvilinear grids, the face metrics.  Errors: INVALID_ARG for inconsistent
 * descriptions (non-positive sizes, unknown kind/bc, krylov_max < 0 or > 64,
 * vertex arrays with a uniform-only feature), NOMEM, CUDA. */
rok_status rok_init(rok_ctx **ctx, const rok_problem_desc *desc, void *cuda_stream);

/* Synchronise and free everything the context owns.  NULL is accepted. */
rok_status rok_destroy(rok_ctx *ctx);

/* Change the stream later calls enqueue on. */
rok_status rok_set_stream(rok_ctx *ctx, void *cuda_stream);

/* f = f(y): the semi-discrete residual (Sec. 3.2, Eq. Nav_Stokes with the
 * MUSCL/Roe/central-viscous finite-volume scheme; appendix for Lorenz-96).
 * y, f: device, N float64, must not overlap. */
rok_status rok_residual(rok_ctx *ctx, const double *y, double *f);

/* jv = J(y) v.  mode ROK_JVP_FD: the one-sided finite difference of
 * Eq. matvecFD, (f(y + eps v) - f(y)) / eps; fy = f(y) if the caller has it,
 * else NULL (it is then computed); eps > 0 is used as given (a power of two
 * keeps the quotient exact), eps <= 0 selects sqrt(2^-52 (1 + ||y||)) / ||v||
 * rounded to the nearest power of two.  mode ROK_JVP_EXACT: the exact
 * directional derivative of the discrete residual by forward-mode dual
 * numbers (the alternative the paper points to in Sec. 2.3); fy and eps are
 * ignored.  All arrays device, N float64. */
rok_status rok_jvp(rok_ctx *ctx, const double *y, const double *fy, const double *v, double *jv,
                   double eps, int mode);

/* Arnoldi process of Sec. 2.2.2 alone (modified Gram-Schmidt, FD JVPs):
 * builds V (rows v_1..v_Meff, each N float64, row-major M x N) and
 * H = V^T J V (M x M, row-major, zero beyond Meff) of K_M(J(y), f(y)).
 * V, H: device; m_eff: host (this call synchronises).  M <= krylov_max. */
rok_status rok_arnoldi(rok_ctx *ctx, const double *y, int M, double *V, double *H, int *m_eff);

/* One ROK4 step of size h with Krylov dimension M (Sec. 2.2.2, Eq. ROK),
 * y in place (device, N float64).  0 <= M <= krylov_max; M = 0 is the
 * explicit RK limit.  info may be NULL (no synchronisation). */
rok_status rok_step(rok_ctx *ctx, double *y, double h, int M, rok_step_info *info);

/* One classical RK4 step (Sec. 2.1, Eq. RK), y in place. */
rok_status rk_step(rok_ctx *ctx, double *y, double h, rok_step_info *info);

/* One ESDIRK3 step (Sec. 2.1, Eqs. Newton, SDIRK_Newton, Newton_Jac_Matrix)
 * with matrix-free Newton-GMRES, y in place.  opts NULL = (30, 1e-6, 5,
 * 1e-10, 10).  Host-driven: synchronises the stream every GMRES iteration. */
rok_status esdirk_step(rok_ctx *ctx, double *y, double h, const esdirk_opts *opts, rok_step_info *info);

/* One Rosenbrock step (Sec. 2.2, Eq. ROS), the paper's ROS4 and ROW
 * comparators (table of methods, Sec. 3.1):
 *   Y_i = y_n + h sum_{j<i} alpha_ij k_j,
 *   (I - h g J_n) k_i = f(Y_i) + h J_n sum_{j<i} gamma_ij k_j   (Eq. ROS_stage_eq),
 *   y_{n+1} = y_n + h sum_j b_j k_j,
 * matrix-free: J_n at y_n by Eq. matvecFD (or exactly with ROK_JVP_EXACT),
 * each stage system by GMRES(m) from 0 with the GMRES fields of opts
 * (gmres_m <= krylov_max, gmres_tol, gmres_restarts; the Newton fields are
 * ignored; NULL: m = 30, tol 1e-6, 5 restarts).  method: ROK_ROS_ROS4 (the
 * L-stable order-4 method of Hairer & Wanner IV.7) or ROK_ROS_ROW
 * (ROS34PW2 of Rang & Angermann, order 3 for any Jacobian approximation).
 * Device y in/out, untouched unless every stage system converged
 * (ROK_ERR_NOT_CONVERGED otherwise) and every value is finite.  info:
 * GMRES iterations, Jacobian-vector products, residual evaluations.
 * Synchronises (GMRES decisions on the host). */
enum { ROK_ROS_ROS4 = 0, ROK_ROS_ROW = 1 };
rok_status ros_step(rok_ctx *ctx, double *y, double h, int method, const esdirk_opts *opts, rok_step_info *info);

/* Time step for a CFL number: dt = cfl / max over cells of
 * (|u.S_i| + c|S_i|)/Vol + (|u.S_j| + c|S_j|)/Vol + 2 nu_eff (|S_i|^2 + |S_j|^2)/Vol^2
 * (S_i, S_j mean face-area vectors, nu_eff = max(4/3, gamma/Pr) mu/rho).
 * dt: host; synchronises. */
rok_status rok_dt_from_cfl(rok_ctx *ctx, const double *y, double cfl, double *dt);

/* Wait for the stream and return (and clear) the latched device status;
 * info (nullable) receives the counters of the last step. */
rok_status rok_sync(rok_ctx *ctx, rok_step_info *info);

/* Capture rok_step in a CUDA graph per (y, M) and replay it (1) or launch
 * kernel by kernel (0, default). */
rok_status rok_set_graph(rok_ctx *ctx, int enable);

/* Modified Gram-Schmidt of the Arnoldi process (Sec. 2.2.2) and its reverse in
 * rok_step_vjp: one persistent cooperative launch per Krylov column where the
 * device holds the whole grid (1, default), or one launch per pass (0) -- the
 * path that grids beyond the persistent kernels' reach (more than 2 x 2048
 * entries per co-resident CTA) always take.  Both compute the same sums in
 * the same order.  Synchronises the context stream and drops its captured
 * step graphs.  ROK_ERR_UNSUPPORTED for 0 with the binary32 basis, which runs
 * on the persistent kernel only. */
rok_status rok_set_persistent(rok_ctx *ctx, int enable);

/* Kernel launch counter (all kernels this context launched) and, when
 * timing is on, the accumulated device time of the residual/JVP stencil
 * launches measured with CUDA events on the context stream. */
typedef struct {
    long long launches;         /* kernels launched since the last reset        */
    long long stencil_launches; /* residual / JVP stencil launches              */
    double stencil_ms;          /* summed event time of timed stencil launches  */
    long long stencil_timed;    /* number of stencil launches timed             */
} rok_counters;
rok_status rok_get_counters(rok_ctx *ctx, rok_counters *c, int reset);
rok_status rok_set_stencil_timing(rok_ctx *ctx, int enable);

const char *rok_status_string(rok_status s);

/* ---- Adaptive time stepping ---------------------------------------------
 *
 * Integrate y' = f(y) from 0 to T with step sizes chosen by an embedded error
 * estimate (the paper compares its methods with adaptive steps, Sec. 4.2).
 * err = sqrt(sum_i (e_i / sc_i)^2 / N), sc_i = atol + rtol max(|y_i|, |ynew_i|);
 * a step is accepted when err <= 1; the next step is
 * h min(facmax, max(facmin, safety err^(-1/(q+1)))), q the embedded order,
 * never larger than h right after a rejection; a non-finite err (or a step that
 * latches a non-finite residual) is rejected with facmin; the last step ends
 * at T.  y: device, N float64, in place.  Synchronises every step.  Returns
 * ROK_ERR_NOT_CONVERGED when max_steps attempts do not reach T. */
typedef struct {
    double atol, rtol;   /* error weights                                         */
    double h0;           /* first trial step (> 0)                                */
    double safety;       /* 0.9 is usual                                          */
    double facmin;       /* smallest step ratio (0.2)                             */
    double facmax;       /* largest step ratio (5)                                */
    int max_steps;       /* accepted + rejected attempts                          */
} rok_adapt_opts;

typedef struct {
    int accepted, rejected;
    double t;            /* time reached                                          */
    double h_next;       /* step the controller proposes next                     */
    long long residual_evals;
} rok_adapt_info;

/* ROK4 steps (Krylov dimension M) with the embedded order-2 estimate
 * e = sum_i (b_i - bhat_i) k_i (q = 2). */
rok_status rok_integrate(rok_ctx *ctx, double *y, double T, int M, const rok_adapt_opts *opts,
                         rok_adapt_info *info);

/* Dormand-Prince 5(4) steps (comparator; q = 4, first same as last). */
rok_status dopri5_integrate(rok_ctx *ctx, double *y, double T, const rok_adapt_opts *opts, rok_adapt_info *info);

/* ---- Reverse mode: gradients of a final-time functional ------------------
 *
 * For a scalar functional of the state after K steps, the gradient with
 * respect to the initial state and the viscosity is accumulated backward step
 * by step: ybar_n = (d y_{n+1} / d y_n)^T ybar_{n+1}, plus each step's
 * viscosity part.  The derivative is that of the discrete step map (the
 * discrete adjoint), with the finite-difference increment eps of
 * Eq. matvecFD held constant.  Supported: every problem and grid of
 * rok_init with finite-difference JVPs (the reverse step of the exact-JVP
 * step returns ROK_ERR_UNSUPPORTED: it would need second derivatives of f).
 * With the binary32 basis the reverse runs in binary64 on the basis the
 * step built, widened exactly: the derivative of the exact-arithmetic
 * Arnoldi process (MGS and classical Gram-Schmidt twice coincide there) at
 * the rounded basis.  Euler / Navier-Stokes grids take a hand-written
 * reverse sweep of the face fluxes (uniform and curvilinear, every boundary
 * condition; a few residuals' cost per product); Lorenz-96 and curvilinear
 * grids of fewer than 2 cells in a direction take J^T u from a compressed
 * Jacobian: 4 px py exact JVPs (px for Lorenz-96), px and py the smallest
 * divisors >= 5 of a periodic extent (the extent itself if none; 5 across
 * walls and far fields).  "The viscosity" mu is desc->mu: the
 * constant viscosity, or the viscosity at t_ref under Sutherland's law
 * (mu(T) = mu g(T); the residual is affine in mu either way). */

/* ybar = J(y)^T ubar (the transposed Jacobian of the residual of
 * rok_residual) and, if mubar is non-NULL (HOST), mubar = ubar . df/dmu(y)
 * (0 for Euler; this call then synchronises).  y, ubar, ybar: device, N
 * float64; ybar must not overlap the inputs.  Deterministic (no atomics). */
rok_status rok_vjp(rok_ctx *ctx, const double *y, const double *ubar, double *ybar, double *mubar);

/* Reverse of one rok_step(ctx, y, h, M): given ybar_in = dJ/dy_{n+1}, writes
 * ybar_out = (dy_{n+1}/dy_n)^T ybar_in and, if mubar is non-NULL (HOST), the
 * viscosity part dJ/dmu contributed by this step.  The step is recomputed from
 * y (= y_n, unchanged).  y, ybar_in, ybar_out: device, N float64; ybar_out may
 * equal ybar_in but not y.  Synchronises.  Workspace: about M + 20 state
 * vectors, allocated on the first call. */
rok_status rok_step_vjp(rok_ctx *ctx, const double *y, double h, int M, const double *ybar_in, double *ybar_out,
                        double *mubar);

/* Tapes: the reverse of a step without recomputing the step.  A tape holds
 * what the reverse of one ROK4 step (Sec. 2.2.2, Eq. ROK; Arnoldi of
 * Sec. 2.2.1 with the JVP of Eq. matvecFD) reads: y_n, the F_i and k_i, the
 * Krylov basis, H with its LU, lambda_i and phi_i, and the last column's
 * orthogonalised JVP, about (10 + M) state vectors.  The tape is plain device
 * memory owned by the caller, 256-byte aligned, rok_tape_bytes bytes for
 * Krylov dimension M, and is only read by the library after it was written.
 *
 * rok_tape_bytes: *bytes (HOST) = the size of a tape for Krylov dimension M.
 * rok_step_record: rok_step(ctx, y, h, M, NULL) that also writes the tape
 *   (y: device, N float64, in/out, y_{n+1} on return; tape: device, must not
 *   overlap y); y_{n+1} is bit-identical to rok_step's.  Synchronises once.
 *   Same support as rok_step_vjp; on an error status y is unchanged.
 * rok_step_vjp_tape: rok_step_vjp(ctx, y_n, h, M, ybar_in, ybar_out, mubar)
 *   from a tape that rok_step_record wrote on a context of the same problem;
 *   bit-identical to it.  ybar_out must overlap neither the tape nor y_n.
 *   ROK_ERR_INVALID_ARG for a tape whose header does not match this context.
 *   Overwrites the context's step internals (as any step does). */
rok_status rok_tape_bytes(rok_ctx *ctx, int M, size_t *bytes);
rok_status rok_step_record(rok_ctx *ctx, double *y, double h, int M, void *tape);
rok_status rok_step_vjp_tape(rok_ctx *ctx, const void *tape, const double *ybar_in, double *ybar_out,
                             double *mubar);

/* ---- Batches: many independent instances stepped together ---------------
 *
 * The paper integrates one problem at a time; a batch steps `count`
 * independent problems with the same ROK4 step (Sec. 2.2.2, Eq. ROK), every
 * kernel launch covering all of them, so that small grids fill the GPU.
 *
 * Instances: uniform periodic grids (xv == NULL, every bc ROK_BC_PERIODIC) of
 * kind ROK_EULER2D or ROK_NS2D.  They fall into three physics groups: Euler,
 * Navier-Stokes with constant viscosity, Navier-Stokes with Sutherland's law.
 * nx, ny, lx, ly and mu are per instance; within a group gamma, muscl_kappa,
 * entropy_fix (and prandtl, resp. t_ref and sutherland_s, where they apply)
 * must agree, and rounding and krylov_max across the whole batch
 * (ROK_ERR_INVALID_ARG otherwise); basis must be ROK_BASIS_FP64 and jvp
 * ROK_JVP_FD (ROK_ERR_UNSUPPORTED otherwise).
 *
 * Layout: the states of all instances form ONE flat device float64 array of
 * `total` entries (rok_batch_layout).  Instance k's 4 nx_k ny_k entries, in the
 * single-problem order y[var][j][i], start at element offsets[k], a multiple
 * of 2048; the entries between instances are padding that the library never
 * reads or writes.  Each instance's result equals that of rok_step on the same
 * description, state and h: bit for bit under ROK_ROUND_STRICT (the same
 * reduction trees), to rounding under ROK_ROUND_FAST.
 *
 * Launch shapes: the residual stencil runs with one of three tile shapes per
 * physics group and the vector passes with a chosen number of 2048-entry
 * chunks per CTA.  rok_batch_tune times the candidates on the batch's own data
 * and keeps the fastest; every candidate yields the same result bits. */
typedef struct rok_batch rok_batch; /* opaque, library-owned */

enum { ROK_TILE_32x8 = 0, ROK_TILE_16x16 = 1, ROK_TILE_64x4 = 2 };
typedef struct {
    int tile[3];          /* stencil tile per group: Euler, NS, NS with Sutherland (ROK_TILE_*) */
    int chunks_per_cta;   /* reduction / MGS passes: 1, 2, 4 or 8                            */
    int vec_chunks_per_cta; /* stage vectors, first basis vector, update: 1, 2, 4 or 8       */
    float stencil_ms[3][3]; /* rok_batch_tune: residual launch time per group and tile (-1: none) */
    float mgs_ms[4];      /* rok_batch_tune: one MGS pass per chunks_per_cta in (1, 2, 4, 8)   */
    float vec_ms[4];      /* rok_batch_tune: one stage-vector pass per vec_chunks_per_cta       */
} rok_batch_tuning;

/* Create a batch of `count` >= 1 instances on the current device; workspace as
 * for rok_init, sized for the flat length.  Errors as rok_init, plus those above. */
rok_status rok_batch_init(rok_batch **batch, const rok_problem_desc *descs, int count, void *cuda_stream);
rok_status rok_batch_destroy(rok_batch *batch);

/* total: flat length; offsets (nullable, host, `count` entries): first entry of
 * each instance. */
rok_status rok_batch_layout(const rok_batch *batch, size_t *total, size_t *offsets);

/* f = f(y) for every instance (flat device arrays, must not overlap). */
rok_status rok_batch_residual(rok_batch *batch, const double *y, double *f);

/* `nsteps` >= 1 ROK4 steps of every instance with Krylov dimension M
 * (0 <= M <= krylov_max), instance k with step size h[k] (HOST array of
 * `count` positive finite values, read during the call).  y in place.  An
 * instance whose step latches an error (non-finite residual or stage solve)
 * keeps its last good state for the remaining steps; its error is reported in
 * info[k].status.  info: nullable HOST array of `count` entries; when given,
 * the call synchronises and returns the first non-OK instance status (or OK),
 * and clears the latched statuses.  With graphs enabled the nsteps steps are
 * captured once per (y, M, nsteps) into one CUDA graph and replayed. */
rok_status rok_batch_step(rok_batch *batch, double *y, const double *h, int M, int nsteps, rok_step_info *info);

/* Time the launch-shape candidates on state y (flat device array, unchanged)
 * and keep the fastest; out (nullable) receives the choice and the times.
 * Synchronises. */
rok_status rok_batch_tune(rok_batch *batch, const double *y, rok_batch_tuning *out);
/* Set the launch shapes explicitly (the time fields are ignored). */
rok_status rok_batch_set_tuning(rok_batch *batch, const rok_batch_tuning *t);
rok_status rok_batch_get_tuning(const rok_batch *batch, rok_batch_tuning *t);
rok_status rok_batch_set_graph(rok_batch *batch, int enable);
/* kernels launched since the last reset (graph replays count their nodes) */
rok_status rok_batch_get_launches(rok_batch *batch, long long *launches, int reset);

/* Allocation-free variant of rok_jvp (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory: code that runs inside a
 * host application which owns every device allocation (a plug-in whose host
 * framework forbids or pools cudaMalloc), and loops that must not call
 * cudaMalloc/cudaFree because those calls synchronise the device.  Such a
 * caller cannot create a rok_ctx (rok_init allocates the Krylov basis and the
 * workspace), so this call takes the problem description directly and keeps
 * its scratch -- the reduction partials of ||y||^2 and ||v||^2, eps, 1/eps and
 * the status word -- in one static device array of about 134 KB that every GPU
 * loading the library holds until the process exits.
 *
 * Computes jv = (f(y + eps v) - fy) / eps exactly as rok_jvp with the same
 * description and rounding mode (same kernels, same result bits).
 *   desc   uniform periodic Euler / Navier-Stokes grids (xv == NULL) or
 *          Lorenz-96; curvilinear grids return ROK_ERR_UNSUPPORTED (their
 *          metrics would need device memory), and so does desc->jvp other than
 *          ROK_JVP_FD (this call computes the finite-difference product only);
 *          desc->krylov_max and desc->basis are not used (no Krylov basis).
 *   y, fy, v, jv  device, N float64 (N = 4 nx ny, Lorenz-96: nx); fy = f(y)
 *          is required; jv must not overlap the inputs.
 *   eps    > 0 used as given; <= 0 selects the power-of-two increment of rok_jvp.
 *   status nullable DEVICE int: receives the latched error bits of this call
 *          (0 = ok, nonzero = a non-finite value was produced).
 * N beyond ROK_NOALLOC_MAX_N returns ROK_ERR_INVALID_ARG without launching.
 * Calls no cudaMalloc, cudaFree or allocating routine.  The first call on a
 * device resolves the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture.  A cudaDeviceReset of a device discards the
 * array and the kept address with it: do not call this entry point on that
 * device again in the same process (reload the library).  All calls
 * share the one array: calls whose execution overlaps on the GPU (different
 * streams, or concurrent host threads) race on it and must be serialised by
 * the caller.  Asynchronous on cuda_stream. */
#define ROK_NOALLOC_MAX_N (4096 * 2048)
rok_status rok_jvp_noalloc(const rok_problem_desc *desc, const double *y, const double *fy, const double *v,
                           double *jv, double eps, int *status, void *cuda_stream);

/* Measurement utility (no counterpart in the paper): FP64 fused-multiply-add
 * throughput of the current device in TFLOP/s (2 flops per FMA), from
 * `repeats` timed launches of independent FMA chains.  Synchronises. */
rok_status rok_fp64_fma_peak(double *tflops, int repeats);

/* Self-test of the reciprocal of the FMA-build stencil (no counterpart in the
 * paper).  r[k] = the stencil's 1/x[k]: the hardware estimate
 * (rcp.approx.ftz.f64) refined by one third-order Newton step.  For
 * 2^-1022 <= |x| <= 2^1022 it is within one unit in the last place of the
 * IEEE quotient 1/x; the stencil applies it only to densities and sums of
 * square roots of densities, which lie far inside that range.  Outside it the
 * estimate's flush to zero decides: a subnormal, zero or infinite x gives NaN
 * (the non-finite check of the residual then reports it), |x| > 2^1022 gives
 * a signed zero.  x, r: DEVICE, n float64 each (n >= 0).  Asynchronous on
 * cuda_stream. */
rok_status rok_selftest_rcp(const double *x, double *r, long long n, void *cuda_stream);

/* Self-test of the bounded waits (no counterpart in the paper).  The
 * persistent Gram-Schmidt column kernels wait for the other CTAs of their
 * launch on per-pass arrival counters, each wait bounded by a poll limit after
 * which the kernel latches a timeout in the context's status and returns
 * (ROK_ERR_TIMEOUT from the step).  This call runs that wait routine in one
 * CTA on a counter that nothing advances, with a limit of `polls` (1 ..
 * 4194304, the kernels' own limit), and reports in *expired (HOST) whether the
 * wait gave up and latched the timeout (1) as designed; *ms (HOST, nullable)
 * is its GPU time.  The context's status is put back as it was and the
 * context stays usable.  Uses the context's counters (not while a step is in flight on its
 * stream).  Synchronises. */
rok_status rok_selftest_wait(rok_ctx *ctx, long long polls, int *expired, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* ROK_H */
