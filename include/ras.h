/*
 * ras.h - C ABI of the GB300 (sm_103a) RAS / RASPEN solver.
 *
 * The library solves the eps-smoothed, reduced first-order optimality system
 * of the L1-regularised semilinear elliptic optimal control problem (P) of
 * Ciaramella, Kartmann & Mueller, arXiv 2411.00546:
 *
 *   F_y = A y + phi(y) - f + (1/nu) (p + mu P_eps(-p/mu)) = 0
 *   F_p = A p + phi'(y) p - y + y_d                     = 0      (Sec. 3.3)
 *
 * on Omega = (0,1)^2 with A = -Laplace (5-point finite differences, zero
 * Dirichlet data) and P_eps the smoothed projection of Sec. 3.1, by the
 * restricted-additive-Schwarz methods of Sec. 4: the nonlinear RAS function
 * (Alg. 3), RASPEN (Alg. 2) and Newton_RAS (Alg. 1 with RAS-preconditioned
 * GMRES).
 *
 * Conventions for every entry point:
 *  - Grid functions (y, p, y_d, f, residuals, directions) are n*n FP64 arrays,
 *    row-major with the x1 index fastest: element [j*n + i] is the node
 *    ((i+1)h, (j+1)h), h = 1/(n+1). Pointers are DEVICE pointers unless the
 *    name says _host. The caller owns them; they must stay valid for the call.
 *  - The library allocates (cudaMalloc) and owns its internal buffers
 *    (local factors, Krylov basis, scratch) from ras_create until ras_destroy.
 *  - All GPU work is enqueued on the CUDA stream given to ras_create. Every
 *    call returns after that work is complete (it synchronises the stream).
 *  - Return value: RAS_OK (0) or a positive success variant, or a negative
 *    RAS_E* code. After an error, ras_last_error() describes it. A CUDA error
 *    is reported as RAS_ECUDA and leaves the handle usable only for
 *    ras_destroy.
 *  - One problem handle may be used by one host thread at a time.
 */
#ifndef RAS_H
#define RAS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define RAS_OK           0   /* converged by the tolerance test               */
#define RAS_OK_FLOOR     1   /* converged: residual at FP64 rounding level     */
#define RAS_EINVAL      -1   /* invalid argument                               */
#define RAS_ENOMEM      -2   /* device allocation failed                       */
#define RAS_ENOCONV     -3   /* iteration limit reached (Alg. 1 / Alg. 2 kmax) */
#define RAS_ESINGULAR   -5   /* zero pivot in a local factorisation            */
#define RAS_ENONFINITE  -6   /* NaN or Inf in a residual                       */
#define RAS_ETIMEOUT    -7   /* a bounded device-side wait ran out; the kernel
                                gave up cleanly and the context stays usable   */
#define RAS_ENOTIMPL    -8   /* not available in this library version          */
#define RAS_ECUDA       -9   /* CUDA runtime error                             */
#define RAS_ESTATE     -10   /* call needs state that is not there (e.g. a JVP
                                 before any ras_apply)                          */

/* Nonlinearity phi of the state equation (Assumption 1: C^2, increasing). */
#define RAS_PHI_CUBIC 0      /* phi(y) = y^3                                  */
#define RAS_PHI_EXP   1      /* phi(y) = exp(y)                               */
#define RAS_PHI_KAPPA 2      /* phi(y) = kappa (y^3 + exp(kappa y)), Sec. 4   */

/* Arithmetic of the local factorisations and solves. */
#define RAS_FP64  0          /* everything in FP64                            */
#define RAS_MIXED 1          /* FP32 local factors and solves; FP64 residuals,
                                iterative refinement of every local Newton
                                direction in FP64, FP64 GMRES, line search and
                                stop tests                                     */

/* Solver parameters. ras_default_opts fills the paper's values (Sec. 5). */
typedef struct {
    double tol;            /* outer tolerance (Alg. 1 / Alg. 2), 1e-10      */
    double inner_tol;      /* tolerance of the local Newton solves, 1e-8     */
    double sigma;          /* relaxed backtracking parameter, 1.1            */
    double eps0;           /* initial smoothing parameter, 1                 */
    double gamma;          /* continuation factor eps <- max(gamma eps, eps_min), 1/5 */
    double eps_min;        /* target smoothing parameter                     */
    int    kmax_outer_raspen;   /* 50  */
    int    kmax_outer_newton;   /* 200 */
    int    kmax_inner;          /* 100; a local solve stopped there keeps its
                                   iterate (Alg. 1) and counts as a local failure */
    int    max_halvings;        /* 20: backtracking halvings per step         */
    int    gmres_restart;       /* 30  */
    int    gmres_maxit;         /* 1000 total Krylov steps per linear solve    */
    double gmres_rtol;          /* 1e-8 relative to the right-hand side        */
    double floor_factor;        /* 16: rounding-floor stop multiplier          */
    int    precision;           /* RAS_FP64 or RAS_MIXED                       */
    int    ir_max;              /* mixed: max refinement corrections, 6        */
    double ir_rtol;             /* mixed: refine until ||r|| <= ir_rtol ||b||, 1e-12 */
    double kappa;               /* parameter of RAS_PHI_KAPPA, 0.1             */
    int    jvp_ir;              /* mixed: FP64 refinement corrections of every
                                   local solve inside the Jacobian action of
                                   Alg. 4, 2 (0 = plain FP32 solves). One
                                   correction leaves the action's relative
                                   error near (cond(J_i) 2^-24)^2 ~ 1e-8, which
                                   moves the final iterate's smaller field (y
                                   beside p when the L1 control is inactive) by
                                   about that much relative to its own size;
                                   two bring it to FP64 rounding level      */
    int    wait_test;           /* 0. 1 = test of the failure path: the first
                                   streamed slab wait of every local solve
                                   gives up at once, the copies already issued
                                   are drained, and the call returns
                                   RAS_ETIMEOUT; set it back to 0 with
                                   ras_set_opts to go on with the handle    */
} ras_opts;

/* Counters of the last solve or RASPEN-function evaluation. */
typedef struct {
    int    status;         /* RAS_OK, RAS_OK_FLOOR or RAS_E*                  */
    int    outer_its;      /* outer Newton steps (RASPEN or Newton_RAS)       */
    int    gmres_its;      /* Krylov steps, summed over the outer steps       */
    int    evaluations;    /* RASPEN-function evaluations (Alg. 3 calls)      */
    int    inner_its_max;  /* max local Newton steps of one subdomain, summed
                              over evaluations                                  */
    long long inner_its_sum;  /* sum over subdomains and evaluations         */
    int    halvings;       /* backtracking halvings, all levels               */
    int    exhausted;      /* steps taken after max_halvings failed halvings  */
    int    local_failures; /* local solves that ended with a negative status:
                              kmax_inner reached (the evaluation goes on with
                              the iterate), or non-finite / singular (the call
                              fails with that status)                          */
    double res0;           /* ||F(x0)|| (Newton_RAS) or ||RASPEN F(x0)||       */
    double res;            /* final norm of the same quantity                 */
    double eps_final;      /* smoothing parameter of the final iterate        */
} ras_stats;

typedef struct ras_problem ras_problem;

/* Fill *o with the paper's settings (Sec. 5): tol 1e-10, inner_tol 1e-8,
 * sigma 1.1, eps0 1, gamma 1/5, eps_min 1e-6 (the paper sweeps eps_min), and
 * this library's defaults for the unspecified rest. Returns RAS_EINVAL on NULL. */
int ras_default_opts(ras_opts* o);

/* Create a problem on an n x n grid split into sx x sy non-overlapping blocks
 * (balanced sizes, larger blocks first), each grown by `overlap` node layers on
 * every side and clipped at the boundary (Sec. 4.2).
 *   phi      RAS_PHI_*; nu, mu > 0 are the cost weights of (P) (Sec. 1).
 *   y_d      device, n*n, copied (the caller keeps ownership).
 *   f        device, n*n, copied; NULL means f = 0.
 *   o        options (copied); NULL means ras_default_opts.
 *   stream   cudaStream_t to use, NULL for the legacy default stream.
 * Limits: n >= 2, 1 <= sx, sy <= n, overlap >= 0, and every local block row
 * has 2*wx <= 512 unknowns (wx = subdomain width in nodes, overlap included)
 * -> RAS_EINVAL. Rows of up to 160 unknowns take the register-tile
 * factorisation and the streamed solves; wider ones (the paper's 2 x s and
 * small s x s layouts) a factorisation of the block in its HBM slot by a
 * cluster of eight 1024-thread CTAs, and solves that stream the blocks by TMA,
 * one CTA per subdomain. Narrow rows check partial pivoting per block and
 * redo a block that needs row interchanges with them; wide rows pivot inside
 * their blocked elimination (partial pivoting with implicit interchanges).
 * On success *out receives the handle. */
int ras_create(int n, int sx, int sy, int overlap, int phi, double nu, double mu,
               const double* y_d, const double* f, const ras_opts* o,
               void* stream, ras_problem** out);

/* Create a problem on the unit cube (Assumption 1 allows Omega in R^2 or R^3;
 * Sec. 2): an n x n x n grid of interior nodes, the 7-point stencil
 * A = -Laplace (beta (6 z - the six neighbours), beta = (n+1)^2), split into
 * sx x sy x sz non-overlapping boxes (balanced sizes, larger first; box index
 * (bz*sy + by)*sx + bx), each grown by `overlap` node layers and clipped.
 * Grid functions are n^3 FP64 with x1 fastest, then x2, then x3 (node
 * (i, j, k) at (k*n + j)*n + i); y_d and f as in ras_create with n^3 entries.
 * The local Jacobian of a box is block tridiagonal over its x3 planes, so
 * every box plane must have 2*wx*wy <= 512 unknowns (wx, wy = box extents
 * along x1 and x2, overlap included; up to 160 on the register-tile path)
 * -> RAS_EINVAL otherwise; 1 <= sz <= n.
 * Every call that takes a handle works on the result (vectors of 2*n^3, or
 * n^3 per field) except ras_residual_static, the batch and the server, which
 * describe square problems only. */
int ras_create3(int n, int sx, int sy, int sz, int overlap, int phi, double nu, double mu,
                const double* y_d, const double* f, const ras_opts* o,
                void* stream, ras_problem** out);

/* 2 for a handle made by ras_create / ras_batch_create (the square), 3 for
 * one made by ras_create3 (the cube); RAS_EINVAL on NULL. */
int ras_problem_dim(const ras_problem* h);

/* A batch of independent problems in one handle (many problems of uneven
 * grid size, one launch per sweep step for all of them). Each entry describes one problem
 * exactly like the arguments of ras_create; y_d and f are device pointers,
 * copied. All problems share the options. The subdomains of all problems form
 * one table: every step of a RASPEN-function evaluation (Alg. 3) is one launch
 * for the whole batch, and the FP32 factorisation is launched once per
 * register-tile class (block size mp = 2*wx rounded up to 32, tile mp/16),
 * with one more launch for the wide-block subdomains of all problems.
 * Limits as in ras_create, per problem; 1 <= count <= 4096. */
typedef struct {
    int n, sx, sy, overlap, phi;
    double nu, mu;
    const double* y_d;
    const double* f;
} ras_problem_desc;
int ras_batch_create(int count, const ras_problem_desc* problems, const ras_opts* o, void* stream,
                     ras_problem** out);

/* Number of problems in the handle (1 for ras_create). */
int ras_problem_count(const ras_problem* h);

/* RASPEN (Alg. 2) for every problem of a batch, in lockstep: the RASPEN-
 * function evaluations and the Krylov steps of all problems still iterating
 * share their launches; each problem stops on its own test. y[k], p[k]: device
 * n_k*n_k arrays (initial guess in, solution out). stats: `count` entries, or
 * NULL. Returns the worst status. The single-problem entry points other than
 * ras_raspen_solve take only handles with one problem (else RAS_EINVAL). */
int ras_batch_raspen_solve(ras_problem* h, double* const* y, double* const* p, ras_stats* stats);

/* ---------------------------------------------------------------- serving
 * Continuous batching of RASPEN_eps solves (Alg. 2): requests of any size and
 * any (nu, mu, phi, y_d, f) are submitted at any time; every ras_server_step
 * admits waiting requests while the budget allows, then advances every
 * admitted request by one phase step: a request in its evaluation phase
 * evaluates the RASPEN function at x_k (eps-continuation in the local solves
 * when k = 0) and tests it (finished, or on to GMRES); a request in its GMRES
 * phase runs one restart cycle of GMRES(m), and when GMRES stops takes
 * x_{k+1} = x_k + d and returns to evaluation. The local solves, Jacobian
 * actions and Krylov vectors of all requests in a phase share launches. A
 * request's iterate, data, GMRES state and local factors stay on the device
 * between steps; a finished request holds its result until fetched. Each
 * request's sequence of operations is that of ras_raspen_solve on the
 * problem alone (same x0 = 0, same options), so its result agrees with the
 * solve alone to rounding.
 *
 * ras_server_create: hbm_budget = device bytes the server may hold (request
 *   storage of admitted and unfetched requests plus the two batch workspaces,
 *   one per phase, each at most the admitted set's workspace estimate: a
 *   request is charged slot + 2 x workspace bytes of ras_server_request_bytes); max_active = most requests
 *   advanced together (1..4096); o = options shared by all requests (NULL:
 *   defaults); stream = cudaStream_t for all work. RAS_EINVAL on bad values.
 * ras_server_request_bytes: host-only estimate for one request: slot bytes
 *   (y, p, y_d, f) and workspace bytes. RAS_EINVAL for an invalid desc.
 * ras_server_submit: desc as for ras_batch_create, but y_d and f are HOST
 *   pointers (n*n doubles, copied before the call returns). Queues the
 *   request (first come, first served); *id receives its id (> 0).
 *   RAS_ENOMEM if the request alone exceeds the budget.
 * ras_server_step: admission, then one phase step of every admitted request; *active = requests still admitted after it, *finished = requests
 *   that finished in it (either pointer may be NULL). With nothing admitted it
 *   only admits. Returns RAS_OK, or RAS_ECUDA / RAS_ETIMEOUT (the server must
 *   then be destroyed).
 * ras_server_counts: requests waiting, admitted, finished and not fetched.
 * ras_server_finished_ids: up to cap ids of finished requests, oldest first;
 *   returns how many were written.
 * ras_server_fetch: copies the result of finished request id to y_host,
 *   p_host (n*n doubles each, either may be NULL) and its stats, frees its slot
 *   and returns its status (RAS_OK or RAS_ENOCONV); RAS_EINVAL for an unknown
 *   id. An idle server (nothing waiting or admitted) then releases its
 *   workspace.
 * ras_server_cancel: drops request id wherever it is (waiting, admitted or
 *   finished), freeing its storage; RAS_EINVAL for an unknown id. Between
 *   steps only (the server is not thread-safe).
 * ras_server_device_bytes: device bytes held now (workspace + slots).
 * The paper has no serving loop: this is a continuous-batching use of Alg. 2
 * and Alg. 3 over independent problems. */
typedef struct ras_server ras_server;
int ras_server_create(size_t hbm_budget, int max_active, const ras_opts* o, void* stream, ras_server** out);
int ras_server_request_bytes(const ras_problem_desc* d, const ras_opts* o, size_t* slot_bytes,
                             size_t* scratch_bytes);
int ras_server_submit(ras_server* s, const ras_problem_desc* d, long long* id);
int ras_server_step(ras_server* s, int* active, int* finished);
int ras_server_counts(const ras_server* s, int* pending, int* active, int* finished);
int ras_server_finished_ids(const ras_server* s, long long* ids, int cap);
int ras_server_fetch(ras_server* s, long long id, double* y_host, double* p_host, ras_stats* st);
int ras_server_cancel(ras_server* s, long long id);
/* CUDA graphs (ras_use_graphs) in the server's workspaces, default off: a
 * workspace's graphs would be captured again after every relayout (whenever
 * the set of requests in a phase changes), which costs more than the
 * per-step host reads they save (on the 32-request stream sample: p50
 * latency 14.5 s with graphs, 13.0 s without). RAS_EINVAL on a NULL server. */
int ras_server_use_graphs(ras_server* s, int enable);
size_t ras_server_device_bytes(const ras_server* s);
const char* ras_server_last_error(const ras_server* s);
void ras_server_destroy(ras_server* s);

/* Set the target smoothing parameter eps_min (> 0; P_eps is not smooth at 0). */
int ras_set_eps(ras_problem* h, double eps_min);

/* Replace the options (validated as in ras_create; layout fixed at create). */
int ras_set_opts(ras_problem* h, const ras_opts* o);

/* Replace y_d (and f; NULL means 0). Device pointers, n*n, copied. */
int ras_set_data(ras_problem* h, const double* y_d, const double* f);

/* F(x, eps) of Sec. 3.3 at x = (y, p): writes Fy, Fp (device, n*n; either may
 * be NULL) and, if norm_host != NULL, ||(Fy, Fp)||_2 to *norm_host. */
int ras_residual(ras_problem* h, const double* y, const double* p, double eps,
                 double* Fy, double* Fp, double* norm_host);

/* The RASPEN function of Alg. 3 / Sec. 4.2 at x = (y, p):
 *   F_eps(x) = sum_i tilde P_i C_i(x),  R_i F_eps(x + P_i C_i(x)) = 0,
 * each C_i computed by Alg. 1 from 0 with a direct local solve; with
 * continuation != 0 the local solves run eps from eps0 down to eps_min, else
 * they start at eps_min. Writes Fy, Fp (device, n*n). Keeps the local
 * Jacobians factorised at x^(i) = x + P_i C_i(x) for ras_jvp. *stats (may be
 * NULL) receives the local iteration counts. Returns the worst local status. */
int ras_apply(ras_problem* h, const double* y, const double* p, int continuation,
              double* Fy, double* Fp, ras_stats* stats);

/* Jacobian action of the RASPEN function at the x of the last ras_apply
 * (Alg. 4): out = F_eps'(x) d = -d - sum_i tilde P_i J_i(x^(i))^-1 B_i d,
 * where B_i d = R_i A (I - P_i R_i) d is the coupling of d outside Omega_i
 * (the transmission identity of Sec. 4.2). Device n*n arrays.
 * RAS_ESTATE if no ras_apply has run. */
int ras_jvp(ras_problem* h, const double* dy, const double* dp, double* oy, double* op);

/* Linear RAS preconditioner at x (Newton_RAS, Sec. 4.1):
 *   z = sum_i tilde P_i (R_i F_eps'(x) P_i)^-1 R_i r.
 * Factorises the local Jacobians at (x, eps), then applies them to r. */
int ras_precondition(ras_problem* h, const double* y, const double* p, double eps,
                     const double* ry, const double* rp, double* zy, double* zp);

/* RASPEN (Alg. 2): Newton on F_eps(x) = 0 with x <- x + d, d from GMRES with
 * the action of Alg. 4; eps-continuation only in the local solves of the first
 * evaluation. (y, p): device n*n, initial guess on entry, solution on exit. */
int ras_raspen_solve(ras_problem* h, double* y, double* p, ras_stats* stats);

/* Newton_RAS (Alg. 1 on F_eps(x) = 0, eps-continuation when eps0 > eps_min,
 * GMRES right-preconditioned by linear RAS). In/out as ras_raspen_solve. */
int ras_newton_ras_solve(ras_problem* h, double* y, double* p, ras_stats* stats);

/* Newton (Alg. 1 on F_eps(x) = 0, eps-continuation when eps0 > eps_min: the
 * paper's Newton / Newton_eps baselines of Sec. 5) with unpreconditioned
 * GMRES on the global Jacobian F_eps'(x) applied matrix-free in FP64 (no local
 * factorisations). In/out as ras_raspen_solve; single-problem handles only
 * (else RAS_EINVAL); RAS_ENOCONV when kmax_outer_newton is reached. */
int ras_newton_solve(ras_problem* h, double* y, double* p, ras_stats* stats);

#define RAS_METHOD_RASPEN     0
#define RAS_METHOD_NEWTON_RAS 1
#define RAS_METHOD_NEWTON     2

/* Checkpoint / resume of an outer iteration (single-problem handles). The
 * state of an outer solve between outer iterations is its iterate x_k (the
 * caller's y, p) and:
 *   method  RAS_METHOD_* of the solve;
 *   k       outer iterations done;
 *   eps     eps_k of the continuation (Newton_RAS / Newton; eps_min for
 *           RASPEN once k > 0, eps0 at k = 0);
 *   res0    ||F(x^0)|| of the original start, and stop = max(tol, tol*res0),
 *           which fix the stop test.
 * ras_get_state: the state at the end of the last ras_raspen_solve /
 * ras_newton_ras_solve / ras_newton_solve call on h (also when it stopped at
 * kmax with RAS_ENOCONV); RAS_ESTATE if there was none.
 * ras_set_state: the next solve call of the same method on h resumes from
 * the state (one-shot), with y, p = x_k as its initial guess: it continues
 * the outer count, keeps the stop test, and applies eps-continuation only
 * where the uninterrupted solve would. Every reduction has a fixed order, so
 * the resumed solve reproduces the uninterrupted one bit for bit. RAS_EINVAL
 * for an invalid state; a solve of another method returns RAS_ESTATE.
 * The paper has no checkpointing; this is the continuation state of Alg. 1
 * and Alg. 2 made explicit. */
typedef struct {
    int method;
    int k;
    double eps;
    double res0;
    double stop;
} ras_state;
int ras_get_state(const ras_problem* h, ras_state* state);
int ras_set_state(ras_problem* h, const ras_state* state);
/* End-to-end call on HOST buffers: copies y_d_host (n*n, NULL keeps the
 * current y_d) and the initial guess y_host, p_host to the device, solves with
 * `method`, and copies the solution back into y_host, p_host. */
int ras_solve_host(ras_problem* h, int method, const double* y_d_host,
                   double* y_host, double* p_host, ras_stats* stats);

/* Local Newton step counts of the last ras_apply, one per subdomain (index
 * i = by*sx + bx), into its_host[0..count). Returns the number written. */
int ras_local_iterations(const ras_problem* h, int* its_host, int count);

/* Number of subdomains; device bytes held by the handle. */
int ras_subdomain_count(const ras_problem* h);
size_t ras_device_bytes(const ras_problem* h);

/* Text of the last error on this handle (never NULL). */
const char* ras_last_error(const ras_problem* h);

/* Release every device buffer of the handle. NULL is a no-op. */
void ras_destroy(ras_problem* h);

/* Kernel launches issued by this library since load (all handles). */
long long ras_launch_count(void);

/* Live kernel timing (diagnostics; not part of the paper's method).
 * ras_profile(h, 1) clears the counters and records a CUDA event pair on the
 * handle's stream around every kernel launch until ras_profile(h, 0).
 * ras_profile_read returns, for one kernel kind, the summed device time (ms),
 * the number of launches and the summed algorithmic work of those launches:
 *   RAS_K_FACTOR     flops, 16 wx^3 wy per factorised subdomain (the
 *                    no-fill band-LU count 2 N_loc kl ku with kl = ku = 2 wx)
 *   RAS_K_DIRECTION  bytes of factor blocks read (2 passes per local solve)
 *   RAS_K_JVP, RAS_K_PRECOND  bytes of factor blocks read (2 passes)
 *   RAS_K_RESIDUAL   bytes (y, p, y_d, f read once, F written once)
 *   others           0
 * Returns RAS_EINVAL for an unknown kind. */
#define RAS_K_INIT       0
#define RAS_K_FACTOR     1
#define RAS_K_DIRECTION  2
#define RAS_K_LINESEARCH 3
#define RAS_K_JVP        4
#define RAS_K_PRECOND    5
#define RAS_K_RESIDUAL   6
#define RAS_K_KRYLOV     7
#define RAS_K_OTHER      8
#define RAS_K_COUNT      9
int ras_profile(ras_problem* h, int enable);
int ras_profile_read(ras_problem* h, int kind, double* ms, long long* launches, double* work);

/* The manufactured solution of the paper's model problem (Sec. 4): for the
 * adjoint pbar (device, n*n), the state ybar solves the state equation
 * F_y(ybar, pbar, eps) = A y + phi(y) - f + (1/nu)(pbar + mu P_eps(-pbar/mu))
 * = 0 (damped Newton from y = 0, each step by conjugate gradients on the
 * symmetric positive definite A + diag(phi'(y)); phi must be increasing), and
 * y_d = -A pbar - phi'(ybar) pbar + ybar, so that (ybar, pbar) solves the
 * optimality system at eps. The handle's y_d is replaced by it (its phi, nu,
 * mu, kappa and f are used); ybar and y_d are also written to y_out and
 * yd_out (device, n*n, either may be NULL). The paper's run: phi =
 * RAS_PHI_KAPPA, kappa 0.1, nu 1e-6, mu 1, f = 0, pbar = 1.3 mu sin(10 pi
 * x1) sin(10 pi x2), eps = 1e-15. Newton stops at ||F_y|| <= 1e-14 of its
 * value at y = 0, or when no step lowers it any more below 1e-9 of it
 * (rounding level); conjugate gradients run to 1e-10 relative residual.
 * Single-problem handles only; RAS_EINVAL for eps <= 0, RAS_ENOCONV if
 * Newton stalls above that level or takes more than 100 steps,
 * RAS_ENONFINITE on a non-finite residual. */
int ras_manufacture(ras_problem* h, const double* pbar, double eps, double* y_out, double* yd_out);

/* CUDA-graph execution (not part of the paper's method; default on).
 * Every Arnoldi step (the operator, the CGS2 products, the Givens update of
 * the Hessenberg column and the stop test) and every local Newton sweep step
 * runs on the device; with graphs on, a GMRES restart cycle is one graph
 * launch (one IF node per step, skipped once every problem has stopped), and
 * so is a RASPEN-function evaluation (Alg. 3: init, a WHILE node over the
 * sweep steps of Alg. 1 in all subdomains, with the factor kernel of each
 * register-tile class chosen on the device from the active count, then the
 * factors at the local solutions and the prolongation). The host reads a
 * cycle or an evaluation once, instead of once per step. Each graph is
 * captured on first use and again after the handle's buffers, layout,
 * options or tuning change. Both modes run the same kernels in the same order and give
 * identical results. While ras_profile is on, cycles run step by step (the
 * per-kernel events cannot sit inside a graph's conditional bodies).
 * RAS_EINVAL on a NULL handle. */
int ras_use_graphs(ras_problem* h, int enable);

/* Launch-shape tuning (not part of the paper's method: how the kernels are
 * shaped on this device, never what they compute beyond rounding order).
 * ras_tuning holds the three launch shapes a handle uses:
 *   factor_wide_max[c]  register-tile class c (padded block size
 *                       mp = 32 (c + 1): 32, 64, 96, 128, 160): the FP32
 *                       factorisation of the class runs one 1024-thread CTA
 *                       per subdomain when at most this many of its
 *                       subdomains factorise in a sweep, else one 256-thread
 *                       CTA per subdomain. -1 (default): the SM count (the
 *                       1024-thread kernel when the sweep fits one wave).
 *                       The two kernels sweep pivot panels of mp/32 and
 *                       mp/16 columns, so their factors agree to FP32
 *                       rounding, not bit for bit.
 *   solve_ctas_per_sm   CTAs per SM of the persistent local-solve kernels
 *                       (direction, Jacobian action, linear RAS); 0
 *                       (default): as many as fit. Results are identical
 *                       (one CTA computes each subdomain whatever the grid).
 *   vec_blocks          CTAs of the segmented vector kernels (GMRES dot
 *                       products, AXPYs), 1..RAS_VEC_BLOCKS_MAX (default
 *                       RAS_VEC_BLOCKS_MAX). This fixes the summation order
 *                       of every inner product, so results can differ in
 *                       the last bits between two settings; one setting
 *                       always gives the same result.
 * ras_autotune times the candidates with CUDA events on the handle's stream,
 * on the handle's own subdomains (all problems of a batch), and installs the
 * fastest (a candidate replaces the default only when at least 2% faster):
 *   factor   per class with subdomains, both kernels at the class's counts
 *            1, 8, 38, 76, 152, 304 (those below its subdomain count) and
 *            its subdomain count, factorising the Jacobians at x = 0,
 *            eps = eps0. At each count the default rule's kernel is kept
 *            unless the other is 2% faster; if that changes the kernel at
 *            any count, factor_wide_max[c] becomes the largest count up to
 *            which the 1024-thread kernel is kept at every timed count (0
 *            if not even at 1), else it stays -1. FP64 handles keep -1 (one
 *            FP64 kernel).
 *   solve    every CTAs-per-SM value up to the number that fits, timing one
 *            linear RAS application (ras_precondition's local solves) with
 *            every subdomain factorised.
 *   vectors  vec_blocks in {152, 304, 456, 608} (multiples of 152, at most
 *            RAS_VEC_BLOCKS_MAX), timing one CGS step of a 16-vector basis
 *            (segmented dot products, reduction, AXPY).
 * It overwrites the handle's internal iterate and local factorisations (a
 * following ras_jvp returns RAS_ESTATE until the next ras_apply); solve
 * results, the caller's buffers and the checkpoint state are untouched.
 * Call it between solves. Takes milliseconds to about a second. `chosen`
 * (may be NULL) receives the installed tuning, `report` (may be NULL) the
 * timings: per launch, in ms; entries after the last timed one are 0.
 * ras_get_tuning / ras_set_tuning read and install a tuning (for example one
 * saved from an earlier ras_autotune of the same shapes); RAS_EINVAL for
 * factor_wide_max[c] < -1, solve_ctas_per_sm < 0 or > 64, or vec_blocks
 * outside 1..RAS_VEC_BLOCKS_MAX. */
#define RAS_NTILE          5
#define RAS_TUNE_MAX       8
#define RAS_VEC_BLOCKS_MAX 608
typedef struct {
    int factor_wide_max[RAS_NTILE];
    int solve_ctas_per_sm;
    int vec_blocks;
} ras_tuning;
typedef struct {
    int factor_count[RAS_NTILE][RAS_TUNE_MAX];      /* subdomains factorised   */
    double factor_ms[RAS_NTILE][RAS_TUNE_MAX][2];   /* [256, 1024 threads]     */
    int solve_ctas_per_sm[RAS_TUNE_MAX];
    double solve_ms[RAS_TUNE_MAX];
    int vec_blocks[RAS_TUNE_MAX];
    double vec_ms[RAS_TUNE_MAX];
} ras_tune_report;
int ras_autotune(ras_problem* h, ras_tuning* chosen, ras_tune_report* report);
int ras_get_tuning(const ras_problem* h, ras_tuning* t);
int ras_set_tuning(ras_problem* h, const ras_tuning* t);

/* Residual without a handle and without any device allocation.
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc or cudaFree, e.g. code running while another allocator (a
 * framework's caching allocator or a pre-reserved pool) owns the device
 * memory, or a latency-bound loop where an allocation's implicit device
 * synchronisation is not acceptable; ras_create allocates, so those callers
 * cannot use ras_residual.
 * Computes F(x, eps) of Sec. 3.3 at x = (y, p) with the same expression as
 * ras_residual (results agree to rounding; the norm's summation order
 * differs): writes Fy, Fp (device n*n, either may be NULL) and, if
 * norm_dev != NULL, ||(Fy, Fp)||_2 to norm_dev[0] (device). y, p, y_d: device
 * n*n; f device n*n or NULL (= 0); phi, nu, mu, kappa as in ras_create /
 * ras_opts; eps > 0.
 * The work is only enqueued on `stream` (cudaStream_t, NULL = legacy default
 * stream); results are ready when the stream reaches it.
 * Scratch: the norm's partial sums live in one fixed array inside the library
 * (1 double per grid row, RAS_STATIC_MAX_N rows, 64 KiB), which every GPU
 * that loads the library holds until the process exits. Each call looks up
 * that array's device address (cudaGetSymbolAddress, no allocation) in the
 * current context, so it stays valid after cudaDeviceReset; the first call on
 * a device may load the library's device code, so make it before any stream
 * capture. Every call writes all the partials it later reads, so nothing has
 * to start at zero; the array keeps the last call's values. All calls share
 * the array: calls whose GPU work overlaps (other streams, other threads)
 * race and give wrong norms.
 * Returns RAS_EINVAL for n < 2, n > RAS_STATIC_MAX_N, a bad phi, nu, mu or
 * eps, or a NULL y, p or y_d; RAS_ECUDA if the lookup or a launch fails. No
 * allocation of any kind is made. */
#define RAS_STATIC_MAX_N 8192
int ras_residual_static(int n, int phi, double nu, double mu, double kappa, double eps,
                        const double* y, const double* p, const double* y_d, const double* f,
                        double* Fy, double* Fp, double* norm_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RAS_H */
