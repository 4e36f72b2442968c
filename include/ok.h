/*
 * ok.h -- C ABI of the GB300 Ohta--Kawasaki Newton-step solver.
 *
 * What it computes (Farrell & Pearson, "A preconditioner for the
 * Ohta--Kawasaki equation", arXiv:1603.04570):
 *   - the P1 finite-element, theta-method discretisation of the Ohta--Kawasaki
 *     equations in (u, w) form with homogeneous Neumann conditions
 *     (Sec. 1, eqns oka, okb, okbcs; Sec. 2 first paragraph);
 *   - at each Newton step the linear system J [du; dw] = f of eqn newton,
 *         J = [ (1 + dt theta sigma) M    dt theta K ]
 *             [ -eps^2 K - M_E            M          ],
 *     solved by right-preconditioned restarted flexible GMRES;
 *   - the preconditioner of eqn prec with A~^{-1} (Chebyshev semi-iteration on
 *     the mass matrix, Sec. 3) and the matching-strategy Schur approximation
 *     S~^{-1} = S_hat^{-1} M S_hat^{-1}, S_hat = M + eps sqrt(c) K,
 *     c = dt theta / (1 + dt theta sigma) (eqns schur, outer_approx, schurinv);
 *     S_hat^{-1} is approximated by geometric multigrid V-cycles (the paper
 *     uses algebraic multigrid, Sec. 2 and Sec. 4).
 *
 * Grids: the unit square cut into n x n squares, each split along its
 * (0,0)-(1,1) diagonal into two P1 triangles (dim = 2), or the unit cube cut
 * into n^3 cubes of 6 Kuhn tetrahedra around the (0,0,0)-(1,1,1) diagonal
 * (dim = 3).  N_v = (n+1)^dim vertices.
 *
 * Array conventions (every function):
 *   - nodal arrays are double, compact lexicographic order, x fastest:
 *     vertex (i,j[,k]) sits at i + (n+1) j [+ (n+1)^2 k];  a field has N_v
 *     entries, a block vector [first field; second field] has 2 N_v;
 *   - every array pointer may be HOST memory (pageable or pinned) or DEVICE
 *     memory of the current CUDA device; the library asks the CUDA runtime
 *     which it is.  Host arrays are staged through the grid's device
 *     buffers, and the call returns only after results are back on the host.
 *     Device arrays are used in place; work is enqueued on `stream`, and
 *     functions that need a scalar on the host (norms, convergence tests)
 *     synchronise that stream.
 *   - the caller owns every array; the library owns the ok_grid handle and all
 *     device workspace it allocated in ok_grid_create.
 *   - `stream` is a cudaStream_t (0 = the legacy default stream).
 *
 * Errors: every function returns an OK_* status.  On failure
 * ok_last_error() returns a message for the calling thread.  A non-finite
 * input is reported as OK_ERR_NONFINITE before work that depends on it runs.
 * No function traps or faults the GPU on purpose.
 *
 * One handle must not be used from two threads at once.
 */
#ifndef OK_GB300_H
#define OK_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ok_stream;   /* a cudaStream_t */

enum ok_status {
  OK_SUCCESS = 0,
  OK_ERR_INVALID_ARG = 1,     /* a size, option or pointer is invalid        */
  OK_ERR_NOMEM = 2,           /* device or pinned host allocation failed     */
  OK_ERR_CUDA = 3,            /* a CUDA runtime call failed                  */
  OK_ERR_NOT_CONVERGED = 4,   /* Newton or GMRES hit its iteration cap       */
  OK_ERR_NONFINITE = 5,       /* NaN/Inf in an input or during the solve     */
  OK_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up          */
  OK_ERR_INTERNAL = 7         /* an unexpected host-side failure (message in
                                 ok_last_error); no exception leaves the ABI  */
};

enum ok_precision {
  OK_FP64 = 0,       /* every step in float64                                      */
  OK_MIXED = 1,      /* preconditioner in float32 under float64 FGMRES, J, residual */
  OK_MIXED_HALF = 2  /* as OK_MIXED, the preconditioned vectors Z of the flexible
                        basis stored in float16 (half the Z memory); J z_j and the
                        update use the stored values, so FGMRES stays consistent */
};

/* Physical and time-stepping parameters of eqns oka/okb and the theta-method. */
typedef struct ok_params {
  double eps;     /* interfacial thickness epsilon                        */
  double sigma;   /* nonlocal energy coefficient sigma                    */
  double m;       /* conserved mean of u                                  */
  double theta;   /* implicitness of the theta-method, in (0, 1]          */
  double dt;      /* timestep                                             */
} ok_params;

/* Solver options.  ok_default_opts() fills the defaults given in brackets. */
typedef struct ok_opts {
  int restart;        /* FGMRES restart length m [30]                           */
  int max_gmres;      /* FGMRES iteration cap per linear solve [500]            */
  int max_newton;     /* Newton steps per timestep [25]                         */
  int newton_extra;   /* extra Newton steps after the stop test passes [0]      */
  int q_A;            /* Chebyshev steps for A~^{-1} [10] (Sec. 4: ten)         */
  int n_V;            /* V-cycles per S_hat^{-1} [5] (Sec. 4: five)             */
  int k_R;            /* 1: S~^{-1}; 2: two Richardson steps on S [1]           */
  int smooth_pre;     /* Chebyshev--Jacobi pre-smoothing steps per level [2]    */
  int smooth_post;    /* post-smoothing steps per level [2]                     */
  int precision;      /* OK_FP64, OK_MIXED or OK_MIXED_HALF [OK_FP64]           */
  int coarse_max;     /* halve the grid while n is even and > coarse_max [4]    */
  int use_graphs;     /* capture each Arnoldi step in a CUDA graph [1]          */
  int fuse_coarse;    /* coarse multigrid levels in one launch: 0 off; 1 the
                         suffix of levels that fits one block's shared memory
                         in one block; 2 with the 2D tile kernels the levels
                         of <= 129 vertices per side and the coarsest solve as
                         one thread-block cluster (when the device supports
                         it), otherwise as 1 [1]                                 */
  int tile_fine;      /* 2D: register-strip tile kernels on the fine levels:
                         0 off, 1 window width per level chosen by the
                         autotuner (ok_grid_tuning), 2 / 3 force 32 / 64
                         columns; 3D: any nonzero value runs the multigrid's
                         stencil steps by z-marching blocks, with 1 their block
                         shape per level from the autotuner, 4 + k shape k on
                         every level, 2 and 3 shape 0 (0: one thread per
                         vertex; all give the same bits) [1]                    */
  int use_pdl;        /* programmatic dependent launch between kernels [1]      */
  int reorth;         /* Gram--Schmidt: 0 second pass only when the first one
                         cancels more than half of ||w||^2, 1 always two
                         passes (classical Gram--Schmidt with
                         reorthogonalisation, CGS2), 2 one classical pass [1]   */
  double gmres_rtol;  /* stop when ||f - J x|| <= gmres_rtol ||f|| [1e-10]      */
  double newton_atol; /* Newton stops when ||F||_2 <= max(atol, rtol ||F_0||)   */
  double newton_rtol; /*   [atol 1e-10, rtol 0]                                 */
  double smooth_lo_frac; /* smoother interval [frac*lmax, lmax] [0.25]          */
} ok_opts;

/* Statistics of one Newton step / one timestep. */
typedef struct ok_step_info {
  int newton_its;       /* Newton steps taken                                   */
  int gmres_its;        /* FGMRES iterations, summed over the Newton steps      */
  int converged;        /* 1 when the stop test passed                          */
  int last_gmres_its;   /* iterations of the last linear solve                  */
  double rel_resid;     /* ||f - J x|| / ||f|| of the last linear solve         */
  double newton_resid;  /* ||F||_2 at exit                                      */
  double newton_resid0; /* ||F||_2 at entry                                     */
  double solve_ms;      /* wall time of the linear solves (host clock)          */
} ok_step_info;

typedef struct ok_grid ok_grid;

/* Fill `o` with the defaults listed in ok_opts. */
void ok_default_opts(ok_opts* o);

/* Create a solver for one grid and parameter set (dim 2 or 3, n cells per
 * side, 2 <= n, (n+1)^dim < 2^31).  Builds the multigrid hierarchy of
 * S_hat = M + eps sqrt(c) K, which depends only on the grid, eps and c and
 * is therefore reused across Newton steps and timesteps (Sec. 2, after eqn
 * schurapprox), and allocates the Krylov workspace on the current device.
 * `o` may be NULL (defaults).  *out receives the handle. */
int ok_grid_create(int dim, int n, const ok_params* p, const ok_opts* o, ok_grid** out);

/* Free a handle and its device memory.  NULL is accepted. */
int ok_grid_destroy(ok_grid* g);

/* Sizes of a handle: vertices, multigrid levels, device bytes held. */
int ok_grid_query(const ok_grid* g, long long* n_vertices, int* n_levels, long long* device_bytes);

/* w0 from eqn okb for a given u0 (Sec. 4, "computed from u0 via okb"):
 * the L2 projection  M w0 = eps^2 K u0 + N(u0),  N(u)_i = int (u^3 - u) phi_i,
 * solved with Chebyshev on M to round-off.  u0, w0: N_v each. */
int ok_init_w(ok_grid* g, const double* u0, double* w0, ok_stream stream);

/* f = -F(u_k, w_k) for the theta-scheme residual with previous state
 * (u_n, w_n) (eqns oka/okb integrated against each P1 basis function):
 *   F1 = M (u - u_n) + dt theta [K w + sigma M (u - m)]
 *                    + dt (1 - theta) [K w_n + sigma M (u_n - m)],
 *   F2 = M w - eps^2 K u - N(u).
 * f has 2 N_v entries; *norm_out (host) receives ||F||_2.  Synchronises. */
int ok_assemble_rhs(ok_grid* g, const double* u_n, const double* w_n,
                    const double* u_k, const double* w_k, double* f,
                    double* norm_out, ok_stream stream);

/* y = J(u_k) z with J of eqn newton; z, y: 2 N_v.  M_E uses u_k. */
int ok_apply_jacobian(ok_grid* g, const double* u_k, const double* z, double* y,
                      ok_stream stream);

/* z = P^{-1} v, the block lower-triangular preconditioner of eqn prec with
 * A~^{-1} and S~^{-1} as configured (precision, q_A, n_V, k_R); v, z: 2 N_v. */
int ok_apply_preconditioner(ok_grid* g, const double* u_k, const double* v, double* z,
                            ok_stream stream);

/* Solve J(u_k) x = f by right-preconditioned restarted FGMRES from x = 0 to
 * the relative tolerance opts.gmres_rtol (eqn newton).  info may be NULL. */
int ok_solve_linear(ok_grid* g, const double* u_k, const double* f, double* x,
                    ok_step_info* info, ok_stream stream);

/* One Newton step for the timestep from (u_n, w_n) (Sec. 2, first paragraph:
 * a Newton iteration per timestep, each solving eqn newton): f = -F(u_k, w_k)
 * as in ok_assemble_rhs, J(u_k) d = f solved as ok_solve_linear does, then
 * (u_k, w_k) += d.  u_k, w_k are in-out; u_n, w_n are read only.  info (may
 * be NULL) receives the FGMRES iterations, the linear solve's relative
 * residual and ||F||_2 before and after the step; converged = 1 when the
 * latter meets the Newton stop test of ok_timestep. */
int ok_newton_step(ok_grid* g, const double* u_n, const double* w_n,
                   double* u_k, double* w_k, ok_step_info* info, ok_stream stream);

/* One theta-method timestep of eqns oka/okb (Sec. 2, first paragraph; Sec. 4
 * runs these with theta = 1/2): Newton from (u, w) at t_n, each step as
 * ok_newton_step, until ||F||_2 <= max(newton_atol, newton_rtol ||F_0||_2),
 * then newton_extra more steps; (u, w) are overwritten with t_{n+1}.
 * Returns OK_ERR_NOT_CONVERGED (state left at the last iterate) when the
 * Newton cap is hit. */
int ok_timestep(ok_grid* g, double* u, double* w, ok_step_info* info, ok_stream stream);

/* A batch of independent simulations.  Each request names its grid handle,
 * its state arrays and its number of timesteps; per-request status and
 * statistics are written back into the request. */
typedef struct ok_request {
  ok_grid* grid;       /* in                                              */
  double* u;           /* in-out, N_v of that grid                         */
  double* w;           /* in-out                                           */
  int steps;           /* in: timesteps to take                            */
  int status;          /* out: OK_* of the first failing step, else 0      */
  int newton_its;      /* out: summed over the steps                       */
  int gmres_its;       /* out                                              */
  double seconds;      /* out: wall time from batch start to completion    */
} ok_request;

typedef struct ok_batch_info {
  int completed;       /* requests that finished with OK_SUCCESS          */
  int failed;
  double seconds;      /* wall time of the whole batch                     */
} ok_batch_info;

/* Run every request to completion (no counterpart in the paper; the batching
 * is this library's serving form).  Requests whose handles have the same grid
 * (dim, n), options and multigrid structure form cohorts of up to 8 on
 * distinct handles, in request order; a cohort advances timestep by timestep
 * in lockstep, and every kernel of an Arnoldi step (the preconditioner's
 * stencil and multigrid kernels, J z, the classical Gram--Schmidt passes) is
 * ONE launch over all of its members still iterating.  Each member keeps its
 * own Newton and FGMRES decisions, so its results are bitwise those of
 * ok_timestep alone.  Cohorts need reorth = 1 (CGS2) and fuse_coarse != 2;
 * other requests, and cohorts of one, run through ok_timestep.  Cohorts run
 * one after another, ordered after `stream` and the members' earlier work;
 * `stream` waits for the whole batch.  A failing request does not stop the
 * others (its state is left as ok_timestep would leave it).  Returns the
 * status of the first failed request. */
int ok_solve_batch(ok_request* reqs, int count, ok_batch_info* out, ok_stream stream);

/* Serving (no counterpart in the paper): whole simulations admitted
 * continuously.  A request is admitted when it has arrived (`arrival`,
 * seconds after the call starts), fewer than `max_inflight` are in flight and
 * its estimated device footprint (Krylov basis dominant) fits in
 * `mem_budget` bytes beside those in flight.  Arrived requests are
 * considered oldest first; a younger one that fits may pass an older one
 * that waits for memory, until the oldest waiting request has waited one
 * second (from then on it alone may enter, so it is not starved).  An
 * admitted request's handle (ok_grid_create) and w0 (ok_init_w when
 * init_w != 0) are set up on a thread of its own; it then joins the group of
 * requests with its (dim, n, options), whose host thread and non-blocking
 * stream advance the group's members a timestep at a time as one cohort
 * (the shared launches of ok_solve_batch, up to 8 members; a member joins at
 * the next timestep boundary and leaves after its last step, when its handle
 * is destroyed and its slot and bytes are released).  Groups run
 * concurrently.  During the call the device blocks of destroyed handles are
 * reused by later handles of the same sizes instead of being freed and
 * allocated again.  A request's arithmetic does not depend on what else runs:
 * its results are bitwise those it gets alone.  Returns the status of the
 * first failed request (all requests run regardless); OK_ERR_NOMEM marks a
 * request whose footprint exceeds the whole budget. */
typedef struct ok_serve_request {
  int dim, n;               /* in: grid                                              */
  ok_params params;         /* in                                                    */
  const ok_opts* opts;      /* in: NULL for the defaults                             */
  double* u;                /* in-out: N_v, host or device                           */
  double* w;                /* in-out: N_v; computed from u first when init_w != 0   */
  int init_w;               /* in                                                    */
  int steps;                /* in: timesteps                                         */
  double arrival;           /* in: seconds after the call starts                     */
  int status;               /* out: OK_*                                             */
  int newton_its, gmres_its;/* out: summed over the steps                            */
  double t_admit, t_done;   /* out: seconds after the call starts                    */
  long long device_bytes;   /* out: footprint charged at admission (estimate)        */
  char message[96];         /* out: ok_last_error() of a failed request, else ""     */
} ok_serve_request;

typedef struct ok_serve_info {
  int completed, failed;
  int peak_inflight;        /* most requests in flight at once                       */
  long long peak_bytes;     /* most estimated bytes in flight at once                */
  double seconds;           /* wall time of the call                                 */
  int peak_cohort;          /* most requests advanced by one cohort timestep         */
  int cohort_steps;         /* cohort timesteps with two or more members             */
} ok_serve_info;

int ok_serve(ok_serve_request* reqs, int count, int max_inflight, long long mem_budget, ok_serve_info* info);

/* Sampled kernel timing (no counterpart in the paper: measurement support).
 * ok_profile(g, 1) clears the counters and, from the next Arnoldi step on,
 * records one CUDA-event pair per kernel class per step on the handle's
 * stream: "precond" (one whole preconditioner application), "apply_j" (the
 * Jacobian kernel), "cgs2" (the four orthogonalisation kernels),
 * "mg_smooth_l0" (the first finest-level Chebyshev smoothing kernel),
 * "cheb_mass_step" (the first Chebyshev step on M); with the 2D tile kernels
 * "tile_mass_cstep" (A~^{-1} r1 and the C-step), "mg_tile_pre_l<k>" and
 * "mg_tile_post_l<k>" (the first pre-/post-smoothing tile kernel of level
 * k = 0..4) and "mg_coarse" (the first coarsest-level solve).  ok_profile(g, 0) stops.
 * Toggling re-captures the handle's CUDA graphs.  ok_profile_read copies up
 * to `max` records into `out` (host) and the number written into *count. */
typedef struct ok_kernel_stat {
  char name[32];
  long long samples;   /* timed launches                  */
  double total_ms;     /* summed duration of those launches */
} ok_kernel_stat;
int ok_profile(ok_grid* g, int enable);
int ok_profile_read(const ok_grid* g, ok_kernel_stat* out, int max, int* count);

/* Spectral diagnostics of the preconditioned Jacobian (Sec. 3, Lemmas 1-2).
 * With A inverted exactly the right-preconditioned Jacobian J P^{-1} has the
 * eigenvalue 1 and the eigenvalues of S~^{-1} S, which Lemma 1 makes real and
 * Lemma 2 (K perturbed to be SPD) places in
 *   [1/2 + sqrt(c) l_- / (2 eps), 1 + sqrt(c) l_+ / (2 eps)),
 * l_- = min(lambda_min(M^{-1} M_E), 0), l_+ = max(lambda_max(M^{-1} M_E), 0),
 * c = dt theta / (1 + dt theta sigma).  Each FGMRES restart cycle is an
 * Arnoldi process on J P^{-1}: J Z_k = V_{k+1} Hbar_k, Z_k = P^{-1} V_k
 * (exactly so while the preconditioner is a fixed linear map, as it is here:
 * fixed Chebyshev steps and V-cycles).  These calls read the Arnoldi matrix
 * of the LAST restart cycle run on `g` (by ok_solve_linear, ok_newton_step,
 * ok_timestep); a call whose right-hand side was zero runs no cycle and
 * leaves the previous one.  A handle that has run no cycle reports k = 0.
 *
 * ok_arnoldi_hessenberg: writes Hbar_k ((k+1) x k, column-major, leading
 *   dimension ldh >= max_k + 1) into the HOST array H, k = min(steps of the
 *   cycle, max_k) into *k; the first k columns of a longer cycle are the
 *   Arnoldi matrix of its first k steps.  The device holds Hbar reduced by
 *   its Givens rotations; it is restored on the host.  Synchronises with
 *   `stream` (the stream of the solve).
 * ok_ritz_values: the eigenvalues (Ritz values) of the square part H_k,
 *   k <= max, into the HOST arrays re[0..k) and im[0..k) (complex pairs
 *   adjacent), k into *count.  OK_ERR_NOT_CONVERGED if the QR iteration does
 *   not converge, OK_ERR_NONFINITE for a non-finite Arnoldi matrix.
 * ok_givens_unrotate: host only, no GPU needed.  H (column-major, ldh >=
 *   k + 1) holds in columns 0..k-1 the triangular factor R left by applying,
 *   to column j of an upper Hessenberg matrix, the rotations i = 0..j that
 *   map rows (i, i+1) as (a, b) -> (cs[i] a + sn[i] b, -sn[i] a + cs[i] b);
 *   overwrites it with that Hessenberg matrix (rows j+2..k of column j zeroed).
 * ok_hessenberg_eigenvalues: host only, no GPU needed.  Eigenvalues of the
 *   k x k upper Hessenberg matrix H (0 <= k <= 4096; column-major, ldh >= k; entries below
 *   the first subdiagonal are ignored) by the implicit double-shift QR
 *   iteration (Francis 1961; Golub and Van Loan, Sec. 7.5), into re/im
 *   (length k, in deflation order, complex pairs adjacent).
 * All four return OK_ERR_INVALID_ARG for NULL arrays or bad sizes. */
int ok_arnoldi_hessenberg(ok_grid* g, double* H, int ldh, int max_k, int* k, ok_stream stream);
int ok_ritz_values(ok_grid* g, double* re, double* im, int max, int* count, ok_stream stream);
int ok_givens_unrotate(int k, double* H, int ldh, const double* cs, const double* sn);
int ok_hessenberg_eigenvalues(int k, const double* H, int ldh, double* re, double* im);

/* y = J(u_k) z like ok_apply_jacobian, for callers that cannot allocate
 * device memory: applications that own all GPU memory through their own
 * allocator or run under a fixed memory budget, and latency-critical loops
 * that cannot afford cudaMalloc's device-wide synchronisation.  The paper has
 * no counterpart; this is an interface convenience of the library.
 *
 * No handle is needed and nothing is allocated: the per-Newton-step
 * coefficients of C = -eps^2 K - M_E(u_k) go to a 16 MiB static device array
 * that every GPU loading the library holds until the process exits.
 *   - dim 2 or 3, n cells per side, p as in ok_grid_create;
 *   - u_k (N_v), z and y (2 N_v) must be DEVICE arrays (no host staging);
 *   - grids needing more than 16 MiB of coefficients are rejected with
 *     OK_ERR_INVALID_ARG (2D: n <= 590; 3D: n <= 54);
 *   - work is enqueued on `stream`; the call does not synchronise;
 *   - every call shares the one array and leaves its coefficients there:
 *     calls whose work overlaps on the GPU race, so serialise them;
 *   - the first call on a device looks up the array's address and uploads
 *     the stencil tables (synchronously): make it before any stream capture.
 * Errors are reported through ok_last_error(). */
int ok_apply_jacobian_noalloc(int dim, int n, const ok_params* p, const double* u_k, const double* z,
                              double* y, ok_stream stream);

/* Choices of the autotuner (no counterpart in the paper).  With
 * tile_fine = 1, ok_grid_create times the compiled kernel shapes of each
 * multigrid level once per (device, dim, n, precision) in the process and
 * keeps the fastest: in 2D the register-strip window shape of every tiled
 * level (float: 0: 32 x 32 vertices in 2-row strips per thread, 1: 64 x 32 in
 * 8-row strips, 2: 64 x 32 in 4-row, 3: 64 x 64 in 4-row, 4: 128 x 32 in
 * 4-row; float64: 0: 32 x 16 by 2, 1: 64 x 32 by 2, 2: 64 x 32 by 4,
 * 3: 32 x 32 by 4, 4: 64 x 16 by 2), in 3D the block shape of the z-marching
 * stencil kernels (0: 32 x 8 columns by 16 planes, 1: 32 x 4 by 32, 2: 64 x 4
 * by 16, 3: 32 x 8 by 32) or 4: one thread per vertex instead.  All choices
 * give the same bits.  Writes up to
 * `max` (level cells per side, choice) pairs, finest level first, into the
 * HOST arrays level_n and choice, their number into *count (0 when nothing
 * was tuned). */
int ok_grid_tuning(const ok_grid* g, int* level_n, int* choice, int max, int* count);

/* The autotuner's choices made (or loaded) so far in this process, kept per
 * (dim, level cells per side, value size): ok_tuning_save writes them to the
 * text file `path` (one "dim n bytes choice" line each); ok_tuning_load reads
 * such a file into the process's choices for the current device, so that
 * later ok_grid_create calls of those shapes use them without timing (a
 * process under a profiler, whose kernel timings differ, then runs the
 * kernels a plain run chose).  Host only; OK_ERR_INVALID_ARG for a NULL or
 * unreadable path or malformed lines. */
int ok_tuning_save(const char* path);
int ok_tuning_load(const char* path);

/* The Ohta--Kawasaki free energy (Sec. 1, the functional E[u] whose H^{-1}
 * gradient flow eqns oka/okb are) of the P1 function with nodal values u
 * (N_v, host or device):
 *   terms[0] = eps^2/2 u^T K u                       (interfacial term),
 *   terms[1] = 1/4 int (1 - u_h^2)^2 dx              (double well, exact quadrature),
 *   terms[2] = sigma/2 (f, phi)_{L2}                 (nonlocal term),
 * with f = u minus its mean and phi the solution of the Neumann problem
 * K phi = M f (the inverse Neumann Laplacian of Sec. 1), solved by conjugate
 * gradients preconditioned with two multigrid V-cycles for M + K (float64)
 * to a relative residual of 1e-12; *E = terms[0] + terms[1] + terms[2].
 * terms (3 doubles) and E are HOST pointers; either may be NULL, not both.
 * The first call on a handle builds that multigrid (device memory about the
 * size of the float64 preconditioner's hierarchy) and keeps it.  Synchronises
 * `stream`.  OK_ERR_NONFINITE for a non-finite u. */
int ok_energy(ok_grid* g, const double* u, double* terms, double* E, ok_stream stream);

/* Number of this library's kernels launched by the process so far (graph
 * replays count every kernel node). */
long long ok_launch_count(void);

/* Message of the last failing call on this thread ("" if none). */
const char* ok_last_error(void);

/* Library version string. */
const char* ok_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OK_GB300_H */
