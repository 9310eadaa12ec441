/*
 * pt.h — C ABI of the GB300 time-parallel inexact-Uzawa solver for parabolic problems.
 *
 * Problem (Neumüller & Smears, "Time-parallel iterative solvers for parabolic
 * evolution equations", §2, eq. 2.1): implicit Euler for u_t - div(a grad u) = f on
 * the unit box (0,1)^dim, homogeneous Dirichlet data, steps tau_n (uniform T/N_t unless
 * pt_options.tau_steps gives them), t_n = tau_1 + ... + tau_n,
 *
 *     (u_n - u_{n-1}) + tau_n A_n u_n = tau_n f_n,  n = 1..N_t,  u_0 = u0,
 *
 * with M = I and the conservative finite-difference operator
 *     (A_n v)_i = sum_d h^-2 [a(x_i - h e_d/2, t_n)(v_i - v_{i-e_d}) + a(x_i + h e_d/2, t_n)(v_i - v_{i+e_d})]
 * or, with pt_options.mass = 1, the P1 finite-element form M (u_n - u_{n-1}) + tau_n A_n u_n =
 * tau_n M f_n (see pt_options.mass).
 * All N_t steps are solved at once: the time-global system B u = F (eq. 2.3-2.4) is
 * rewritten as the symmetric saddle-point system of eq. 2.7 and solved by the inexact
 * Uzawa iteration of §3, eq. 3.1, preconditioned by the DST-in-time Schur-complement
 * preconditioner of §4, eq. 4.4-4.6, with geometric-multigrid V-cycles (or, in 1-D,
 * exact tridiagonal solves) for the spatial blocks.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grids: `n[d]` interior points per axis with h = 1/(n+1); n + 1 must be a power of two
 *   (multigrid coarsening n -> (n-1)/2); all axes equal for dim >= 2.
 * - Arrays exchanged with the caller are packed FP64, layout [N_t][n_z][n_y][n_x], x
 *   fastest, interior points only (n_s = prod n[d] values per step).
 * - `*_on_device` = 1 means the pointer is CUDA device memory of the current device,
 *   0 means host memory.  Inputs are copied; the caller keeps ownership of every
 *   pointer it passes and may free it when the call returns.
 * - Work is ordered on the stream given in pt_options.stream (NULL = legacy default
 *   stream).  Calls that return results to host memory synchronise that stream.
 * - Errors: every call returns a pt_status; PT_OK = 0.  On failure pt_last_error()
 *   returns a thread-local message.  No exception crosses the ABI.  A pt_problem is
 *   not thread-safe; distinct problems may be used from distinct threads.
 */
#ifndef PT_H_
#define PT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PT_OK = 0,
  PT_EINVAL = 1,     /* invalid argument (sizes, pointers, options) */
  PT_ENOMEM = 2,     /* device allocation failed */
  PT_ENOTCONV = 3,   /* max_it reached before tol; outputs are still written */
  PT_EDIVERGED = 4,  /* residual became non-finite or grew past 1e30 */
  PT_ECUDA = 5,      /* a CUDA runtime call failed */
  PT_ETIMEOUT = 6,   /* a bounded wait expired */
  PT_EBUSY = 7       /* resource busy (e.g. server queue full) */
} pt_status;

typedef struct {
  int dim;  /* 1, 2 or 3 */
  int n[3]; /* interior points per axis (entries beyond dim ignored) */
} pt_grid;

typedef enum { PT_TRIG_ONE = 0, PT_TRIG_SIN = 1, PT_TRIG_COS = 2 } pt_trig;

/* Coefficient a(x,t) = a0 + c * prod_d g_d(pi*mx[d]*x_d) * g_t(pi*mt*t), g in {1, sin, cos};
 * must stay positive on the grid (A_n symmetric positive definite, §2). */
typedef struct {
  double a0;
  double c;
  int fx[3];    /* pt_trig per axis */
  double mx[3];
  int ft;       /* pt_trig in time */
  double mt;
} pt_coeff;

enum { PT_PREC_FP64 = 0, PT_PREC_MIXED = 1 };
enum { PT_SOLVER_MG = 0, PT_SOLVER_EXACT_1D = 1 };

typedef struct {
  int precision;         /* PT_PREC_FP64: everything in FP64.  PT_PREC_MIXED: preconditioner
                            (V-cycles, DSTs, block solves) in FP32; residuals, dot products
                            and the updates of u and p in FP64 (iterative refinement). */
  double omega;          /* Uzawa damping (§3, eq. 3.1); <= 0 selects 1.5 / (1 + alpha) with
                            alpha = max((a0+|c|)/a0, a0/(a0-|c|)), the constant of eq. 2.2 for
                            the coefficient range against its time mean (0.5 for |c| = a0/2) */
  int spatial_solver;    /* PT_SOLVER_MG, or PT_SOLVER_EXACT_1D (dim == 1 only) */
  int n_vcycles;         /* V-cycles per H_k solve of the Schur preconditioner (1..4; 0 selects 2:
                            the second cycle brings H~ close to H and roughly halves the Uzawa
                            iterations); the A~_n solves always use one V-cycle */
  double jacobi_weight;  /* weighted-Jacobi smoothing weight; <= 0 selects 2/3, 4/5, 6/7 by dim */
  void* stream;          /* cudaStream_t for all work of this problem; NULL = default stream */
  int check_every;       /* iterations between host polls of the device convergence flag; 0 = auto */
  int autotune;          /* Before the first solve, time the candidate launch configurations
                            (temporal-transform tile width, multigrid coarse-level split) on the
                            problem's own data and keep the fastest; the choice is cached per grid,
                            precision, solvers and power-of-two bucket of N_t in the process and,
                            when the environment variable PT_TUNE_CACHE names a file, in that JSON
                            file.  1: on; 0 or -1: off (the defaults).  Measured on the 512-problem
                            batch workload: 9.79e7 DOF/s tuned (tuning included), 1.01e8 with the
                            tuning cached, 1.02e8 untuned -- the launch choices it has matter less
                            than run-to-run noise there, so it is opt-in. */
  int dst_cols;          /* complex columns per CTA of the temporal transform; 0 = automatic */
  int coarse_elems;      /* multigrid levels with at most this many points per slice run in one
                            CTA per slice; 0 = 1024; else a power of two in [64, 4096] */
  int no_graphs;         /* 1: launch kernels one by one instead of replaying a captured CUDA
                            graph of the iteration (kernel timing via pt_profile_* also does) */
  int h_solver;          /* H_k solves of the Schur preconditioner: 0 = automatic (exact, by spatial
                            sine transforms, when the reference coefficient is constant in space,
                            dim is 2 or 3 and n + 1 <= 4096; else V-cycles), 1 = V-cycles,
                            2 = exact (PT_EINVAL if unavailable) */
  int krylov;            /* 0: the Uzawa iteration of eq. 3.1; m in [1, 64]: flexible GMRES(m)
                            right-preconditioned by one inexact Uzawa step (FP64 only) */
  int mass;              /* M of eq. 2.1.  0: M = I (finite differences).  1: P1 finite elements on
                            the uniform mesh (1-D; 2-D with every grid square cut along its lower-left
                            to upper-right diagonal), the system divided by h^d: M is the P1 mass
                            matrix over h^d (1-D [1/6, 2/3, 1/6]; 2-D 1/2 at the point, 1/12 at the
                            four axis neighbours and the upper-right and lower-left ones), A_n the
                            stiffness matrix over h^d with the coefficient at the edge midpoints (the
                            finite-difference operator above), F_n = tau_n M f_n with f the nodal
                            values (+ M u0 for n = 1), and H_k = mu_k M + tau Abar.  dim <= 2, FP64,
                            krylov = 0; in 2-D the H_k solves are V-cycles (h_solver 2 is refused). */
  const double* tau_steps; /* NULL: N_t uniform steps T/N_t.  Else a host array of the N_t step
                            lengths tau_1..tau_N (§2, eq. 2.1), each finite and > 0, summing to T
                            within 1e-10 T (else PT_EINVAL); copied at create.  t_n = tau_1 + ... +
                            tau_n; B = K + diag(tau_n A_n), F_n = tau_n f_n (+ u0 for n = 1).  The
                            Schur preconditioner keeps the reference pair of eq. 2.2: tau = T/N_t
                            and Abar, the operator of the coefficient's time mean over (0, T); the
                            default omega takes alpha of eq. 2.2 with the step ratios tau_n/tau. */
} pt_options;

typedef struct pt_problem pt_problem; /* opaque, library-owned */

/* Create a problem and upload its data.
 *   grid, N_t >= 1, T > 0, coeff: the PDE and its discretisation (see above).
 *   f  : [N_t][n_s] values f(x_i, t_n), n = 1..N_t (host or device, see f_on_device); NULL means
 *        f = 0 (see also pt_problem_set_rhs_uniform).
 *   u0 : [n_s] initial datum u_I, or NULL for zero.
 *   opts: may be NULL (all defaults).
 * Forms F = [tau_1 f_1 + u0, tau_2 f_2, ..., tau_N f_N] on the device (§2, after eq. 2.4),
 * allocates all device state, and returns the handle in *out.
 * Errors: PT_EINVAL (bad sizes/options/pointers), PT_ENOMEM, PT_ECUDA. */
pt_status pt_problem_create(const pt_grid* grid, int N_t, double T, const pt_coeff* coeff,
                            const double* f, int f_on_device, const double* u0, int u0_on_device,
                            const pt_options* opts, pt_problem** out);

/* Replace the source f (and u0) of an existing problem; same layouts as pt_problem_create. */
pt_status pt_problem_set_rhs(pt_problem* p, const double* f, int f_on_device, const double* u0,
                             int u0_on_device);

/* Replace the source by the synthetic field f(x_i, t_n) = 2 U - 1, U in [0,1) from the top 53 bits
 * of draw q of SplitMix64 (Steele, Lea & Flood 2014) started at `seed`, q = (n-1) n_s + i the
 * packed index of the point; generated on the device (no host copy).  u0 as in
 * pt_problem_set_rhs. */
pt_status pt_problem_set_rhs_uniform(pt_problem* p, unsigned long long seed, const double* u0,
                                     int u0_on_device);

/* Inexact Uzawa (§3, eq. 3.1) from u = p = 0 until ||F - B u_j|| / ||F|| <= tol or max_it updates.
 *   u_out   : [N_t][n_s] solution u_1..u_N (host or device per u_out_on_device), or NULL.
 *   res_hist: host array of max_it + 1 doubles receiving ||F - B u_j||/||F||, j = 0..iters
 *             (res_hist[0] = 1); or NULL.
 *   iters   : host int receiving the number of updates performed; or NULL.
 * Returns PT_OK, PT_ENOTCONV (u_out still written) or PT_EDIVERGED, or an error.  PT_ETIMEOUT
 * means a bounded wait inside one of the row-streamed kernels (mixed precision) ran out: the
 * solve stopped at the next residual check and its iterate is not meaningful. */
pt_status pt_solve(pt_problem* p, double tol, int max_it, double* u_out, int u_out_on_device,
                   double* res_hist, int* iters);

/* Solve several problems together: one CUDA graph per launch holds one Uzawa iteration of every
 * unfinished problem (each problem's captured iteration as a child graph), so problems of any
 * grid and N_t share each launch; a problem that has converged stops doing work on the device
 * (its kernels see its done flag) and is dropped from the graph when it is rebuilt.
 *   ps[count]: distinct problems on the current device (each keeps its own data and options).
 *   tol[count], max_it[count]: per-problem stopping rules as in pt_solve.
 *   iters[count], status[count]: outputs (may be NULL); status[i] is PT_OK, PT_ENOTCONV or
 *   PT_EDIVERGED.  Solutions stay on the device: read them with pt_problem_get_state.
 * Returns PT_OK when every problem finished (whatever its status), or an error. */
pt_status pt_solve_batch(pt_problem** ps, int count, const double* tol, const int* max_it, int* iters,
                         pt_status* status);

/* ---- Serving: continuous batching of solves on one GPU -----------------------------------
 * A server owns one worker thread and the device current at creation.  Submitted requests are
 * queued; at every iteration boundary the worker admits queued requests while their estimated
 * device memory fits `hbm_budget` (0: 85 % of the free memory) and fewer than `max_active`
 * (0: 256) solves are active, keeps their state resident on the device, and advances all
 * active solves by graph launches that hold one Uzawa iteration of each (pt_solve_batch's
 * mechanism).  Finished solves are copied to host memory and their device memory is freed at
 * once, so later requests are admitted while others are still running. */
typedef struct pt_server pt_server;

pt_status pt_server_create(size_t hbm_budget, int max_active, pt_server** out);

/* Queue one solve.  The problem arguments are those of pt_problem_create (host arrays only; they
 * are copied); f == NULL selects the synthetic source of pt_problem_set_rhs_uniform with f_seed.
 * opts->stream is ignored.  *ticket identifies the request.  PT_ENOMEM if the request alone
 * exceeds the budget, PT_EBUSY once the server is being destroyed. */
pt_status pt_server_submit(pt_server* sv, const pt_grid* grid, int N_t, double T, const pt_coeff* coeff,
                           const double* f, unsigned long long f_seed, const double* u0,
                           const pt_options* opts, double tol, int max_it, unsigned long long* ticket);

/* Wait at most timeout_ms (< 0: no limit) for a request; then copy its solution ([N_t][n_s], host,
 * may be NULL), iteration count and solve status (PT_OK / PT_ENOTCONV / PT_EDIVERGED) and forget
 * the ticket.  PT_ETIMEOUT if it is not finished in time (the request stays queued or running);
 * the creation error of the request if it could not be started. */
pt_status pt_server_wait(pt_server* sv, unsigned long long ticket, int timeout_ms, double* u_out,
                         int* iters, pt_status* solve_status);

/* Latency percentiles (submit to result on the host) over the finished requests, space-time DOFs
 * per second from the first submission to the last completion, and the number finished. */
pt_status pt_server_stats(pt_server* sv, double* p50_ms, double* p99_ms, double* dofs_per_s, int* completed);

/* Finish every queued and running request, then stop the worker and free everything. */
void pt_server_destroy(pt_server* sv);

/* Copy the current iterates u_j and p_j (packed [N_t][n_s], FP64) of the problem's last solve.
 * The pair (u_j, p_j) is the complete state of the stationary Uzawa iteration (a checkpoint).
 * Either output may be NULL; on_device selects device (1) or host (0) memory for both. */
pt_status pt_problem_get_state(pt_problem* p, double* u_out, double* p_out, int on_device);

/* Device memory: *bytes_out = an upper estimate of what pt_problem_create allocates for this
 * grid, N_t and options (the serving loop's admission rule; no device work, no allocation), or
 * the bytes a created problem holds.  PT_EINVAL on NULL arguments. */
pt_status pt_problem_estimate_bytes(const pt_grid* grid, int N_t, const pt_options* opts, size_t* bytes_out);
pt_status pt_problem_device_bytes(const pt_problem* p, size_t* bytes_out);

/* Release all device memory of the problem; NULL is ignored. */
void pt_problem_destroy(pt_problem* p);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* pt_last_error(void);
const char* pt_status_string(pt_status s);

/* ---- Component entry points (device buffers, packed [N_t][n_s] FP64) ----------------
 * They run one stage of the method on the problem's grid, coefficient and stream, with the
 * problem's precision, and are what the per-kernel parity tests call.  in and out may not
 * alias.  Errors: PT_EINVAL on NULL pointers, PT_ECUDA. */

/* out = B u = (K (x) M) u + diag(tau_n A_n) u, u_0 := 0  (§2, eq. 2.3-2.4). */
pt_status pt_apply_B(pt_problem* p, const double* u_dev, double* out_dev);

/* out = S u with S = K^T A~^-1 K + K + K^T + A (§2, eq. 2.5; K = K (x) M, A = diag(tau_n A_n)) and
 * A~^-1 the problem's spatial solver of tau_n A_n: the exact Schur complement when that solver is
 * exact (1-D exact tridiagonal solves), else its inexact form.  FP64 problems only (PT_EINVAL). */
pt_status pt_apply_S(pt_problem* p, const double* u_dev, double* out_dev);

/* out = Phi^-T r: out_k = sum_n r_n sin((2k-1) n pi / (2N)), k = 1..N (§4, eq. 4.3 transposed). */
pt_status pt_dst_forward(pt_problem* p, const double* r_dev, double* out_dev);

/* out = Phi^-1 y: out_n = sum_k y_k sin((2k-1) n pi / (2N)), n = 1..N (§4, eq. 4.3). */
pt_status pt_dst_inverse(pt_problem* p, const double* y_dev, double* out_dev);

/* out = A~^-1 r: slice n gets the spatial solver of tau_n A_n (one V-cycle, or the exact
 * tridiagonal solve in 1-D) applied to r_n (§3, eq. 3.2).  Returns after the work has finished
 * on the stream (it reads back whether a bounded wait of a row-streamed kernel ran out:
 * PT_ETIMEOUT, out not meaningful). */
pt_status pt_precond_A(pt_problem* p, const double* r_dev, double* out_dev);

/* out = H~^-1 r = Phi^-1 Hhat~^-1 Phi^-T r with Hhat~_k^-1 = (2 tau/N) H~_k^-1 Abar H~_k^-1,
 * H_k = mu_k M + tau Abar, mu_k = 2 sin((2k-1) pi/(4N))  (§4, eq. 4.4-4.6).  Returns after the
 * work has finished, as pt_precond_A. */
pt_status pt_precond_H(pt_problem* p, const double* r_dev, double* out_dev);

/* ---- Allocation-free transform ------------------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot let the
 * library allocate device memory, because another allocator owns the device (for example a
 * framework's caching allocator that holds all of it) or because they run latency-critical
 * loops where a cudaMalloc, which may synchronise the device, is not acceptable.
 *
 * out_k = sum_n r_n sin((2k-1) n pi / (2N)) for each of `ncols` columns: the same transform as
 * pt_dst_forward, on caller-owned device arrays r_dev and out_dev of layout [N_t][ncols]
 * (FP64), without a pt_problem and without allocating anything.  Its working memory is one
 * file-scope device array of 16.2 MiB, reserved on a device when the library's device code is
 * loaded there (under CUDA's lazy module loading: at the first call on that device) and kept
 * until the process exits; limits: N_t a power of two <= 8192 and N_t * ceil32(ncols) <= 2^21
 * (else PT_EINVAL with a message naming the limit).  The first call on each device looks up
 * that array's device address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  The address stays valid for the life of the device's context: do not call this
 * entry point on a device after cudaDeviceReset.  All calls share the array, which keeps the last call's contents (each call rewrites
 * the tables and the padded copy of its input before using them), so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  Work is ordered on `stream` (NULL = legacy default stream); the
 * call returns without synchronising.  r_dev and out_dev may not alias. */
pt_status pt_dst_forward_noalloc(const double* r_dev, double* out_dev, int N_t, long long ncols,
                                 void* stream);

/* Number of kernel launches issued by this library since load (all problems); used to report
 * how many GPU kernels a timed region launched. */
unsigned long long pt_kernel_launch_count(void);

/* ---- Per-kernel timing (tracing) ------------------------------------------------------
 * pt_profile_enable(1) makes every later launch record a CUDA event pair on its stream; 0 stops
 * recording.  Per kernel name the library accumulates the event-measured time, the number of
 * launches, the algorithmic bytes (each operand read once, each result written once) and the
 * FP64 operation count of those launches.  pt_profile_reset clears the totals.
 * pt_profile_get(index, ...) synchronises the pending events and fills the totals of entry
 * `index` (name truncated to name_len - 1 characters); it returns the number of entries, or
 * -1 if index is out of range; index < 0 only returns the count.  Any output may be NULL. */
void pt_profile_enable(int on);
void pt_profile_reset(void);
int pt_profile_get(int index, char* name, int name_len, double* total_ms, double* bytes,
                   double* flops, unsigned long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* PT_H_ */
