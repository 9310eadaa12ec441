// Internal declarations shared by the CUDA translation units of the solver.
//
// Device layout of every space-time vector ("padded layout"): for a grid with n interior
// points per axis, pitch P = n + 1 (a power of two) and slice stride S = P^dim, the value at
// time slot t and interior coordinates (x, y, z) lives at  base[t*S + (z*P + y)*P + x].
// Positions with any coordinate equal to n are "ghosts" and always hold zero; so do the
// `guard` elements in front of slot 0.  The ghost at x = n of one row is the left neighbour
// of the next row, the ghost row y = n of one plane is the lower neighbour of the next
// plane, and so on, so a stencil reads its Dirichlet zeros without branches.  Every kernel
// writes zero (or nothing) at ghost positions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pt.h"

namespace pt {

constexpr int kMaxLevels = 16;
constexpr int kReduceBlocks = 1024;  // fixed grid of the residual reduction (deterministic)
constexpr int kCoarseMaxElems = 1024; // levels with P^dim <= this run inside one CTA per slice

// Counts every kernel launch of the library (reported by pt_kernel_launch_count) and, when
// timing is enabled, brackets it with CUDA events on its stream.  `bytes` is the algorithmic
// traffic of the launch (every operand read once, every result written once) and `flops` its
// FP64 arithmetic, both used for roofline figures.
// Kernels of the mixed-precision refinement do their work only on one kind of iteration (the
// FP64 step or the FP32 iterations between) and return at once on the other.  While kernels are
// timed one by one, the solve loop tells the scopes which kind the next iteration is
// (set_step_kind, per host thread), and a scope whose kernel works only on the other kind books
// no bytes or flops for that launch (its time still counts).
enum StepKind { kAnyStep = -1, kInnerStep = 0, kOuterStep = 1 };
void set_step_kind(int kind);

class LaunchScope {
 public:
  LaunchScope(const char* name, cudaStream_t st, double bytes = 0.0, double flops = 0.0,
              int works_on = kAnyStep);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  double bytes_, flops_;
  void* e0_;
};
void note_launch(int count = 1);
bool profiling_enabled();
// Raise the dynamic shared-memory limit of kernel `func` to `bytes` on the current device.
// cudaFuncSetAttribute acts per device, so the call is made once per (device, kernel) pair;
// the record of which pairs are done is guarded by a mutex (launches may come from several
// host threads, e.g. the serving worker and a caller).  Returns the CUDA status of the call.
cudaError_t set_smem_limit(const void* func, int bytes);
// Number of CTAs of kernel `func` (threads per CTA, dynamic shared memory) resident at once on
// the current device -- SM count x occupancy, computed once per (device, kernel) -- clamped to
// [1, cap].  A persistent grid of this size runs in one wave.
int resident_grid(const void* func, int threads, size_t smem, int cap);
// Launches between capture_begin and capture_end (same thread) are recorded into a CUDA graph:
// they are not counted as executed; capture_end returns how many were recorded.
void capture_begin();
unsigned long long capture_end();

struct Level {
  int n;             // interior points per axis
  int P;             // pitch n + 1
  int logP;          // log2(P)
  long long S;       // slice stride P^dim
  long long guard;   // zero elements in front of slot 0 (>= P^(dim-1) + ... + P + 1, rounded)
  double h;          // 1 / (n + 1)
  long long tab;     // offset of this level's coefficient tables (2*dim arrays of P entries)
};

// Coefficient of one batch of slices at one level:
//   a(face) = a0 + cth[b] * g_face(axis d) * prod_{e != d} g_node(axis e)
// cth[b] = c * g_t(pi m_t t_b) for the slice's time (or c * mean over steps for Abar).
template <typename T>
struct StencilGeom {
  int dim, n, P, logP;
  long long S;
  const T* tab;   // level tables: node_x, face_x, node_y, face_y, node_z, face_z (P each)
  T a0;
  T h2inv;        // 1/h^2
  int mass = 0;   // mass matrix M of eq. 2.1 in K (x) M: 0 = identity, 1 = P1 mass over h^d (dim <= 2)
};

// Per-step factors of the time grid (§2, eq. 2.1), [N] each: the step lengths tau_n, and against
// the reference step tau = T/N of the preconditioner sigma_n = tau_n / tau and rho_n = tau / tau_n
// (all 1 for uniform steps).  tau_n A_n = sigma_n (tau A_n), and the V-cycle being homogeneous of
// degree -1 in the operator, A~^-1 for tau_n A_n is rho_n times the V-cycle for tau A_n: the kernels
// that form the A~ input scale it by rho_n, and the multigrid kernels keep the scale tau.
template <typename T>
struct Steps {
  const T* tau;
  const T* sig;
  const T* rho;   // null: no scaling of the A~ input (the Krylov path's operator application)
  bool uniform;   // all steps equal (sigma = rho = 1): kernels may skip the factors
};

// Batched operator L_b = sig[b] I + s * A(cth[b]) on one level, used by the V-cycle.
template <typename T>
struct OpBatch {
  const T* sig;   // [B] mass shift (0 for tau_n A_n, mu_k for H_k = mu_k M + tau Abar)
  const T* cth;   // [B] coefficient time factors (times c)
  T s;            // scale of A (tau)
  T omega;        // Jacobi weight
  int mass = 0;   // M in sig M + s A: 0 = identity, 1 = P1 mass over h^d (dim <= 2)
};

// ---- stencil / residual kernels (kernels_stencil.cu) --------------------------------------
// F (padded) = scale * pack(src) (+ u0 on slot 0 when u0 != nullptr), src packed [N][ns].
// scale_t: [N] per-slice factors (the step lengths) replacing scale when not null.
void launch_pack(const double* src, const double* u0, double* dst, double scale, const double* scale_t, int dim,
                 int n, int P, int logP, long long S, int N, cudaStream_t st);
// F (padded) = scale * (2 U - 1) (+ u0 on slot 0), U from SplitMix64(seed) at the packed index
void launch_pack_uniform(unsigned long long seed, const double* u0, double* dst, double scale,
                         const double* scale_t, int dim, int n, int logP, long long S, int N, cudaStream_t st);
template <typename T>
void launch_unpack(const T* src, double* dst, int dim, int n, int P, int logP, long long S, int N,
                   cudaStream_t st);
template <typename T>
void launch_pack_typed(const double* src, T* dst, int dim, int n, int P, int logP, long long S,
                       int N, cudaStream_t st);

// out = B u (FP64)
void launch_apply_B(const double* u, double* out, StencilGeom<double> g, const double* cth, Steps<double> sp,
                    int N, cudaStream_t st);

// rho_n r_p with r_p = K u - tau_n A_n p - F   (written in precision Tp)
template <typename Tp>
void launch_resid_p(const double* u, const double* p, const double* F, Tp* rp, StencilGeom<double> g,
                    const double* cth, Steps<double> sp, int N, const int* done, cudaStream_t st);

// r_u = F - K^T p - (K + K^T + tau_n A_n) u, partial sums of ||F - B u||^2 per block
template <typename Tp>
void launch_resid_u(const double* u, const double* p, const double* F, Tp* ru, double* partials,
                    StencilGeom<double> g, const double* cth, Steps<double> sp, int N, const int* done,
                    cudaStream_t st);

// Mixed precision: bres = F - B u (FP64, stored, norm partials) and rho_n r_p, r_p = -bres -
// tau_n A_n (p + u) with the second stencil in FP32; then r_u = bres - K^T (p + u) (no stencil).
void launch_resid_bres_mixed(const double* u, const double* p, const double* F, double* bres, float* rp,
                             double* partials, StencilGeom<double> g, const double* cth, Steps<double> sp, int N,
                             const int* done, cudaStream_t st);
template <typename Tp>
void launch_resid_u_from_bres(const double* bres, const double* u, const double* p, Tp* ru, long long S,
                              int N, int dim, int n, const int* done, cudaStream_t st, double sgn = 1.0);
// 2-D (n + 1 >= 32) fused outer residual: bres = F - B u (FP64, stored, norm partials over a fixed
// grid of kReduceBlocks blocks) and rho_n r_p, r_p = -bres - tau_n A (p + u), in precision W (FP32:
// the w-stencil in FP32; FP64: all in FP64).  tab / tabf: level-0 coefficient tables in FP64 / FP32;
// tau: the reference step (the stencils are formed for tau A_n and scaled by sigma_n).
// jd: cached (w/D, D) pairs of tau A_n at level 0, or null (FP64: the stencils then use D)
template <typename W>
void launch_resid_bres_2d(const double* u, const double* p, const double* F, double* bres, W* rp,
                          double* partials, const double* tab, const float* tabf, const double* cth, double a0,
                          double tau, double h, int n, int logP, long long S, int N, const int* done,
                          const double* jd, Steps<double> sp, cudaStream_t st);

// out = scale * A(cthbar) z on one batch (Abar apply of the Hhat block solve)
template <typename T>
void launch_apply_A_scaled(const T* z, T* out, StencilGeom<T> g, T cth, T scale, int N,
                           const int* done, cudaStream_t st);

// x[i] *= f[i >> logS] (padded space-time vector, one factor per slot)
template <typename T>
void launch_scale_slices(T* x, const T* f, int logS, long long total, cudaStream_t st);

// partial sums of ||v||^2 (padded vector, ghosts are zero)
void launch_norm2_partials(const double* v, long long count, double* partials, cudaStream_t st);
// out = M v per slice (g.mass: identity or P1 mass), x = a x
void launch_apply_mass(const double* v, double* out, StencilGeom<double> g, int N, cudaStream_t st);
void launch_scale(double* x, double a, long long total, cudaStream_t st);
// out = rho_t (K (x) M) u;  acc += (K^T (x) M)(z + u)   (the Schur complement apply, eq. 2.5)
void launch_apply_K(const double* u, double* out, StencilGeom<double> g, const double* rho, int N, cudaStream_t st);
void launch_add_KT(double* acc, const double* z, const double* u, StencilGeom<double> g, int N, cudaStream_t st);

// Device state of one solve.
struct SolveState {
  int done;      // 1 once converged / failed / exhausted
  int status;    // pt_status of the solve
  int iters;     // number of Uzawa updates performed
  int j;         // index of the iterate whose residual the next finalize records
  double fnorm2; // ||F||^2
  double last_res;
  double tol;
  int max_it;
  int outer;     // mixed precision: this iteration starts with the FP64 refinement step
  int fault;     // set by a streamed kernel whose bounded wait ran out; the next finalize ends the
                 // solve with PT_ETIMEOUT
};

// Mixed precision as iterative refinement (kernels_ir.cu): FP64 step every kOuter iterations
// (and on request of the FP32 residual estimate), FP32 iterations on the corrections between.
constexpr int kOuter = 16;
void launch_ir_begin(SolveState* st, int kouter, cudaStream_t s);
void launch_ir_fold(double* u, double* p, float* du, float* dp, long long total, const SolveState* st,
                    cudaStream_t s);
void launch_ir_outer(const double* u, const double* p, const double* F, float* R1, float* R2, float* rp,
                     double* partials, StencilGeom<double> g, const double* cth, Steps<double> sp, int N,
                     const SolveState* st, cudaStream_t s);
void launch_ir_inner(const float* du, const float* dp, const float* R1, const float* R2, float* bp, float* rp,
                     double* partials, StencilGeom<float> g, const float* cth, Steps<float> sp, int N,
                     const SolveState* st, cudaStream_t s);
// 2-D (n + 1 >= 32) warp-strip forms of launch_ir_outer / launch_ir_inner (kernels_resid2d.cu);
// tab / tabf: level-0 FP64 / FP32 tables
void launch_ir_outer_2d(const double* u, const double* p, const double* F, float* R1, float* R2, float* rp,
                        double* partials, const double* tab, const float* tabf, const double* cth, double a0,
                        double tau, double h, int n, int logP, long long S, int N, Steps<double> sp,
                        const SolveState* st, cudaStream_t s);
// Occupancy queries of the streamed 2-D and 3-D kernels, done at problem setup (outside any
// stream capture).
void prepare_ir_inner_2d();
void prepare_ir_inner_3d();
void prepare_level3_rows();  // the row-streamed 3-D FP32 V-cycle levels (kernels_mg.cu)
void launch_ir_inner_2d(const float* du, const float* dp, const float* R1, const float* R2, float* bp, float* rp,
                        double* partials, const float* tabf, const float* cthf, double a0, double tau, double h,
                        int n, int logP, long long S, int N, Steps<float> sp, SolveState* st, cudaStream_t s);
void launch_ir_inner_3d(const float* du, const float* dp, const float* R1, const float* R2, float* bp, float* rp,
                        double* partials, const float* tabf, const float* cthf, double a0, double tau, double h,
                        int n, int logP, long long S, int N, Steps<float> sp, SolveState* st, cudaStream_t s);
void launch_ir_outer_3d(const double* u, const double* p, const double* F, float* R1, float* R2, float* rp,
                        double* partials, const double* tab, const float* tabf, const double* cth, double a0,
                        double tau, double h, int n, int logP, long long S, int N, Steps<double> sp,
                        const SolveState* st, cudaStream_t s);
void launch_ir_resid_u(const float* bp, const float* R2, const float* du, const float* dp, float* ru, long long S,
                       int N, const SolveState* st, cudaStream_t s);
void launch_ir_finalize(const double* partials, SolveState* state, double* hist, cudaStream_t s);

// sum partials in fixed order; residual of iterate state->j -> hist[j], sets flags, advances j.
void launch_finalize_residual(const double* partials, SolveState* state, double* hist, cudaStream_t st);
// start of a solve: ||F||^2 and the reset of the counters
void launch_finalize_fnorm(const double* partials, SolveState* state, double tol, int max_it,
                           cudaStream_t st);

// out[i] = states[i]->done for a batch of solves
void launch_gather_done(SolveState* const* states, int count, int* out, cudaStream_t st);
// the control kernel of the device-side batch loop (see pt_solve_batch): rounds += 1; continue
// while more than keep_above of states[idx[0..count)] are unfinished and rounds < limit
void launch_batch_control(SolveState* const* states, const int* idx, int count, int keep_above, int* rounds,
                          int limit, cudaGraphConditionalHandle handle, cudaStream_t st);

// elementwise y += a * x over count padded entries (x in Tp)
template <typename Tp>
void launch_axpy(double* y, const Tp* x, double a, long long count, const int* done, cudaStream_t st);

// ---- multigrid (kernels_mg.cu) ----------------------------------------------------------
struct MGLevelBufs {
  void* b;  // rhs
  void* x;  // smoothed iterate / correction
  void* r;  // residual
};

template <typename T>
struct MGPlan {
  int dim, nlev, lc;  // number of levels, first level solved by the one-CTA coarse kernel
  Level lev[kMaxLevels];
  const T* tab;       // all level tables
  T a0;
  MGLevelBufs buf[kMaxLevels];
  int B;              // slices in the batch
  int* fault;         // SolveState::fault of the owning problem (bounded waits of streamed kernels)
};

// One V(1,1) cycle with zero initial guess on all B slices: x = V(b).
// mode 0: out = x;  mode 1: out += x (accumulate, out in FP64 when accum_fp64 != 0).
template <typename T>
void vcycle(const MGPlan<T>& plan, OpBatch<T> op, const T* b0, void* out, int mode, int out_fp64,
            const int* done, cudaStream_t st);

// r = b - L x for a batch of slices on one level (L = sig I + s A(cth) per slice)
template <typename T>
void launch_op_residual(const T* b, const T* x, T* r, StencilGeom<T> g, OpBatch<T> op, int B,
                        const int* done, cudaStream_t st);

// Levels lc..nlev-1 of a V-cycle (one CTA per slice); input bl at level lc.
template <typename T>
void vcycle_coarse(const MGPlan<T>& plan, OpBatch<T> op, const T* bl, void* out, int mode, int out_fp64,
                   const int* done, cudaStream_t st);

// Fused 2-D V-cycle (kernels_mg2d.cu); mode 1 accumulates into out (precision T when !out_fp64).  var: variable face coefficients (else the constant a0);
// dinv_slice[l]: per-level [B] arrays of w/D for constant coefficients; jinv[l]: per-level cached
// w/D (padded layout) for variable coefficients, or nullptr to compute it in the kernels.
template <typename T>
void vcycle2d(const MGPlan<T>& plan, OpBatch<T> op, const T* b0, void* out, int mode, int out_fp64,
              bool var, const T* const* dinv_slice, const T* const* jinv, const int* done,
              cudaStream_t st);
template <typename T>
void launch_make_jinv(T* jinv, StencilGeom<T> g, OpBatch<T> op, int B, cudaStream_t st);

// exact batched tridiagonal solve for 1-D: x_b = (sig_b I + s A(cth_b))^-1 r_b
template <typename T>
void launch_tridiag(const T* r, void* out, int mode, int out_fp64, StencilGeom<T> g, OpBatch<T> op,
                    int B, T* work, const int* done, cudaStream_t st);

// ---- temporal DST (kernels_dst.cu) ------------------------------------------------------
template <typename T>
struct DstPlan {
  int N, logN;
  const T* tw;    // [N/2] (cos, sin)(2 pi k / N) interleaved (N a power of two)
  const T* pre;   // [N]   (cos, sin)(pi m / (2N)) interleaved
  // Bluestein tables, used when M > 0 (N not a power of two): M = 2^logM >= 2N - 1
  int M = 0, logM = 0;
  const T* chirp = nullptr;  // [N] e^{i pi m^2 / N}
  const T* gfwd = nullptr;   // [M] FFT_M of the chirp filter for the e^{-} transform, bit-reversed, / M
  const T* ginv = nullptr;   // [M] same for the e^{+} transform
  const T* twM = nullptr;    // [M/2] e^{2 pi i k / M}
  int C = 0;                 // complex columns per CTA (0: chosen from shared-memory size)
  const T* twS = nullptr;    // [N] e^{-2 pi i e / N} (power-of-two N: radix-8 Stockham kernels)
};

// in-place forward transform: x_k <- sum_n x_n sin((2k-1) n pi/(2N)) for every interior column
// (ghost columns of the grid with n interior points per axis are written as zero)
template <typename T>
void launch_dst_forward(T* x, long long S, int dim, int n, int logP, DstPlan<T> plan, const int* done,
                        cudaStream_t st);

// inverse + update: u_n += omega * sum_k y_k sin((2k-1) n pi/(2N)); u in FP64 (mode 1), u of
// type T (mode 2), or out = transform (mode 0, out of type T)
template <typename T>
void launch_dst_inverse(const T* y, void* out, int mode, double omega, long long S, int dim, int n,
                        int logP, DstPlan<T> plan, const int* done, cudaStream_t st);

// Spatial sine transforms of type I (kernels_dsti.cu), in place on padded slices, n + 1 <= 4096:
//   rows:  every x-line v <- S v;  cols: every line along axis 1 (y) or 2 (z) v <- S v, or with
//   `scale`, v <- S diag(g) S v with g the exact block-solve factor from the table `gtab`.
// Tables (type T): tw [n+1] complex e^{-2 pi i e/(n+1)}; sn [(n+1)/2 + 1] sin(pi j/(n+1)) / 2;
// gtab padded like the data (B slots): c0 l / (mu_k + tau l)^2, l = sum over the axes of
// lam[pos] = (4 a0/h^2) sin^2(pi (pos+1) h/2) (FP64 tables lam [n+1], mu [B]), 0 at ghosts.
constexpr int kDstiMaxM = 4096;
template <typename T>
void launch_dsti_rows(T* x, int dim, int n, int logP, long long S, int B, const void* tw, const void* sn,
                      cudaStream_t st);
// Without gtab (FP32), the scaled call forms the factor per point from DstiFactor, as
// c l / (m_k + l)^2 with m_k = mu_k / tau and c = c0 / tau^2: lam [n+1] and m [B] in the kernel's
// type.
struct DstiFactor {
  const void* lam;
  const void* m;
  double c;
};
template <typename T>
void launch_dsti_cols(T* x, int dim, int n, int logP, long long S, int B, int axis, const void* tw,
                      const void* sn, const void* gtab, bool scale, cudaStream_t st,
                      const DstiFactor* factor = nullptr);
// Planes that fit in one CTA's shared memory (32 <= n + 1 <= kPlaneMaxM): x and y transforms of a
// whole plane in one pass.  mode 0 (2-D, FP32): the whole block solve S_x S_y diag(g) S_y S_x
// (factor as in launch_dsti_cols); mode 1 (3-D): S_y S_x; mode 2 (3-D): S_x S_y; mode 3 (3-D):
// S_z diag(g) S_z on the x-z planes.
constexpr int kPlaneMaxM = 128;
template <typename T>
bool dsti_plane_ok(int dim, int n);
template <typename T>
void launch_dsti_plane(T* x, int dim, int n, int logP, long long S, int B, int mode, const void* tw, const void* sn,
                       const void* gtab, cudaStream_t st, const DstiFactor* factor);
// FP64 2-D: y-part of the exact block solve by tridiagonal eliminations (kernels_dsti.cu);
// w padded like the data: the LU pivots 1/d'_i of every (k, x-frequency) column.
template <typename T>
void launch_hsolve_trid_table(T* w, const double* lam, const double* mu, double tau, double a0h2, int n, int logP,
                              long long S, int N, cudaStream_t st);
template <typename T>
void launch_hsolve_trid(T* X, const T* w, const double* lam, double tau, double a0h2, double scale, int n,
                        int logP, long long S, int N, cudaStream_t st);
template <typename T>
void launch_dsti_scale_table(T* g, const double* lam, const double* mu, double tau, double c0, int dim, int logP,
                             long long S, int B, cudaStream_t st);

// Krylov acceleration (kernels_krylov.cu): pairs (p, u) of padded FP64 space-time vectors.
void launch_apply_saddle(const double* zp, const double* zu, double* op, double* ou, StencilGeom<double> g,
                         const double* cth, Steps<double> sp, int N, cudaStream_t st);
// partials [nv (+1 with self: <w, w>)][kReduceBlocks]
void launch_multidot(const double* const* vp, const double* const* vu, const double* wp, const double* wu, int nv,
                     int self, long long total, double* partials, cudaStream_t st);
void launch_multiaxpy(const double* const* vp, const double* const* vu, const double* c, int nv, double* wp,
                      double* wu, long long total, cudaStream_t st);
// (yp, yu) = s (xp, xu), times rho[t] on slice t (slices of 2^logS elements) when rho is not null
void launch_scale_pair(const double* xp, const double* xu, double s, double* yp, double* yu, long long total,
                       cudaStream_t st, const double* rho = nullptr, int logS = 0);
void launch_uzawa_ru(const double* vu, const double* zp, double* ru, long long S, int N, cudaStream_t st);

// Problem hooks for the serving loop (defined in capi.cu).
pt_status problem_begin(pt_problem* p, double tol, int max_it);   // reset + captured iteration graph
cudaGraph_t problem_graph(pt_problem* p, unsigned long long* kernels);
SolveState* problem_state(pt_problem* p);
pt_status problem_result(pt_problem* p, int* iters, pt_status* status);
size_t problem_bytes(const pt_problem* p);
long long problem_dofs(const pt_problem* p);
size_t estimate_problem_bytes(const pt_grid* g, int N_t, const pt_options* o);

// Set the thread-local message returned by pt_last_error().
void set_last_error(const char* msg);

// Forward transform of ncols packed columns at pitch S (a multiple of 32) without event
// recording; used by the allocation-free entry point.
void launch_dst_forward_plain(double* x, long long S, int ncols, DstPlan<double> plan, cudaStream_t st);

}  // namespace pt
