// C ABI of the solver (include/pt.h): problem set-up, the inexact Uzawa loop of §3, eq. 3.1,
// and the component entry points.  All arithmetic runs in the kernels of the other
// translation units; this file owns device memory, tables and the launch sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "pt_internal.cuh"

namespace {
thread_local std::string g_err;

pt_status fail(pt_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define PT_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)

#define PT_CHECK_LAUNCH()                                                                \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess) return fail(PT_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

double trig(int kind, double arg) {
  if (kind == PT_TRIG_SIN) return std::sin(arg);
  if (kind == PT_TRIG_COS) return std::cos(arg);
  return 1.0;
}
}  // namespace


namespace pt {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace pt

using namespace pt;

struct pt_problem {
  int dim = 0, n = 0, N = 0, logN = 0;
  double T = 0.0, tau = 0.0;
  pt_coeff coeff{};
  pt_options opt{};
  int mixed = 0;
  int exact1d = 0;
  int mass = 0;                                 // M of eq. 2.1: 0 identity, 1 P1 mass over h^d
  double omega = 0.5;
  double jacobi = 0.0;
  cudaStream_t st = nullptr;
  int device = 0;
  int nlev = 0, lc = 0;
  Level lev[kMaxLevels];
  long long ns = 0;   // interior points per slice
  // device memory
  std::vector<void*> allocs;
  double *u = nullptr, *p = nullptr, *F = nullptr;
  void *W1 = nullptr, *W2 = nullptr;            // preconditioner precision, fine level
  void* W3 = nullptr;                           // residual between V-cycles of an H_k solve
  double* bres = nullptr;                       // F - B u of the current iterate (FP64, 2-D)
  bool hdst = false;                            // exact H_k solves by spatial sine transforms
  void* dsti_tw = nullptr;                      // [n+1] complex e^{-2 pi i e / (n+1)}   (type T)
  void* dsti_sn = nullptr;                      // [(n+1)/2 + 1] sin(pi j / (n+1)) / 2
  double* dsti_lam = nullptr;                   // [n+1] (4 a0/h^2) sin^2(pi k h / 2) at k-1, 0 at n
  double* dsti_mu = nullptr;                    // [N] mu_k
  void* dsti_g = nullptr;                       // padded, type T: block-solve factor of each point (FP64)
  void* dsti_lamT = nullptr;                    // FP32: lam and mu_k / tau in FP32, the factor formed per point
  void* dsti_muT = nullptr;
  void* hy_w = nullptr;                         // 2-D: padded LU pivots (type T) of the y-tridiagonal H_k
  int nv_h = 2;                                 // V-cycles per H_k solve
  void* mg_b[kMaxLevels] = {};
  void* mg_x[kMaxLevels] = {};
  void* mg_r[kMaxLevels] = {};
  double* tab_d = nullptr;
  float* tab_f = nullptr;
  double* cth_d = nullptr;                      // [N] c * g_t(pi m_t t_n)
  std::vector<double> steps;                    // host copy of tau_1..tau_N (empty: uniform T/N)
  std::vector<double> tn;                       // t_1..t_N
  double* stp_d = nullptr;                      // [3N] tau_n | sigma_n = tau_n/tau | rho_n = tau/tau_n
  float* stp_f = nullptr;                       // the same in FP32
  void* sigA = nullptr;                         // [N] zeros       (precond precision)
  void* cthA = nullptr;                         // [N] c g_t(t_n)
  void* sigH = nullptr;                         // [N] mu_k
  void* cthH = nullptr;                         // [N] c * gbar (time mean of g_t over (0, T))
  double cthbar = 0.0;
  void* dst_tw = nullptr;                       // [N/2] complex
  void* dst_pre = nullptr;                      // [N] complex
  int blueM = 0, blueLogM = 0;                  // Bluestein length (N not a power of two)
  void* dst_twS = nullptr;                      // [N] complex e^{-2 pi i e / N} (power-of-two N)
  // Krylov acceleration (FP64): V[0..m], Z[0..m-1] and a work pair, device pointer tables
  int kr_m = 0;
  std::vector<double*> kr_vp, kr_vu, kr_zp, kr_zu;
  double* kr_wp = nullptr;
  double* kr_wu = nullptr;
  double* kr_zero = nullptr;      // a zero right-hand side (2-D: Sad by the residual kernels)
  double** kr_tab = nullptr;      // device: [vp(m+1) | vu(m+1) | zp(m) | zu(m)]
  double* kr_coef = nullptr;      // device [m + 1]
  double* kr_part = nullptr;      // device [(m + 1) * kReduceBlocks]
  float* ir_du = nullptr;                       // mixed: FP32 corrections of u and p, residuals
  float* ir_dp = nullptr;
  float* ir_R1 = nullptr;
  float* ir_R2 = nullptr;
  float* ir_bp = nullptr;
  void* blue_chirp = nullptr;                   // [N] complex
  void* blue_gfwd = nullptr;                    // [M] complex
  void* blue_ginv = nullptr;                    // [M] complex
  void* blue_tw = nullptr;                      // [M/2] complex
  void* tri_work = nullptr;
  bool hvar = true;                             // Abar has a non-constant coefficient
  void* dinvH[kMaxLevels] = {};                 // [N] w / D of H_k per level (constant Abar)
  void* jinvA[kMaxLevels] = {};                 // cached (w / D, D) of tau A_n per level (FP64, 2-D)
  double* partials = nullptr;
  SolveState* state = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  double* tmpA = nullptr;                       // FP64 padded scratch for component calls
  double* tmpB = nullptr;
  SolveState* host_state = nullptr;             // pinned
  size_t bytes = 0;
  int dstC = 0;                                 // temporal-transform columns per CTA (0 = auto)
  int coarse_elems = kCoarseMaxElems;           // one-CTA coarse-level threshold
  int lc_min = 0;                               // smallest lc whose buffers exist (largest threshold)
  int lc_max = 0;                               // largest lc whose buffers exist (smallest threshold)
  bool tuned = false;
  // captured iteration graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_iters = 0;
  unsigned long long graph_kernels = 0;
  double* graph_hist = nullptr;
  int graph_dstC = -1, graph_lc = -1;
};

namespace {

// Zero elements in front of slot 0: the lowest index a kernel reads is the diagonal corner
// (-1, -1, -1) of the prolongation, at -(P^(d-1) + ... + P + 1).
long long padded_guard(const Level& L, int dim) {
  long long g = 0, pk = 1;
  for (int d = 0; d < dim; ++d) {
    g += pk;
    pk *= L.P;
  }
  return (g + 31) & ~31LL;
}

template <typename T>
T* alloc_padded(pt_problem* p, const Level& L, int slots, pt_status* st) {
  const long long guard = padded_guard(L, p->dim);
  const size_t count = (size_t)(guard + L.S * (long long)slots + 64);
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    *st = fail(PT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return nullptr;
  }
  p->allocs.push_back(ptr);
  p->bytes += count * sizeof(T);
  e = cudaMemsetAsync(ptr, 0, count * sizeof(T), p->st);
  if (e != cudaSuccess) {
    *st = fail(PT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    return nullptr;
  }
  return (T*)ptr + guard;
}

void* alloc_bytes(pt_problem* p, size_t bytes, pt_status* st) {
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) {
    *st = fail(PT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return nullptr;
  }
  p->allocs.push_back(ptr);
  p->bytes += bytes;
  return ptr;
}

template <typename T>
pt_status upload(pt_problem* p, void* dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  PT_CUDA(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, p->st));
  PT_CUDA(cudaStreamSynchronize(p->st));
  return PT_OK;
}

template <typename T>
StencilGeom<T> geom(const pt_problem* p, int l) {
  StencilGeom<T> g;
  g.dim = p->dim;
  g.n = p->lev[l].n;
  g.P = p->lev[l].P;
  g.logP = p->lev[l].logP;
  g.S = p->lev[l].S;
  g.tab = (sizeof(T) == 8 ? (const T*)(const void*)p->tab_d : (const T*)(const void*)p->tab_f) + p->lev[l].tab;
  g.a0 = (T)p->coeff.a0;
  g.h2inv = (T)(1.0 / (p->lev[l].h * p->lev[l].h));
  g.mass = p->mass;
  return g;
}

template <typename T>
MGPlan<T> mg_plan(const pt_problem* p) {
  MGPlan<T> m;
  m.dim = p->dim;
  m.nlev = p->nlev;
  m.lc = p->lc;
  for (int l = 0; l < p->nlev; ++l) {
    m.lev[l] = p->lev[l];
    m.buf[l].b = p->mg_b[l];
    m.buf[l].x = p->mg_x[l];
    m.buf[l].r = p->mg_r[l];
  }
  m.tab = sizeof(T) == 8 ? (const T*)(const void*)p->tab_d : (const T*)(const void*)p->tab_f;
  m.a0 = (T)p->coeff.a0;
  m.B = p->N;
  m.fault = &p->state->fault;
  return m;
}

// per-step factors tau_n, sigma_n, rho_n (device tables)
Steps<double> steps_d(const pt_problem* p) {
  return {p->stp_d, p->stp_d + p->N, p->stp_d + 2 * p->N, p->steps.empty()};
}
Steps<float> steps_f(const pt_problem* p) {
  return {p->stp_f, p->stp_f + p->N, p->stp_f + 2 * p->N, p->steps.empty()};
}

template <typename T>
OpBatch<T> op_A(const pt_problem* p) {
  OpBatch<T> o;
  o.sig = (const T*)p->sigA;
  o.cth = (const T*)p->cthA;
  o.s = (T)p->tau;
  o.omega = (T)p->jacobi;
  return o;
}

template <typename T>
OpBatch<T> op_H(const pt_problem* p) {
  OpBatch<T> o;
  o.sig = (const T*)p->sigH;
  o.cth = (const T*)p->cthH;
  o.s = (T)p->tau;
  o.omega = (T)p->jacobi;
  o.mass = p->mass;  // H_k = mu_k M + tau Abar
  return o;
}

template <typename T>
DstPlan<T> dst_plan(const pt_problem* p) {
  DstPlan<T> d;
  d.N = p->N;
  d.logN = p->logN;
  d.tw = (const T*)p->dst_tw;
  d.pre = (const T*)p->dst_pre;
  d.M = p->blueM;
  d.logM = p->blueLogM;
  d.chirp = (const T*)p->blue_chirp;
  d.gfwd = (const T*)p->blue_gfwd;
  d.ginv = (const T*)p->blue_ginv;
  d.twM = (const T*)p->blue_tw;
  d.C = p->dstC;
  d.twS = (const T*)p->dst_twS;
  return d;
}

// In-place radix-2 FFT (sign -1) of n = 2^k complex values on the host, for the Bluestein
// filter spectra (computed once per problem).
void host_fft(std::vector<double>& re, std::vector<double>& im) {
  const size_t n = re.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      std::swap(re[i], re[j]);
      std::swap(im[i], im[j]);
    }
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const double ang = -2.0 * M_PI / (double)len;
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const double wr = std::cos(ang * k), wi = std::sin(ang * k);
        const size_t a = i + k, b = i + k + len / 2;
        const double xr = re[b] * wr - im[b] * wi, xi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - xr;
        im[b] = im[a] - xi;
        re[a] += xr;
        im[a] += xi;
      }
  }
}

// A~^-1 applied to rhs b (precision T, fine padded) -> out (mode 0 write T, mode 1 += into FP64)
template <typename T>
void apply_precond_A(pt_problem* p, const T* b, void* out, int mode, int out_fp64, const int* done) {
  if (p->exact1d) {
    launch_tridiag<T>(b, out, mode, out_fp64, geom<T>(p, 0), op_A<T>(p), p->N, (T*)p->tri_work, done,
                      p->st);
  } else if (p->dim == 2) {
    const T* jinv[kMaxLevels];
    for (int l = 0; l < kMaxLevels; ++l) jinv[l] = (const T*)p->jinvA[l];
    vcycle2d<T>(mg_plan<T>(p), op_A<T>(p), b, out, mode, out_fp64, true, nullptr,
                p->jinvA[0] ? jinv : nullptr, done, p->st);
  } else {
    vcycle<T>(mg_plan<T>(p), op_A<T>(p), b, out, mode, out_fp64, done, p->st);
  }
}

// One V-cycle for all H_k: out = V(b) (mode 0) or out += V(b) (mode 1)
template <typename T>
void vcycle_H(pt_problem* p, const T* b, T* out, int mode, const int* done) {
  if (p->dim == 2 && !p->mass) {
    const T* dinv[kMaxLevels];
    for (int l = 0; l < kMaxLevels; ++l) dinv[l] = (const T*)p->dinvH[l];
    vcycle2d<T>(mg_plan<T>(p), op_H<T>(p), b, out, mode, 0, p->hvar, p->hvar ? nullptr : dinv, nullptr,
                done, p->st);
  } else {
    vcycle<T>(mg_plan<T>(p), op_H<T>(p), b, out, mode, 0, done, p->st);
  }
}

// H_k solve (§4, eq. 4.6): exact in 1-D if requested, else nv_h V-cycles x <- x + V(b - H_k x)
template <typename T>
void apply_Hk_solve(pt_problem* p, const T* b, T* out, const int* done) {
  if (p->exact1d) {
    launch_tridiag<T>(b, out, 0, 0, geom<T>(p, 0), op_H<T>(p), p->N, (T*)p->tri_work, done, p->st);
    return;
  }
  vcycle_H<T>(p, b, out, 0, done);
  for (int c = 1; c < p->nv_h; ++c) {
    launch_op_residual<T>(b, out, (T*)p->W3, geom<T>(p, 0), op_H<T>(p), p->N, done, p->st);
    vcycle_H<T>(p, (const T*)p->W3, out, 1, done);
  }
}

// W1 = rhat (after the temporal transform) -> yhat = (2 tau/N) H~_k^-1 Abar H~_k^-1 rhat for all k
// (§4, eq. 4.4/4.6); returns the buffer holding yhat (W1 for the exact transform solve, else W2).
template <typename T>
T* block_solve(pt_problem* p, const int* done) {
  T* W1 = (T*)p->W1;
  T* W2 = (T*)p->W2;
  if (p->hdst) {
    const Level& L = p->lev[0];
    if (p->hy_w) {
      // FP64 2-D: S_x [T_k^-1 Z T_k^-1]_y S_x, the y-part by tridiagonal eliminations
      launch_dsti_rows<T>(W1, p->dim, p->n, L.logP, L.S, p->N, p->dsti_tw, p->dsti_sn, p->st);
      launch_hsolve_trid<T>(W1, (const T*)p->hy_w, p->dsti_lam, p->tau, p->coeff.a0 / (L.h * L.h),
                            (2.0 * p->tau / p->N) * (2.0 / L.P), p->n, L.logP, L.S, p->N, p->st);
      launch_dsti_rows<T>(W1, p->dim, p->n, L.logP, L.S, p->N, p->dsti_tw, p->dsti_sn, p->st);
      return W1;
    }
    const DstiFactor f = {p->dsti_lamT, p->dsti_muT,
                          (2.0 * p->tau / p->N) * std::pow(2.0 / L.P, p->dim) / (p->tau * p->tau)};
    if (dsti_plane_ok<T>(p->dim, p->n)) {
      // whole planes in shared memory: one pass (2-D) or the xy passes around the z-axis pass (3-D)
      if (p->dim == 2) {
        launch_dsti_plane<T>(W1, 2, p->n, L.logP, L.S, p->N, 0, p->dsti_tw, p->dsti_sn, p->dsti_g, p->st,
                             p->dsti_g ? nullptr : &f);
      } else {
        launch_dsti_plane<T>(W1, 3, p->n, L.logP, L.S, p->N, 1, p->dsti_tw, p->dsti_sn, nullptr, p->st, nullptr);
        launch_dsti_plane<T>(W1, 3, p->n, L.logP, L.S, p->N, 3, p->dsti_tw, p->dsti_sn, p->dsti_g, p->st,
                             p->dsti_g ? nullptr : &f);
        launch_dsti_plane<T>(W1, 3, p->n, L.logP, L.S, p->N, 2, p->dsti_tw, p->dsti_sn, nullptr, p->st, nullptr);
      }
      return W1;
    }
    // x, (y,) the last axis forward-scale-inverse, (y,) x: S_x S_y S_z diag(g) S_z S_y S_x
    const int last = p->dim - 1;
    launch_dsti_rows<T>(W1, p->dim, p->n, L.logP, L.S, p->N, p->dsti_tw, p->dsti_sn, p->st);
    if (p->dim == 3)
      launch_dsti_cols<T>(W1, p->dim, p->n, L.logP, L.S, p->N, 1, p->dsti_tw, p->dsti_sn, p->dsti_g, false,
                          p->st);
    launch_dsti_cols<T>(W1, p->dim, p->n, L.logP, L.S, p->N, last, p->dsti_tw, p->dsti_sn, p->dsti_g, true,
                        p->st, p->dsti_g ? nullptr : &f);
    if (p->dim == 3)
      launch_dsti_cols<T>(W1, p->dim, p->n, L.logP, L.S, p->N, 1, p->dsti_tw, p->dsti_sn, p->dsti_g, false,
                          p->st);
    launch_dsti_rows<T>(W1, p->dim, p->n, L.logP, L.S, p->N, p->dsti_tw, p->dsti_sn, p->st);
    return W1;
  }
  apply_Hk_solve<T>(p, W1, W2, done);
  launch_apply_A_scaled<T>(W2, W1, geom<T>(p, 0), (T)p->cthbar, (T)(2.0 * p->tau / p->N), p->N, done,
                           p->st);
  apply_Hk_solve<T>(p, W1, W2, done);
  return W2;
}

// One Uzawa iteration (§3, eq. 3.1) on the problem's stream; every kernel returns at once when
// the device done flag is set, and the finalize kernel advances the iteration index itself, so
// the same launch sequence serves every iteration (and can be captured into a graph).
template <typename T>
void enqueue_iteration(pt_problem* p) {
  const int* done = &p->state->done;
  const StencilGeom<double> g = geom<double>(p, 0);
  T* W1 = (T*)p->W1;
  T* W2 = (T*)p->W2;
  const DstPlan<T> dp = dst_plan<T>(p);
  if (p->mixed) {
    // iterative refinement: FP64 step (fold + residual) or FP32 step on the corrections
    const Level& L0 = p->lev[0];
    const long long total = L0.S * p->N;
    const StencilGeom<float> gf = geom<float>(p, 0);
    launch_ir_begin(p->state, kOuter, p->st);
    launch_ir_fold(p->u, p->p, p->ir_du, p->ir_dp, total, p->state, p->st);
    if (p->dim == 3 && L0.P >= 32)
      launch_ir_outer_3d(p->u, p->p, p->F, p->ir_R1, p->ir_R2, (float*)W1, p->partials, p->tab_d + L0.tab,
                         p->tab_f + L0.tab, p->cth_d, p->coeff.a0, p->tau, L0.h, p->n, L0.logP, L0.S, p->N,
                         steps_d(p), p->state, p->st);
    else if (p->dim == 2 && L0.P >= 32)
      launch_ir_outer_2d(p->u, p->p, p->F, p->ir_R1, p->ir_R2, (float*)W1, p->partials, p->tab_d + L0.tab,
                         p->tab_f + L0.tab, p->cth_d, p->coeff.a0, p->tau, L0.h, p->n, L0.logP, L0.S, p->N,
                         steps_d(p), p->state, p->st);
    else
      launch_ir_outer(p->u, p->p, p->F, p->ir_R1, p->ir_R2, (float*)W1, p->partials, g, p->cth_d, steps_d(p),
                      p->N, p->state, p->st);
    if (p->dim == 3 && L0.P >= 32)
      launch_ir_inner_3d(p->ir_du, p->ir_dp, p->ir_R1, p->ir_R2, p->ir_bp, (float*)W1, p->partials,
                         p->tab_f + L0.tab, (const float*)p->cthA, p->coeff.a0, p->tau, L0.h, p->n, L0.logP, L0.S,
                         p->N, steps_f(p), p->state, p->st);
    else if (p->dim == 2 && L0.P >= 32)
      launch_ir_inner_2d(p->ir_du, p->ir_dp, p->ir_R1, p->ir_R2, p->ir_bp, (float*)W1, p->partials,
                         p->tab_f + L0.tab, (const float*)p->cthA, p->coeff.a0, p->tau, L0.h, p->n, L0.logP, L0.S,
                         p->N, steps_f(p), p->state, p->st);
    else
      launch_ir_inner(p->ir_du, p->ir_dp, p->ir_R1, p->ir_R2, p->ir_bp, (float*)W1, p->partials, gf,
                      (const float*)p->cthA, steps_f(p), p->N, p->state, p->st);
    launch_ir_finalize(p->partials, p->state, p->hist, p->st);
    apply_precond_A<T>(p, W1, p->ir_dp, 1, 0, done);
    launch_ir_resid_u(p->ir_bp, p->ir_R2, p->ir_du, p->ir_dp, (float*)W1, L0.S, p->N, p->state, p->st);
    launch_dst_forward<T>(W1, L0.S, p->dim, p->n, L0.logP, dp, done, p->st);
    T* yhat = block_solve<T>(p, done);
    launch_dst_inverse<T>(yhat, p->ir_du, 2, p->omega, L0.S, p->dim, p->n, L0.logP, dp, done, p->st);
    return;
  }
  if (p->bres && p->dim == 2 && p->lev[0].P >= 32) {
    // outer residual first (and the convergence test), then the p-update and the stencil-free r_u
    const Level& L0 = p->lev[0];
    launch_resid_bres_2d<T>(p->u, p->p, p->F, p->bres, W1, p->partials, p->tab_d + L0.tab, p->tab_f + L0.tab,
                            p->cth_d, p->coeff.a0, p->tau, L0.h, p->n, L0.logP, L0.S, p->N, done,
                            (const double*)p->jinvA[0], steps_d(p), p->st);
    launch_finalize_residual(p->partials, p->state, p->hist, p->st);
    apply_precond_A<T>(p, W1, p->p, 1, 1, done);
    launch_resid_u_from_bres<T>(p->bres, p->u, p->p, W1, L0.S, p->N, p->dim, p->n, done, p->st);
  } else if (p->mixed) {
    // outer residual in FP64 first (and the convergence test), then the p-update and r_u
    launch_resid_bres_mixed(p->u, p->p, p->F, p->bres, (float*)W1, p->partials, g, p->cth_d, steps_d(p), p->N,
                            done, p->st);
    launch_finalize_residual(p->partials, p->state, p->hist, p->st);
    apply_precond_A<T>(p, W1, p->p, 1, 1, done);
    launch_resid_u_from_bres<float>(p->bres, p->u, p->p, (float*)W1, p->lev[0].S, p->N, p->dim, p->n, done,
                                    p->st);
  } else {
    launch_resid_p<T>(p->u, p->p, p->F, W1, g, p->cth_d, steps_d(p), p->N, done, p->st);
    apply_precond_A<T>(p, W1, p->p, 1, 1, done);
    launch_resid_u<T>(p->u, p->p, p->F, W1, p->partials, g, p->cth_d, steps_d(p), p->N, done, p->st);
    launch_finalize_residual(p->partials, p->state, p->hist, p->st);
  }
  launch_dst_forward<T>(W1, p->lev[0].S, p->dim, p->n, p->lev[0].logP, dp, done, p->st);
  T* yhat = block_solve<T>(p, done);
  launch_dst_inverse<T>(yhat, p->u, 1, p->omega, p->lev[0].S, p->dim, p->n, p->lev[0].logP, dp, done, p->st);
  (void)W2;
}

void enqueue_iteration_any(pt_problem* p) {
  if (p->mixed)
    enqueue_iteration<float>(p);
  else
    enqueue_iteration<double>(p);
}

// start of a solve: u = p = 0, ||F||^2, counters, tolerance and limit
pt_status enqueue_reset(pt_problem* p, double tol, int max_it) {
  const long long total = p->lev[0].S * p->N;
  PT_CUDA(cudaMemsetAsync(p->u, 0, sizeof(double) * total, p->st));
  PT_CUDA(cudaMemsetAsync(p->p, 0, sizeof(double) * total, p->st));
  if (p->mixed) {
    PT_CUDA(cudaMemsetAsync(p->ir_du, 0, sizeof(float) * total, p->st));
    PT_CUDA(cudaMemsetAsync(p->ir_dp, 0, sizeof(float) * total, p->st));
  }
  launch_norm2_partials(p->F, total, p->partials, p->st);
  launch_finalize_fnorm(p->partials, p->state, tol, max_it, p->st);
  PT_CHECK_LAUNCH();
  return PT_OK;
}

void drop_graph(pt_problem* p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->graph_exec = nullptr;
  p->graph = nullptr;
  p->graph_iters = 0;
}

// Capture `iters` consecutive iterations into a graph (on an internal stream).
pt_status ensure_graph(pt_problem* p, int iters) {
  if (p->graph_exec && p->graph_iters == iters && p->graph_hist == p->hist && p->graph_dstC == p->dstC &&
      p->graph_lc == p->lc)
    return PT_OK;
  drop_graph(p);
  if (!p->cap) PT_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
  cudaStream_t saved = p->st;
  p->st = p->cap;
  capture_begin();
  cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < iters; ++k) enqueue_iteration_any(p);
    e = cudaStreamEndCapture(p->cap, &p->graph);
  }
  p->graph_kernels = capture_end();
  p->st = saved;
  if (e != cudaSuccess) {
    cudaGetLastError();
    drop_graph(p);
    return fail(PT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  PT_CUDA(cudaGraphInstantiate(&p->graph_exec, p->graph, 0));
  p->graph_iters = iters;
  p->graph_hist = p->hist;
  p->graph_dstC = p->dstC;
  p->graph_lc = p->lc;
  return PT_OK;
}

pt_status ensure_hist(pt_problem* p, int max_it) {
  if (max_it + 1 > p->hist_cap) {
    pt_status st = PT_OK;
    if (!(p->hist = (double*)alloc_bytes(p, sizeof(double) * (max_it + 1), &st))) return st;
    p->hist_cap = max_it + 1;
  }
  return PT_OK;
}

pt_status read_state(pt_problem* p, SolveState* out) {
  PT_CUDA(cudaMemcpyAsync(p->host_state, p->state, sizeof(SolveState), cudaMemcpyDeviceToHost, p->st));
  PT_CUDA(cudaStreamSynchronize(p->st));
  *out = *p->host_state;
  return PT_OK;
}

pt_status finish_solve(pt_problem* p, int* iters_out, double* res_hist) {
  SolveState hs;
  pt_status st = read_state(p, &hs);
  if (st != PT_OK) return st;
  if (hs.done != 1) return fail(PT_ECUDA, "solver state not finalised");
  if (iters_out) *iters_out = hs.iters;
  if (res_hist) {
    PT_CUDA(cudaMemcpyAsync(res_hist, p->hist, sizeof(double) * (hs.iters + 1), cudaMemcpyDeviceToHost, p->st));
    PT_CUDA(cudaStreamSynchronize(p->st));
  }
  if (hs.status == PT_ENOTCONV) g_err = "max_it reached before tol";
  if (hs.status == PT_EDIVERGED) g_err = "residual became non-finite";
  return (pt_status)hs.status;
}

long long padded_total(const pt_problem* p) { return p->lev[0].S * p->N; }

// Iterations per captured graph: small problems take 8 per launch, so that in a shared launch
// (batch or server) they advance several iterations while a large problem does one.
int graph_iterations(const pt_problem* p) { return padded_total(p) >= (1LL << 22) ? 1 : 8; }

pt_status uzawa(pt_problem* p, double tol, int max_it, int* iters_out, double* res_hist) {
  pt_status st = enqueue_reset(p, tol, max_it);
  if (st != PT_OK) return st;
  const long long total = padded_total(p);
  const bool small = total < (1LL << 22);
  int check = p->opt.check_every;
  if (check <= 0) check = small ? 8 : 1;
  const bool profiling = profiling_enabled();
  const bool graphs = !p->opt.no_graphs && !profiling;
  // kernels timed one by one: poll every iteration so that the scopes of the refinement kernels
  // know which kind of iteration comes next (the first one is the FP64 step, j = 0)
  if (profiling) check = 1;
  struct StepKindReset {
    ~StepKindReset() { set_step_kind(kAnyStep); }
  } reset_kind;
  if (profiling && p->mixed) set_step_kind(kOuterStep);
  const int per_launch = graphs ? std::min(check, graph_iterations(p)) : 1;
  if (graphs && (st = ensure_graph(p, per_launch)) != PT_OK) return st;
  long long launched = 0, since_poll = 0;
  for (;;) {
    if (graphs) {
      PT_CUDA(cudaGraphLaunch(p->graph_exec, p->st));
      note_launch((int)p->graph_kernels);
    } else {
      enqueue_iteration_any(p);
      PT_CHECK_LAUNCH();
    }
    launched += per_launch;
    since_poll += per_launch;
    if (since_poll >= check || launched > max_it) {
      since_poll = 0;
      SolveState hs;
      if ((st = read_state(p, &hs)) != PT_OK) return st;
      if (hs.done == 1) break;
      if (profiling && p->mixed) set_step_kind((hs.done == 2 || hs.j % kOuter == 0) ? kOuterStep : kInnerStep);
      // (the mixed form may take one extra launch: the FP64 step that confirms the last estimate)
      if (launched > (long long)max_it + 2 * per_launch + 2) return fail(PT_ECUDA, "solver did not stop at max_it");
    }
  }
  return finish_solve(p, iters_out, res_hist);
}

// ---- Krylov acceleration: flexible GMRES(m) preconditioned by one inexact Uzawa step --------
// Solves Sad (p, u) = (F, F) (the system the Uzawa iteration of eq. 3.1 solves) with the right
// preconditioner M^-1 (v_p, v_u) = (-A~^-1 v_p, H~^-1 (v_u - K^T z_p)): the block lower-triangular
// M = [-A~, 0; K^T, H~] of the Uzawa step with omega = 1.  Classical Gram-Schmidt with selective
// reorthogonalisation, Givens rotations on the host.  The history holds the preconditioned saddle-point residual
// relative to ||(F, F)||; a cycle ends when it reaches the tolerance, and the solve ends only when
// ||F - B u|| / ||F|| of the updated u (computed in FP64) does, else it restarts with a tenfold
// smaller inner target.

pt_status krylov_alloc(pt_problem* p, int m) {
  if (p->kr_m == m) return PT_OK;
  if (p->kr_m != 0) return fail(PT_EINVAL, "the Krylov restart length of a problem cannot change");
  pt_status st = PT_OK;
  const Level& L0 = p->lev[0];
  auto vec = [&]() -> double* { return alloc_padded<double>(p, L0, p->N, &st); };
  for (int k = 0; k <= m; ++k) {
    double* a = vec();
    double* b = a ? vec() : nullptr;
    if (!b) return st;
    p->kr_vp.push_back(a);
    p->kr_vu.push_back(b);
  }
  for (int k = 0; k < m; ++k) {
    double* a = vec();
    double* b = a ? vec() : nullptr;
    if (!b) return st;
    p->kr_zp.push_back(a);
    p->kr_zu.push_back(b);
  }
  if (!(p->kr_wp = vec()) || !(p->kr_wu = vec())) return st;
  if (p->bres && !(p->kr_zero = vec())) return st;
  std::vector<double*> tab;
  tab.insert(tab.end(), p->kr_vp.begin(), p->kr_vp.end());
  tab.insert(tab.end(), p->kr_vu.begin(), p->kr_vu.end());
  tab.insert(tab.end(), p->kr_zp.begin(), p->kr_zp.end());
  tab.insert(tab.end(), p->kr_zu.begin(), p->kr_zu.end());
  if (!(p->kr_tab = (double**)alloc_bytes(p, sizeof(double*) * tab.size(), &st))) return st;
  PT_CUDA(cudaMemcpyAsync(p->kr_tab, tab.data(), sizeof(double*) * tab.size(), cudaMemcpyHostToDevice, p->st));
  if (!(p->kr_coef = (double*)alloc_bytes(p, sizeof(double) * (m + 1), &st))) return st;
  if (!(p->kr_part = (double*)alloc_bytes(p, sizeof(double) * (m + 2) * kReduceBlocks, &st))) return st;
  p->kr_m = m;
  return PT_OK;
}

// dots <w, v_k>, first <= k < first + nv, and with self <w, w> last (host result, fixed order)
pt_status krylov_dots(pt_problem* p, int nv, const double* wp, const double* wu, std::vector<double>& out,
                      int first = 0, int self = 0) {
  const long long total = p->lev[0].S * p->N;
  launch_multidot((const double* const*)(p->kr_tab + first), (const double* const*)(p->kr_tab + p->kr_m + 1 + first),
                  wp, wu, nv, self, total, p->kr_part, p->st);
  const int rows = nv + (self ? 1 : 0);
  std::vector<double> part((size_t)rows * kReduceBlocks);
  PT_CUDA(cudaMemcpyAsync(part.data(), p->kr_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, p->st));
  PT_CUDA(cudaStreamSynchronize(p->st));
  out.assign(rows, 0.0);
  for (int k = 0; k < rows; ++k)
    for (int b = 0; b < kReduceBlocks; ++b) out[k] += part[(size_t)k * kReduceBlocks + b];
  return PT_OK;
}

// (wp, wu) += sum_k c_k x_k over the table rows [first, first + nv) (vp) and the matching u rows
pt_status krylov_axpy(pt_problem* p, int first_p, int first_u, const std::vector<double>& c, double* wp,
                      double* wu) {
  const long long total = p->lev[0].S * p->N;
  PT_CUDA(cudaMemcpyAsync(p->kr_coef, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice, p->st));
  launch_multiaxpy((const double* const*)(p->kr_tab + first_p), (const double* const*)(p->kr_tab + first_u),
                   p->kr_coef, (int)c.size(), wp, wu, total, p->st);
  PT_CHECK_LAUNCH();
  return PT_OK;
}

// ||F - B u||^2 / ||F||^2 of the current u (FP64): the r_u kernel's partial sums
pt_status krylov_true_residual(pt_problem* p, double* res) {
  const StencilGeom<double> g = geom<double>(p, 0);
  launch_resid_u<double>(p->u, p->p, p->F, (double*)p->W2, p->partials, g, p->cth_d, steps_d(p), p->N, nullptr,
                         p->st);
  std::vector<double> part(kReduceBlocks);
  PT_CUDA(cudaMemcpyAsync(part.data(), p->partials, sizeof(double) * kReduceBlocks, cudaMemcpyDeviceToHost, p->st));
  SolveState hs;
  pt_status st = read_state(p, &hs);
  if (st != PT_OK) return st;
  double s = 0.0;
  for (double v : part) s += v;
  *res = std::sqrt(s / hs.fnorm2);
  return PT_OK;
}

// (op, ou) = Sad (zp, zu).  2-D FP64 (stored-residual path): with F = 0 the outer-residual kernel
// gives bres = -B z_u and op = -bres - tau_n A (z_p + z_u) = K z_u - tau_n A z_p (no rho_n scaling:
// a null rho), and the second residual kernel sgn (bres - K^T (z_p + z_u)) with sgn = -1 gives ou.
void krylov_apply(pt_problem* p, const double* zp, const double* zu, double* op, double* ou) {
  const Level& L0 = p->lev[0];
  const Steps<double> sp = steps_d(p);
  if (p->kr_zero) {
    launch_resid_bres_2d<double>(zu, zp, p->kr_zero, p->bres, op, p->partials, p->tab_d + L0.tab,
                                 p->tab_f + L0.tab, p->cth_d, p->coeff.a0, p->tau, L0.h, p->n, L0.logP, L0.S, p->N,
                                 nullptr, (const double*)p->jinvA[0], {sp.tau, sp.sig, nullptr, sp.uniform}, p->st);
    launch_resid_u_from_bres<double>(p->bres, zu, zp, ou, L0.S, p->N, p->dim, p->n, nullptr, p->st, -1.0);
  } else {
    launch_apply_saddle(zp, zu, op, ou, geom<double>(p, 0), p->cth_d, sp, p->N, p->st);
  }
}

// z = M^-1 v for the pair k of the table
void krylov_precondition(pt_problem* p, int k) {
  const Level& L0 = p->lev[0];
  double* vp = p->kr_vp[k];
  double* vu = p->kr_vu[k];
  double* zp = p->kr_zp[k];
  double* zu = p->kr_zu[k];
  double* a = (double*)p->W2;
  double* W1 = (double*)p->W1;
  apply_precond_A<double>(p, vp, a, 0, 1, nullptr);  // a = V-cycles for tau A_n on v_p
  // z_p = -rho_n a = -A~^-1 v_p for tau_n A_n (both halves: same buffers)
  launch_scale_pair(a, a, -1.0, zp, zp, L0.S * p->N, p->st, steps_d(p).rho, L0.logP * p->dim);
  launch_uzawa_ru(vu, zp, W1, L0.S, p->N, p->st);             // W1 = v_u - K^T z_p
  const DstPlan<double> dp = dst_plan<double>(p);
  launch_dst_forward<double>(W1, L0.S, p->dim, p->n, L0.logP, dp, nullptr, p->st);
  double* yhat = block_solve<double>(p, nullptr);
  cudaMemsetAsync(zu, 0, sizeof(double) * L0.S * p->N, p->st);
  launch_dst_inverse<double>(yhat, zu, 1, 1.0, L0.S, p->dim, p->n, L0.logP, dp, nullptr, p->st);
}

pt_status krylov_solve(pt_problem* p, double tol, int max_it, int* iters_out, double* res_hist) {
  const int m = p->opt.krylov;
  pt_status st = krylov_alloc(p, m);
  if (st != PT_OK) return st;
  if ((st = enqueue_reset(p, tol, max_it)) != PT_OK) return st;  // u = p = 0, ||F||^2
  const long long total = p->lev[0].S * p->N;
  const StencilGeom<double> g = geom<double>(p, 0);
  double* xp = p->p;
  double* xu = p->u;
  std::vector<double> hist;
  double res_true = 1.0;
  hist.push_back(1.0);
  int it = 0;
  double inner_tol = tol;
  double beta0 = 0.0;
  pt_status out = PT_ENOTCONV;
  std::vector<double> dots, dots2;
  while (it < max_it) {
    // r = (F, F) - Sad x  -> V_0 = r / beta
    krylov_apply(p, xp, xu, p->kr_wp, p->kr_wu);
    launch_scale_pair(p->kr_wp, p->kr_wu, -1.0, p->kr_wp, p->kr_wu, total, p->st);
    {
      // add (F, F): F is not in the table, use it as a one-term sum through the work slot of V_m
      launch_scale_pair(p->F, p->F, 1.0, p->kr_vp[m], p->kr_vu[m], total, p->st);
      if ((st = krylov_axpy(p, m, 2 * m + 1, {1.0}, p->kr_wp, p->kr_wu)) != PT_OK) return st;
    }
    // beta = ||r||
    if ((st = krylov_dots(p, 0, p->kr_wp, p->kr_wu, dots, 0, 1)) != PT_OK) return st;
    const double beta = std::sqrt(std::max(dots[0], 0.0));
    if (beta0 == 0.0) beta0 = beta > 0.0 ? beta : 1.0;
    if (!(beta > 0.0)) {
      out = PT_OK;
      break;
    }
    launch_scale_pair(p->kr_wp, p->kr_wu, 1.0 / beta, p->kr_vp[0], p->kr_vu[0], total, p->st);
    std::vector<std::vector<double>> H(m + 1, std::vector<double>(m, 0.0));
    std::vector<double> cs(m, 0.0), sn(m, 0.0), gv(m + 1, 0.0);
    gv[0] = beta;
    int j = 0;
    for (; j < m && it < max_it; ++j) {
      krylov_precondition(p, j);
      krylov_apply(p, p->kr_zp[j], p->kr_zu[j], p->kr_wp, p->kr_wu);
      // classical Gram-Schmidt with selective reorthogonalisation: the copy of w in V_{j+1} gives
      // ||w|| in the same pass; a second pass only when the projection removed more than half of
      // w's norm squared (Kahan-Parlett "twice is enough")
      double h = 0.0;
      bool exact_norm = true;
      for (int pass = 0; pass < 2; ++pass) {
        if ((st = krylov_dots(p, j + 1, p->kr_wp, p->kr_wu, dots, 0, 1)) != PT_OK) return st;
        const double w2 = std::max(dots[j + 1], 0.0);
        std::vector<double> c(j + 1);
        double proj = 0.0;
        for (int i = 0; i <= j; ++i) {
          H[i][j] += dots[i];
          c[i] = -dots[i];
          proj += dots[i] * dots[i];
        }
        if ((st = krylov_axpy(p, 0, m + 1, c, p->kr_wp, p->kr_wu)) != PT_OK) return st;
        const double rest = w2 - proj;  // ||w - sum h_i v_i||^2 in exact arithmetic
        h = std::sqrt(std::max(rest, 0.0));
        if (rest > 0.5 * w2) {
          exact_norm = false;  // no cancellation: the Pythagorean value is accurate
          break;
        }
      }
      if (exact_norm) {  // two passes and still a large cancellation: measure ||w|| directly
        if ((st = krylov_dots(p, 0, p->kr_wp, p->kr_wu, dots2, 0, 1)) != PT_OK) return st;
        h = std::sqrt(std::max(dots2[0], 0.0));
      }
      H[j + 1][j] = h;
      if (h > 0.0) launch_scale_pair(p->kr_wp, p->kr_wu, 1.0 / h, p->kr_vp[j + 1], p->kr_vu[j + 1], total, p->st);
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i][j] + sn[i] * H[i + 1][j];
        H[i + 1][j] = -sn[i] * H[i][j] + cs[i] * H[i + 1][j];
        H[i][j] = t;
      }
      const double r = std::hypot(H[j][j], H[j + 1][j]);
      cs[j] = r > 0.0 ? H[j][j] / r : 1.0;
      sn[j] = r > 0.0 ? H[j + 1][j] / r : 0.0;
      H[j][j] = r;
      H[j + 1][j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++it;
      const double est = std::fabs(gv[j + 1]) / beta0;
      hist.push_back(est);
      if (!(est <= 1e30)) return fail(PT_EDIVERGED, "Krylov residual became non-finite");
      if (est <= inner_tol || h == 0.0) {
        ++j;
        break;
      }
    }
    // x += Z y, H(0:j, 0:j) y = g(0:j)
    std::vector<double> y(j, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double s = gv[i];
      for (int k = i + 1; k < j; ++k) s -= H[i][k] * y[k];
      y[i] = H[i][i] != 0.0 ? s / H[i][i] : 0.0;
    }
    if (j > 0 && (st = krylov_axpy(p, 2 * m + 2, 3 * m + 2, y, xp, xu)) != PT_OK) return st;
    if ((st = krylov_true_residual(p, &res_true)) != PT_OK) return st;
    hist.back() = res_true;  // the solve's own criterion for the iterate it has now
    if (res_true <= tol) {
      out = PT_OK;
      break;
    }
    inner_tol = std::min(inner_tol, std::fabs(gv[j]) / beta0) * 0.1;
  }
  if (iters_out) *iters_out = it;
  if (res_hist) {
    for (size_t k = 0; k < hist.size() && (int)k <= max_it; ++k) res_hist[k] = hist[k];
  }
  // record the outcome in the device state (iteration count and status), as the Uzawa path does
  SolveState hs;
  if ((st = read_state(p, &hs)) != PT_OK) return st;
  hs.done = 1;
  hs.status = out;
  hs.iters = it;
  hs.last_res = res_true;
  PT_CUDA(cudaMemcpyAsync(p->state, &hs, sizeof(SolveState), cudaMemcpyHostToDevice, p->st));
  PT_CUDA(cudaStreamSynchronize(p->st));
  if (out == PT_ENOTCONV) g_err = "max_it reached before tol";
  return out;
}

// ---- autotuner ------------------------------------------------------------------------
struct TuneChoice {
  int dstC, coarse_elems;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;
bool g_tune_file_loaded = false;

// Problems share a tuning when they have the same grid, precision and solvers and their N_t falls
// in the same power-of-two bucket with the same temporal-transform kind (radix for powers of two,
// Bluestein otherwise): the launch shapes scale alike within a bucket, so a batch or a request
// stream of many N_t tunes once per bucket.
std::string tune_key(const pt_problem* p) {
  long long bucket = 1;
  while (bucket < p->N) bucket <<= 1;
  std::ostringstream k;
  k << "d" << p->dim << "_n" << p->n << "_N" << bucket << (bucket == p->N ? "r" : "b") << "_"
    << (p->mixed ? "mixed" : "fp64") << "_" << (p->exact1d ? "exact" : "mg") << (p->hdst ? "_hdst" : "")
    << (p->mass ? "_p1" : "");
  return k.str();
}

// temporal-transform columns per CTA (0: automatic) that fit this problem's shared memory and slice
std::vector<int> tune_cols(const pt_problem* p) {
  std::vector<int> cols = {0};
  for (int c = 1; c <= 16; c *= 2) {
    const long long L = p->blueM > 0 ? p->blueM + 1 : p->N + 1;
    const long long bytes = (long long)c * L * 2 * (p->mixed ? 4 : 8) * 2;
    if (p->lev[0].S % (2 * c) == 0 && bytes <= 200 * 1024 && 2 * c <= p->lev[0].S) cols.push_back(c);
  }
  return cols;
}

void tune_file_load() {
  if (g_tune_file_loaded) return;
  g_tune_file_loaded = true;
  const char* path = std::getenv("PT_TUNE_CACHE");
  if (!path) return;
  std::ifstream in(path);
  std::string line;
  // one entry per line: "key": [dstC, coarse_elems],
  while (std::getline(in, line)) {
    const size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1), b0 = line.find('['), c = line.find(',', b0),
                 b1 = line.find(']', b0);
    if (q0 == std::string::npos || q1 == std::string::npos || b0 == std::string::npos || c == std::string::npos ||
        b1 == std::string::npos)
      continue;
    TuneChoice t;
    t.dstC = std::atoi(line.substr(b0 + 1, c - b0 - 1).c_str());
    t.coarse_elems = std::atoi(line.substr(c + 1, b1 - c - 1).c_str());
    g_tune_cache[line.substr(q0 + 1, q1 - q0 - 1)] = t;
  }
}

void tune_file_save() {
  const char* path = std::getenv("PT_TUNE_CACHE");
  if (!path) return;
  std::ofstream out(path);
  out << "{\n";
  size_t i = 0;
  for (auto& kv : g_tune_cache)
    out << "  \"" << kv.first << "\": [" << kv.second.dstC << ", " << kv.second.coarse_elems << "]"
        << (++i < g_tune_cache.size() ? "," : "") << "\n";
  out << "}\n";
}

int lc_for(const pt_problem* p, int elems) {
  for (int l = 0; l < p->nlev; ++l)
    if (p->lev[l].S <= elems) return l;
  return p->nlev - 1;
}

void apply_choice(pt_problem* p, TuneChoice t) {
  // a choice tuned on another problem of the bucket: the largest valid column count <= its own
  const std::vector<int> cols = tune_cols(p);
  int c = 0;
  for (int v : cols)
    if (v <= t.dstC) c = std::max(c, v);
  t.dstC = c;
  p->dstC = t.dstC;
  p->coarse_elems = t.coarse_elems;
  p->lc = std::min(std::max(lc_for(p, t.coarse_elems), p->lc_min), p->lc_max);
}

// Time a few iterations of each candidate (transform tile width x coarse-level split) on the
// problem's own data and keep the fastest.  The numbers produced do not depend on the choice
// beyond rounding (columns are independent in the transform; the coarse split only moves levels
// between kernels), and the solve that follows starts from zero again.
pt_status autotune(pt_problem* p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_file_load();
  const std::string key = tune_key(p);
  auto it = g_tune_cache.find(key);
  if (it != g_tune_cache.end()) {
    apply_choice(p, it->second);
    p->tuned = true;
    return PT_OK;
  }
  const std::vector<int> cols = tune_cols(p);
  std::vector<int> coarse = {kCoarseMaxElems};
  if (!p->exact1d)
    for (int e : {256, 4096})
      if (lc_for(p, e) >= p->lc_min && lc_for(p, e) <= p->lc_max && lc_for(p, e) != lc_for(p, kCoarseMaxElems))
        coarse.push_back(e);
  pt_status st = ensure_hist(p, 1 << 20);
  if (st != PT_OK) return st;
  cudaEvent_t e0, e1;
  PT_CUDA(cudaEventCreate(&e0));
  PT_CUDA(cudaEventCreate(&e1));
  TuneChoice best{0, kCoarseMaxElems};
  float best_ms = 1e30f;
  for (int ce : coarse) {
    for (int c : cols) {
      apply_choice(p, TuneChoice{c, ce});
      if ((st = enqueue_reset(p, 0.0, 1 << 20)) != PT_OK) break;
      enqueue_iteration_any(p);
      PT_CUDA(cudaEventRecord(e0, p->st));
      for (int k = 0; k < 2; ++k) enqueue_iteration_any(p);
      PT_CUDA(cudaEventRecord(e1, p->st));
      PT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      PT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = TuneChoice{c, ce};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PT_OK) return st;
  apply_choice(p, best);
  g_tune_cache[key] = best;
  tune_file_save();
  p->tuned = true;
  return PT_OK;
}

bool is_pow2(long long v) { return v >= 1 && (v & (v - 1)) == 0; }
int ilog2(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

pt_status validate(const pt_grid* grid, int N_t, double T, const pt_coeff* coeff, const pt_options* o) {
  if (!grid || !coeff) return fail(PT_EINVAL, "grid and coeff are required");
  if (grid->dim < 1 || grid->dim > 3) return fail(PT_EINVAL, "dim must be 1, 2 or 3");
  for (int d = 0; d < grid->dim; ++d) {
    if (grid->n[d] != grid->n[0]) return fail(PT_EINVAL, "all axes must have the same n");
    if (grid->n[d] < 1 || !is_pow2((long long)grid->n[d] + 1))
      return fail(PT_EINVAL, "n + 1 must be a power of two >= 2");
  }
  if (grid->n[0] > 32767) return fail(PT_EINVAL, "n too large");
  if (N_t < 1 || N_t > 8192) return fail(PT_EINVAL, "N_t must be in [1, 8192]");
  if (!is_pow2(N_t)) {
    const int fp64 = !o || o->precision == PT_PREC_FP64;
    if (N_t > (fp64 ? 2048 : 4096))
      return fail(PT_EINVAL, "N_t that is not a power of two must be <= 2048 (FP64) or 4096 (mixed)");
  }
  if (!(T > 0.0) || !std::isfinite(T)) return fail(PT_EINVAL, "T must be positive");
  if (!std::isfinite(coeff->a0) || !std::isfinite(coeff->c)) return fail(PT_EINVAL, "non-finite coefficient");
  if (std::fabs(coeff->c) >= coeff->a0) return fail(PT_EINVAL, "need |c| < a0 so that a > 0");
  for (int d = 0; d < 3; ++d)
    if (coeff->fx[d] < 0 || coeff->fx[d] > 2) return fail(PT_EINVAL, "fx must be a pt_trig");
  if (coeff->ft < 0 || coeff->ft > 2) return fail(PT_EINVAL, "ft must be a pt_trig");
  if (o) {
    if (o->precision != PT_PREC_FP64 && o->precision != PT_PREC_MIXED) return fail(PT_EINVAL, "bad precision");
    if (o->spatial_solver != PT_SOLVER_MG && o->spatial_solver != PT_SOLVER_EXACT_1D)
      return fail(PT_EINVAL, "bad spatial_solver");
    if (o->spatial_solver == PT_SOLVER_EXACT_1D && grid->dim != 1)
      return fail(PT_EINVAL, "exact spatial solves are available in 1-D only");
    if (o->n_vcycles < 0 || o->n_vcycles > 4) return fail(PT_EINVAL, "n_vcycles must be in [0, 4]");
    if (o->mass != 0 && o->mass != 1) return fail(PT_EINVAL, "mass must be 0 (identity) or 1 (P1)");
    if (o->mass == 1) {
      if (grid->dim > 2) return fail(PT_EINVAL, "the P1 mass matrix is available in 1-D and 2-D");
      if (o->precision != PT_PREC_FP64) return fail(PT_EINVAL, "the P1 mass matrix is FP64 only");
      if (o->krylov != 0) return fail(PT_EINVAL, "the P1 mass matrix is not available with krylov");
      if (grid->dim == 2 && o->h_solver == 2)
        return fail(PT_EINVAL, "exact H_k solves are not available with the 2-D P1 mass");
    }
    if (o->krylov < 0 || o->krylov > 64) return fail(PT_EINVAL, "krylov must be in [0, 64]");
    if (o->tau_steps) {
      double sum = 0.0;
      for (int i = 0; i < N_t; ++i) {
        const double v = o->tau_steps[i];
        if (!(v > 0.0) || !std::isfinite(v)) return fail(PT_EINVAL, "time steps must be finite and positive");
        sum += v;
      }
      if (!(std::fabs(sum - T) <= 1e-10 * T)) return fail(PT_EINVAL, "the time steps must sum to T");
    }
    if (o->krylov > 0 && o->precision != PT_PREC_FP64)
      return fail(PT_EINVAL, "the Krylov-accelerated solve is FP64 only");
    if (o->h_solver < 0 || o->h_solver > 2) return fail(PT_EINVAL, "h_solver must be 0, 1 or 2");
    if (o->dst_cols != 0 && (o->dst_cols < 0 || o->dst_cols > 16 || !is_pow2(o->dst_cols)))
      return fail(PT_EINVAL, "dst_cols must be 0 or a power of two <= 16");
    if (o->coarse_elems != 0 && (o->coarse_elems < 64 || o->coarse_elems > 4096 || !is_pow2(o->coarse_elems)))
      return fail(PT_EINVAL, "coarse_elems must be 0 or a power of two in [64, 4096]");
  }
  return PT_OK;
}

template <typename T>
pt_status setup_precision(pt_problem* p) {
  pt_status st = PT_OK;
  const Level& L0 = p->lev[0];
  p->W1 = alloc_padded<T>(p, L0, p->N, &st);
  if (!p->W1) return st;
  p->W2 = alloc_padded<T>(p, L0, p->N, &st);
  if (!p->W2) return st;
  if (!p->exact1d && p->nv_h > 1) {
    p->W3 = alloc_padded<T>(p, L0, p->N, &st);
    if (!p->W3) return st;
  }
  if (!p->exact1d) {
    // fused 2-D kernels keep no level-0 iterate and no residuals; with the P1 mass the H_k
    // V-cycles run on the generic level kernels, which do
    const bool fused = p->dim == 2 && !p->mass;
    for (int l = 0; l <= p->lc_max && l < p->nlev; ++l) {
      if (l > 0) {
        p->mg_b[l] = alloc_padded<T>(p, p->lev[l], p->N, &st);
        if (!p->mg_b[l]) return st;
      }
      if (!fused || l > 0) {
        p->mg_x[l] = alloc_padded<T>(p, p->lev[l], p->N, &st);
        if (!p->mg_x[l]) return st;
      }
      if (!fused && l < p->lc_max) {
        p->mg_r[l] = alloc_padded<T>(p, p->lev[l], p->N, &st);
        if (!p->mg_r[l]) return st;
      }
    }
  } else {
    p->tri_work = alloc_bytes(p, sizeof(T) * 2 * (size_t)L0.P * p->N, &st);
    if (!p->tri_work) return st;
  }
  // per-slice operator parameters
  std::vector<double> zeros(p->N, 0.0), cthA(p->N), mu(p->N), cthH(p->N, p->cthbar);
  for (int i = 0; i < p->N; ++i) {
    cthA[i] = p->coeff.c * trig(p->coeff.ft, M_PI * p->coeff.mt * p->tn[i]);
    mu[i] = 2.0 * std::sin((2.0 * (i + 1) - 1.0) * M_PI / (4.0 * p->N));
  }
  const size_t nb = sizeof(T) * p->N;
  if (!(p->sigA = alloc_bytes(p, nb, &st))) return st;
  if (!(p->cthA = alloc_bytes(p, nb, &st))) return st;
  if (!(p->sigH = alloc_bytes(p, nb, &st))) return st;
  if (!(p->cthH = alloc_bytes(p, nb, &st))) return st;
  if ((st = upload<T>(p, p->sigA, zeros)) != PT_OK) return st;
  if ((st = upload<T>(p, p->cthA, cthA)) != PT_OK) return st;
  if ((st = upload<T>(p, p->sigH, mu)) != PT_OK) return st;
  if ((st = upload<T>(p, p->cthH, cthH)) != PT_OK) return st;
  // Abar with a constant coefficient: its Jacobi factor w / (mu_k + 2 dim tau a0 / h^2) per level
  p->hvar = !(std::fabs(p->cthbar) <= 1e-14 * std::fabs(p->coeff.a0));
  if (!p->exact1d && p->dim == 2 && !p->hvar && !p->mass) {
    for (int l = 0; l < p->lc_max; ++l) {
      std::vector<double> dv(p->N);
      const double a0s = p->tau * p->coeff.a0 / (p->lev[l].h * p->lev[l].h);
      for (int k = 0; k < p->N; ++k) dv[k] = p->jacobi / (mu[k] + 2.0 * p->dim * a0s);
      if (!(p->dinvH[l] = alloc_bytes(p, nb, &st))) return st;
      if ((st = upload<T>(p, p->dinvH[l], dv)) != PT_OK) return st;
    }
  }
  // exact H_k solves by spatial sine transforms (constant reference coefficient, 2-D and 3-D)
  // (not with the 2-D P1 mass: its diagonal coupling is not diagonalised by the sine transforms)
  p->hdst = !p->exact1d && p->dim >= 2 && !p->hvar && p->opt.h_solver != 1 && p->n + 1 <= kDstiMaxM && !p->mass;
  if (p->hdst) {
    const int M = p->n + 1;
    std::vector<double> tw(2 * M), sn(M / 2 + 1), lam(M, 0.0), mud(mu.begin(), mu.end());
    for (int e = 0; e < M; ++e) {
      tw[2 * e] = std::cos(2.0 * M_PI * e / M);  // e^{-2 pi i e / M}
      tw[2 * e + 1] = -std::sin(2.0 * M_PI * e / M);
    }
    for (int j = 0; j <= M / 2; ++j) sn[j] = 0.5 * std::sin(M_PI * j / M);
    const double h = 1.0 / M;
    for (int k = 1; k <= p->n; ++k) {
      const double s = std::sin(M_PI * k * h / 2.0);
      lam[k - 1] = 4.0 * p->coeff.a0 / (h * h) * s * s;
    }
    if (!(p->dsti_tw = alloc_bytes(p, sizeof(T) * tw.size(), &st))) return st;
    if (!(p->dsti_sn = alloc_bytes(p, sizeof(T) * sn.size(), &st))) return st;
    if (!(p->dsti_lam = (double*)alloc_bytes(p, sizeof(double) * lam.size(), &st))) return st;
    if (!(p->dsti_mu = (double*)alloc_bytes(p, sizeof(double) * mud.size(), &st))) return st;
    if ((st = upload<T>(p, p->dsti_tw, tw)) != PT_OK) return st;
    if ((st = upload<T>(p, p->dsti_sn, sn)) != PT_OK) return st;
    if ((st = upload<double>(p, p->dsti_lam, lam)) != PT_OK) return st;
    if ((st = upload<double>(p, p->dsti_mu, mud)) != PT_OK) return st;
    const Level& L = p->lev[0];
    if (p->dim == 2 && sizeof(T) == 8) {
      // FP64 2-D: x by transforms, y by tridiagonal eliminations (fewer FP64 operations; their
      // relative error ~ cond(T_k) eps64 <= 1e-9 for n + 1 <= 4096.  In FP32 cond(T_k) eps32 would
      // reach 1e-3 at 255^2, so the FP32 form keeps the transforms, exact to ~eps32 log n.)
      T* w = alloc_padded<T>(p, L, p->N, &st);
      if (!w) return st;
      p->hy_w = w;
      launch_hsolve_trid_table<T>(w, p->dsti_lam, p->dsti_mu, p->tau, p->coeff.a0 / (L.h * L.h), p->n, L.logP,
                                  L.S, p->N, p->st);
    } else if (sizeof(T) == 4) {
      // FP32: the factor is formed per point in the column kernel from lam and mu_k / tau in FP32
      std::vector<double> m(mud);
      for (double& v : m) v /= p->tau;
      if (!(p->dsti_lamT = alloc_bytes(p, sizeof(T) * lam.size(), &st))) return st;
      if (!(p->dsti_muT = alloc_bytes(p, sizeof(T) * m.size(), &st))) return st;
      if ((st = upload<T>(p, p->dsti_lamT, lam)) != PT_OK) return st;
      if ((st = upload<T>(p, p->dsti_muT, m)) != PT_OK) return st;
    } else {
      // the point-wise block-solve factor, computed once in FP64 (c0 as in block_solve)
      const double c0 = (2.0 * p->tau / p->N) * std::pow(2.0 / L.P, p->dim);
      T* g = alloc_padded<T>(p, L, p->N, &st);
      if (!g) return st;
      p->dsti_g = g;
      launch_dsti_scale_table<T>(g, p->dsti_lam, p->dsti_mu, p->tau, c0, p->dim, L.logP, L.S, p->N, p->st);
    }
  } else if (p->opt.h_solver == 2) {
    return fail(PT_EINVAL,
                "exact H_k solves need dim >= 2, n + 1 <= 4096 and a reference coefficient constant in space");
  }
  // FP64 2-D: cache (w / D, D) of every tau A_n (a division per point per smoothing step, and
  // four FP64 operations per stencil, otherwise)
  if (!p->exact1d && p->dim == 2 && sizeof(T) == 8) {
    for (int l = 0; l < p->lc_max; ++l) {
      T* j = alloc_padded<T>(p, p->lev[l], 2 * p->N, &st);  // pairs (w / D, D)
      if (!j) return st;
      p->jinvA[l] = j;
      launch_make_jinv<T>(j, geom<T>(p, l), op_A<T>(p), p->N, p->st);
    }
  }
  // DST tables: twiddles e^{2 pi i k/N}, k < N/2, and e^{i pi m/(2N)}, m < N
  std::vector<double> tw(2 * std::max(1, p->N / 2)), pre(2 * p->N);
  for (int k = 0; k < p->N / 2; ++k) {
    tw[2 * k] = std::cos(2.0 * M_PI * k / p->N);
    tw[2 * k + 1] = std::sin(2.0 * M_PI * k / p->N);
  }
  if (p->N == 1) {
    tw[0] = 1.0;
    tw[1] = 0.0;
  }
  for (int m = 0; m < p->N; ++m) {
    pre[2 * m] = std::cos(M_PI * m / (2.0 * p->N));
    pre[2 * m + 1] = std::sin(M_PI * m / (2.0 * p->N));
  }
  if (!(p->dst_tw = alloc_bytes(p, sizeof(T) * tw.size(), &st))) return st;
  if (!(p->dst_pre = alloc_bytes(p, sizeof(T) * pre.size(), &st))) return st;
  if ((st = upload<T>(p, p->dst_tw, tw)) != PT_OK) return st;
  if ((st = upload<T>(p, p->dst_pre, pre)) != PT_OK) return st;
  if (is_pow2(p->N)) {
    std::vector<double> tws(2 * p->N);
    for (int e = 0; e < p->N; ++e) {
      tws[2 * e] = std::cos(2.0 * M_PI * e / p->N);  // e^{-2 pi i e / N}
      tws[2 * e + 1] = -std::sin(2.0 * M_PI * e / p->N);
    }
    if (!(p->dst_twS = alloc_bytes(p, sizeof(T) * tws.size(), &st))) return st;
    if ((st = upload<T>(p, p->dst_twS, tws)) != PT_OK) return st;
  }
  if (!is_pow2(p->N)) {
    // Bluestein: chirp c_m = e^{i pi m^2 / N} (phase reduced mod 2N), filters g with g_m = g_{M-m}
    // = c_m (e^{-} DFT) or conj(c_m) (e^{+} DFT), their M-point spectra in bit-reversed order / M
    const int N = p->N, M = p->blueM, logM = p->blueLogM;
    std::vector<double> chirp(2 * N), twm(2 * (M / 2)), gf(2 * M), gi(2 * M);
    for (int m = 0; m < N; ++m) {
      const long long q = ((long long)m * m) % (2LL * N);
      chirp[2 * m] = std::cos(M_PI * (double)q / N);
      chirp[2 * m + 1] = std::sin(M_PI * (double)q / N);
    }
    for (int k = 0; k < M / 2; ++k) {
      twm[2 * k] = std::cos(2.0 * M_PI * k / M);
      twm[2 * k + 1] = std::sin(2.0 * M_PI * k / M);
    }
    for (int sgn = 0; sgn < 2; ++sgn) {
      std::vector<double> re(M, 0.0), im(M, 0.0);
      for (int m = 0; m < N; ++m) {
        const double cr = chirp[2 * m], ci = sgn == 0 ? chirp[2 * m + 1] : -chirp[2 * m + 1];
        re[m] = cr;
        im[m] = ci;
        if (m > 0) {
          re[M - m] = cr;
          im[M - m] = ci;
        }
      }
      host_fft(re, im);
      std::vector<double>& g = sgn == 0 ? gf : gi;
      for (int j = 0; j < M; ++j) {
        int r = 0;
        for (int b = 0; b < logM; ++b) r |= ((j >> b) & 1) << (logM - 1 - b);
        g[2 * j] = re[r] / M;
        g[2 * j + 1] = im[r] / M;
      }
    }
    if (!(p->blue_chirp = alloc_bytes(p, sizeof(T) * chirp.size(), &st))) return st;
    if (!(p->blue_tw = alloc_bytes(p, sizeof(T) * twm.size(), &st))) return st;
    if (!(p->blue_gfwd = alloc_bytes(p, sizeof(T) * gf.size(), &st))) return st;
    if (!(p->blue_ginv = alloc_bytes(p, sizeof(T) * gi.size(), &st))) return st;
    if ((st = upload<T>(p, p->blue_chirp, chirp)) != PT_OK) return st;
    if ((st = upload<T>(p, p->blue_tw, twm)) != PT_OK) return st;
    if ((st = upload<T>(p, p->blue_gfwd, gf)) != PT_OK) return st;
    if ((st = upload<T>(p, p->blue_ginv, gi)) != PT_OK) return st;
  }
  return PT_OK;
}

// Host arrays move through the preconditioner work buffer W1 (free between solves; its start is
// aligned to 32 elements by the guard) in chunks of whole slices: contiguous copies and no device
// allocation per call.  Slices per chunk, 0 if not even one fits (then a temporary is allocated).
int staging_slices(const pt_problem* p) {
  const size_t avail = (size_t)p->lev[0].S * p->N * (p->mixed ? sizeof(float) : sizeof(double));
  return (int)std::min<size_t>((size_t)p->N, avail / (sizeof(double) * (size_t)p->ns));
}

// F = M (tau_n f_n + u0 on the first step): the load of the nodal values and the M u_I of
// §2 (after eq. 2.4) for the P1 mass; nothing to do for M = I.  W1 (FP64 with the P1 mass) holds
// the product before it is copied back.
pt_status apply_mass_to_F(pt_problem* p) {
  if (!p->mass) return PT_OK;
  const Level& L = p->lev[0];
  launch_apply_mass(p->F, (double*)p->W1, geom<double>(p, 0), p->N, p->st);
  PT_CHECK_LAUNCH();
  PT_CUDA(cudaMemcpyAsync(p->F, p->W1, sizeof(double) * (size_t)L.S * p->N, cudaMemcpyDeviceToDevice, p->st));
  return PT_OK;
}

pt_status load_rhs(pt_problem* p, const double* f, int f_dev, const double* u0, int u0_dev,
                   const unsigned long long* seed = nullptr) {
  const size_t fbytes = sizeof(double) * (size_t)p->ns * p->N;
  const double* fd = f;
  const double* u0d = u0;
  void* tf = nullptr;
  void* tu = nullptr;
  const Level& L = p->lev[0];
  if (u0 && !u0_dev) {
    PT_CUDA(cudaMallocAsync(&tu, sizeof(double) * p->ns, p->st));
    PT_CUDA(cudaMemcpyAsync(tu, u0, sizeof(double) * p->ns, cudaMemcpyHostToDevice, p->st));
    u0d = (const double*)tu;
  }
  const int chunk = staging_slices(p);
  if (!seed && f && !f_dev && chunk >= 1) {
    // F_n = tau_n f_n (+ u0 for n = 1), chunk by chunk through W1
    const size_t slice = sizeof(double) * (size_t)p->ns;
    double* stg = (double*)p->W1;
    for (int t0 = 0; t0 < p->N; t0 += chunk) {
      const int c = std::min(chunk, p->N - t0);
      PT_CUDA(cudaMemcpyAsync(stg, f + (size_t)t0 * p->ns, slice * c, cudaMemcpyHostToDevice, p->st));
      launch_pack(stg, t0 == 0 ? u0d : nullptr, p->F + (size_t)t0 * L.S, 0.0, p->stp_d + t0, p->dim, L.n, L.P,
                  L.logP, L.S, c, p->st);
      PT_CHECK_LAUNCH();
    }
    if (tu) PT_CUDA(cudaFreeAsync(tu, p->st));
    return apply_mass_to_F(p);
  }
  if (f && !f_dev) {
    PT_CUDA(cudaMallocAsync(&tf, fbytes, p->st));
    PT_CUDA(cudaMemcpyAsync(tf, f, fbytes, cudaMemcpyHostToDevice, p->st));
    fd = (const double*)tf;
  }
  // F_n = tau_n f_n (+ u0 for n = 1)
  if (seed)
    launch_pack_uniform(*seed, u0d, p->F, 0.0, p->stp_d, p->dim, L.n, L.logP, L.S, p->N, p->st);
  else if (fd)
    launch_pack(fd, u0d, p->F, 0.0, p->stp_d, p->dim, L.n, L.P, L.logP, L.S, p->N, p->st);
  else
    launch_pack_uniform(0, u0d, p->F, 0.0, nullptr, p->dim, L.n, L.logP, L.S, p->N, p->st);  // f = 0
  PT_CHECK_LAUNCH();
  if (tf) PT_CUDA(cudaFreeAsync(tf, p->st));
  if (tu) PT_CUDA(cudaFreeAsync(tu, p->st));
  return apply_mass_to_F(p);
}

pt_status create_impl(const pt_grid* grid, int N_t, double T, const pt_coeff* coeff, const double* f,
                      int f_dev, const double* u0, int u0_dev, const pt_options* opts, pt_problem* p) {
  pt_status st = PT_OK;
  PT_CUDA(cudaGetDevice(&p->device));
  p->dim = grid->dim;
  p->n = grid->n[0];
  p->N = N_t;
  p->logN = ilog2(N_t);
  if (!is_pow2(N_t)) {
    p->blueLogM = ilog2(2LL * N_t - 1);
    p->blueM = 1 << p->blueLogM;
  }
  p->T = T;
  p->tau = T / N_t;
  p->coeff = *coeff;
  if (opts) p->opt = *opts;
  // time grid: t_n and the per-step factors against the reference step tau = T/N (eq. 2.2)
  p->tn.resize(N_t);
  if (p->opt.tau_steps) {
    p->steps.assign(p->opt.tau_steps, p->opt.tau_steps + N_t);
    double t = 0.0;
    for (int i = 0; i < N_t; ++i) p->tn[i] = (t += p->steps[i]);
  } else {
    for (int i = 0; i < N_t; ++i) p->tn[i] = (i + 1) * p->tau;
  }
  p->opt.tau_steps = nullptr;  // the caller's array need not outlive the call
  double sig_max = 1.0, rho_max = 1.0;
  for (double v : p->steps) {
    sig_max = std::max(sig_max, v / p->tau);
    rho_max = std::max(rho_max, p->tau / v);
  }
  p->mixed = p->opt.precision == PT_PREC_MIXED;
  p->mass = p->opt.mass;
  p->nv_h = p->opt.n_vcycles > 0 ? p->opt.n_vcycles : 2;
  p->exact1d = p->opt.spatial_solver == PT_SOLVER_EXACT_1D;
  if (p->opt.omega > 0.0) {
    p->omega = p->opt.omega;
  } else {
    // alpha of eq. 2.2 for a in [a0 - |c|, a0 + |c|] against the mean coefficient a0, with the
    // step ratios: (1/alpha) tau a0 <= tau_n a <= alpha tau a0
    const double a0 = coeff->a0, c = std::fabs(coeff->c);
    const double alpha = std::max(sig_max * (a0 + c) / a0, rho_max * a0 / (a0 - c));
    p->omega = 1.5 / (1.0 + alpha);
  }
  p->jacobi = p->opt.jacobi_weight > 0.0 ? p->opt.jacobi_weight
                                         : (p->dim == 1 ? 2.0 / 3.0 : (p->dim == 2 ? 0.8 : 6.0 / 7.0));
  p->st = (cudaStream_t)p->opt.stream;
  // levels
  const int P0 = p->n + 1;
  p->nlev = 0;
  for (int P = P0; P >= 2; P >>= 1) {
    Level& L = p->lev[p->nlev];
    L.P = P;
    L.n = P - 1;
    L.logP = ilog2(P);
    L.S = 1;
    for (int d = 0; d < p->dim; ++d) L.S *= P;
    L.h = 1.0 / P;
    L.guard = padded_guard(L, p->dim);
    ++p->nlev;
  }
  p->coarse_elems = p->opt.coarse_elems > 0 ? p->opt.coarse_elems : kCoarseMaxElems;
  p->dstC = p->opt.dst_cols;
  p->lc = lc_for(p, p->coarse_elems);
  // buffers cover every coarse split the autotuner may choose (thresholds 256 .. 4096 points)
  p->lc_min = std::min(p->lc, lc_for(p, 4096));
  p->lc_max = std::max(p->lc, lc_for(p, 256));
  p->ns = 1;
  for (int d = 0; d < p->dim; ++d) p->ns *= p->n;
  // coefficient tables (node and face values of g_d per level)
  std::vector<double> tab;
  for (int l = 0; l < p->nlev; ++l) {
    Level& L = p->lev[l];
    L.tab = (long long)tab.size();
    for (int d = 0; d < p->dim; ++d) {
      for (int i = 0; i < L.P; ++i)
        tab.push_back(i < L.n ? trig(coeff->fx[d], M_PI * coeff->mx[d] * (i + 1) * L.h) : 0.0);
      for (int j = 0; j < L.P; ++j) tab.push_back(trig(coeff->fx[d], M_PI * coeff->mx[d] * (j + 0.5) * L.h));
    }
  }
  if (!(p->tab_d = (double*)alloc_bytes(p, sizeof(double) * tab.size(), &st))) return st;
  if (!(p->tab_f = (float*)alloc_bytes(p, sizeof(float) * tab.size(), &st))) return st;
  if ((st = upload<double>(p, p->tab_d, tab)) != PT_OK) return st;
  if ((st = upload<float>(p, p->tab_f, tab)) != PT_OK) return st;
  // time factors c g_t(t_n); reference coefficient (eq. 2.2, an average): the time mean of a over
  // (0, T), a0 + c gbar prod g_d with gbar = (1/T) int_0^T g_t(pi m_t t) dt in closed form -- the
  // same for every time grid (for uniform steps and a coefficient periodic over (0, T), the mean
  // of the A_n)
  std::vector<double> cth(p->N);
  for (int i = 0; i < p->N; ++i) cth[i] = coeff->c * trig(coeff->ft, M_PI * coeff->mt * p->tn[i]);
  const double wT = M_PI * coeff->mt * p->T;
  double gbar = 1.0;
  if (coeff->ft == PT_TRIG_SIN)
    gbar = wT == 0.0 ? 0.0 : (1.0 - std::cos(wT)) / wT;
  else if (coeff->ft == PT_TRIG_COS)
    gbar = wT == 0.0 ? 1.0 : std::sin(wT) / wT;
  p->cthbar = coeff->c * gbar;
  if (!(p->cth_d = (double*)alloc_bytes(p, sizeof(double) * p->N, &st))) return st;
  if ((st = upload<double>(p, p->cth_d, cth)) != PT_OK) return st;
  std::vector<double> stp(3 * (size_t)p->N);
  for (int i = 0; i < p->N; ++i) {
    const bool u = p->steps.empty();
    stp[i] = u ? p->tau : p->steps[i];
    stp[p->N + i] = u ? 1.0 : p->steps[i] / p->tau;
    stp[2 * p->N + i] = u ? 1.0 : p->tau / p->steps[i];
  }
  if (!(p->stp_d = (double*)alloc_bytes(p, sizeof(double) * stp.size(), &st))) return st;
  if (!(p->stp_f = (float*)alloc_bytes(p, sizeof(float) * stp.size(), &st))) return st;
  if ((st = upload<double>(p, p->stp_d, stp)) != PT_OK) return st;
  if ((st = upload<float>(p, p->stp_f, stp)) != PT_OK) return st;
  // state vectors
  const Level& L0 = p->lev[0];
  if (!(p->u = alloc_padded<double>(p, L0, p->N, &st))) return st;
  if (!(p->p = alloc_padded<double>(p, L0, p->N, &st))) return st;
  if (!(p->F = alloc_padded<double>(p, L0, p->N, &st))) return st;
  if (!p->mixed && !p->mass && p->dim == 2 && L0.P >= 32 && !(p->bres = alloc_padded<double>(p, L0, p->N, &st)))
    return st;
  if (p->mixed) {
    float** ir[5] = {&p->ir_du, &p->ir_dp, &p->ir_R1, &p->ir_R2, &p->ir_bp};
    for (float** b : ir)
      if (!(*b = alloc_padded<float>(p, L0, p->N, &st))) return st;
    if (p->dim == 2) prepare_ir_inner_2d();
    if (p->dim == 3) {
      prepare_ir_inner_3d();
      prepare_level3_rows();
    }
  }
  st = p->mixed ? setup_precision<float>(p) : setup_precision<double>(p);
  if (st != PT_OK) return st;
  if (!(p->partials = (double*)alloc_bytes(p, sizeof(double) * kReduceBlocks, &st))) return st;
  if (!(p->state = (SolveState*)alloc_bytes(p, sizeof(SolveState), &st))) return st;
  PT_CUDA(cudaMemsetAsync(p->state, 0, sizeof(SolveState), p->st));
  PT_CUDA(cudaMallocHost((void**)&p->host_state, sizeof(SolveState)));
  return load_rhs(p, f, f_dev, u0, u0_dev);
}

template <typename T>
pt_status pack_into(pt_problem* p, const double* src, T* dst) {
  const Level& L = p->lev[0];
  launch_pack_typed<T>(src, dst, p->dim, L.n, L.P, L.logP, L.S, p->N, p->st);
  PT_CHECK_LAUNCH();
  return PT_OK;
}

template <typename T>
pt_status unpack_from(pt_problem* p, const T* src, double* dst) {
  const Level& L = p->lev[0];
  launch_unpack<T>(src, dst, p->dim, L.n, L.P, L.logP, L.S, p->N, p->st);
  PT_CHECK_LAUNCH();
  PT_CUDA(cudaStreamSynchronize(p->st));
  return PT_OK;
}

pt_status ensure_tmp(pt_problem* p) {
  pt_status st = PT_OK;
  if (!p->tmpA && !(p->tmpA = alloc_padded<double>(p, p->lev[0], p->N, &st))) return st;
  if (!p->tmpB && !(p->tmpB = alloc_padded<double>(p, p->lev[0], p->N, &st))) return st;
  return PT_OK;
}

template <typename T>
pt_status comp_dst_forward(pt_problem* p, const double* r, double* out) {
  pt_status st;
  if ((st = pack_into<T>(p, r, (T*)p->W1)) != PT_OK) return st;
  launch_dst_forward<T>((T*)p->W1, p->lev[0].S, p->dim, p->n, p->lev[0].logP, dst_plan<T>(p), nullptr, p->st);
  PT_CHECK_LAUNCH();
  return unpack_from<T>(p, (const T*)p->W1, out);
}

template <typename T>
pt_status comp_dst_inverse(pt_problem* p, const double* y, double* out) {
  pt_status st;
  if ((st = pack_into<T>(p, y, (T*)p->W1)) != PT_OK) return st;
  launch_dst_inverse<T>((const T*)p->W1, p->W2, 0, 1.0, p->lev[0].S, p->dim, p->n, p->lev[0].logP,
                        dst_plan<T>(p), nullptr, p->st);
  PT_CHECK_LAUNCH();
  return unpack_from<T>(p, (const T*)p->W2, out);
}

// Operator calls outside a solve: a streamed kernel whose bounded wait ran out has set the state's
// fault flag (no finalize kernel follows to turn it into the solve status), so it is read here,
// after the call's work has finished, and cleared.
pt_status take_fault(pt_problem* p, pt_status st) {
  if (st != PT_OK) return st;
  int fault = 0;
  PT_CUDA(cudaMemcpyAsync(&fault, &p->state->fault, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  PT_CUDA(cudaStreamSynchronize(p->st));
  if (fault == 0) return PT_OK;
  PT_CUDA(cudaMemsetAsync(&p->state->fault, 0, sizeof(int), p->st));
  return fail(PT_ETIMEOUT, "a bounded wait inside a streamed kernel ran out");
}

template <typename T>
pt_status comp_precond_A(pt_problem* p, const double* r, double* out) {
  pt_status st;
  if ((st = pack_into<T>(p, r, (T*)p->W1)) != PT_OK) return st;
  if (!p->steps.empty()) {  // A~^-1 for tau_n A_n = rho_n times the solver for tau A_n
    const Level& L0 = p->lev[0];
    const T* rho = sizeof(T) == 8 ? (const T*)(const void*)steps_d(p).rho : (const T*)(const void*)steps_f(p).rho;
    launch_scale_slices<T>((T*)p->W1, rho, L0.logP * p->dim, L0.S * p->N, p->st);
  }
  apply_precond_A<T>(p, (const T*)p->W1, p->W2, 0, 0, nullptr);
  PT_CHECK_LAUNCH();
  return unpack_from<T>(p, (const T*)p->W2, out);
}

template <typename T>
pt_status comp_precond_H(pt_problem* p, const double* r, double* out) {
  pt_status st;
  if ((st = pack_into<T>(p, r, (T*)p->W1)) != PT_OK) return st;
  launch_dst_forward<T>((T*)p->W1, p->lev[0].S, p->dim, p->n, p->lev[0].logP, dst_plan<T>(p), nullptr, p->st);
  T* yhat = block_solve<T>(p, nullptr);
  T* dest = yhat == (T*)p->W1 ? (T*)p->W2 : (T*)p->W1;
  launch_dst_inverse<T>(yhat, dest, 0, 1.0, p->lev[0].S, p->dim, p->n, p->lev[0].logP, dst_plan<T>(p), nullptr,
                        p->st);
  PT_CHECK_LAUNCH();
  return unpack_from<T>(p, dest, out);
}

}  // namespace

namespace pt {

// Hooks used by the serving loop (server.cu).
pt_status problem_begin(pt_problem* p, double tol, int max_it) {
  pt_status st = ensure_hist(p, max_it);
  if (st != PT_OK) return st;
  if (p->opt.autotune > 0 && !p->tuned && (st = autotune(p)) != PT_OK) return st;
  if ((st = enqueue_reset(p, tol, max_it)) != PT_OK) return st;
  if ((st = ensure_graph(p, graph_iterations(p))) != PT_OK) return st;
  PT_CUDA(cudaStreamSynchronize(p->st));
  return PT_OK;
}

cudaGraph_t problem_graph(pt_problem* p, unsigned long long* kernels) {
  if (kernels) *kernels = p->graph_kernels;
  return p->graph;
}

SolveState* problem_state(pt_problem* p) { return p->state; }

pt_status problem_result(pt_problem* p, int* iters, pt_status* status) {
  SolveState hs;
  pt_status st = read_state(p, &hs);
  if (st != PT_OK) return st;
  if (iters) *iters = hs.iters;
  if (status) *status = (pt_status)hs.status;
  return PT_OK;
}

size_t problem_bytes(const pt_problem* p) { return p->bytes; }

long long problem_dofs(const pt_problem* p) { return p->ns * p->N; }

// Upper estimate of the device bytes pt_problem_create will allocate (admission control).
size_t estimate_problem_bytes(const pt_grid* g, int N_t, const pt_options* o) {
  const int d = g->dim;
  double P = g->n[0] + 1.0, padded = N_t;
  for (int k = 0; k < d; ++k) padded *= P;
  const bool mixed = o && o->precision == PT_PREC_MIXED;
  const double s = mixed ? 4.0 : 8.0;
  const double lev = 1.0 / ((1 << d) - 1);  // levels below the finest, relative to it
  double per = 24.0 + 3.0 * s;              // u, p, F and three work vectors
  if (mixed) per += 20.0;                   // FP32 corrections and residuals of the refinement
  if (!mixed && d == 2) per += 8.0;         // stored outer residual
  if (d >= 2 && !mixed) per += s;           // FP64 block-solve factor / pivot table (exact H_k
                                            // solves; FP32 forms the factor per point)
  per += (d == 2 ? 2.0 : 3.0) * s * lev;    // multigrid right-hand sides, iterates (and residuals)
  if (d != 2) per += 2.0 * s;               // generic path: level-0 iterate and residual
  if (d == 2 && !mixed) per += 16.0 * (1.0 + lev);  // cached (Jacobi factor, diagonal) pairs
  return (size_t)(padded * per * 1.05) + (size_t)(4u << 20);
}

}  // namespace pt

extern "C" {

const char* pt_last_error(void) { return g_err.c_str(); }

const char* pt_status_string(pt_status s) {
  switch (s) {
    case PT_OK: return "PT_OK";
    case PT_EINVAL: return "PT_EINVAL";
    case PT_ENOMEM: return "PT_ENOMEM";
    case PT_ENOTCONV: return "PT_ENOTCONV";
    case PT_EDIVERGED: return "PT_EDIVERGED";
    case PT_ECUDA: return "PT_ECUDA";
    case PT_ETIMEOUT: return "PT_ETIMEOUT";
    case PT_EBUSY: return "PT_EBUSY";
  }
  return "PT_UNKNOWN";
}

pt_status pt_problem_create(const pt_grid* grid, int N_t, double T, const pt_coeff* coeff,
                            const double* f, int f_on_device, const double* u0, int u0_on_device,
                            const pt_options* opts, pt_problem** out) {
  g_err.clear();
  if (!out) return fail(PT_EINVAL, "out is NULL");
  *out = nullptr;
  pt_status st = validate(grid, N_t, T, coeff, opts);
  if (st != PT_OK) return st;
  pt_problem* p = new pt_problem();
  st = create_impl(grid, N_t, T, coeff, f, f_on_device, u0, u0_on_device, opts, p);
  if (st == PT_OK) {
    cudaError_t e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) st = fail(PT_ECUDA, cudaGetErrorString(e));
  }
  if (st != PT_OK) {
    pt_problem_destroy(p);
    return st;
  }
  *out = p;
  return PT_OK;
}

pt_status pt_problem_set_rhs(pt_problem* p, const double* f, int f_on_device, const double* u0,
                             int u0_on_device) {
  g_err.clear();
  if (!p) return fail(PT_EINVAL, "problem is NULL");
  PT_CUDA(cudaSetDevice(p->device));
  return load_rhs(p, f, f_on_device, u0, u0_on_device);
}

pt_status pt_problem_set_rhs_uniform(pt_problem* p, unsigned long long seed, const double* u0,
                                     int u0_on_device) {
  g_err.clear();
  if (!p) return fail(PT_EINVAL, "problem is NULL");
  PT_CUDA(cudaSetDevice(p->device));
  pt_status st = load_rhs(p, nullptr, 0, u0, u0_on_device, &seed);
  if (st == PT_OK) PT_CUDA(cudaStreamSynchronize(p->st));
  return st;
}

pt_status pt_solve(pt_problem* p, double tol, int max_it, double* u_out, int u_out_on_device,
                   double* res_hist, int* iters) {
  g_err.clear();
  if (!p) return fail(PT_EINVAL, "problem is NULL");
  if (max_it < 0 || !(tol >= 0.0)) return fail(PT_EINVAL, "need max_it >= 0 and tol >= 0");
  PT_CUDA(cudaSetDevice(p->device));
  pt_status st = ensure_hist(p, max_it);
  if (st != PT_OK) return st;
  if (p->opt.autotune > 0 && !p->tuned && (st = autotune(p)) != PT_OK) return st;
  st = p->opt.krylov > 0 ? krylov_solve(p, tol, max_it, iters, res_hist) : uzawa(p, tol, max_it, iters, res_hist);
  if (st != PT_OK && st != PT_ENOTCONV && st != PT_EDIVERGED) return st;
  if (u_out) {
    const Level& L = p->lev[0];
    const size_t bytes = sizeof(double) * (size_t)p->ns * p->N;
    double* dst = u_out;
    void* tmp = nullptr;
    const int chunk = staging_slices(p);
    if (!u_out_on_device && chunk >= 1) {  // through W1, chunk by chunk (see load_rhs)
      const size_t slice = sizeof(double) * (size_t)p->ns;
      double* stg = (double*)p->W1;
      for (int t0 = 0; t0 < p->N; t0 += chunk) {
        const int c = std::min(chunk, p->N - t0);
        launch_unpack<double>(p->u + (size_t)t0 * L.S, stg, p->dim, L.n, L.P, L.logP, L.S, c, p->st);
        PT_CHECK_LAUNCH();
        PT_CUDA(cudaMemcpyAsync(u_out + (size_t)t0 * p->ns, stg, slice * c, cudaMemcpyDeviceToHost, p->st));
      }
      PT_CUDA(cudaStreamSynchronize(p->st));
      return st;
    }
    if (!u_out_on_device) {
      PT_CUDA(cudaMallocAsync(&tmp, bytes, p->st));
      dst = (double*)tmp;
    }
    launch_unpack<double>(p->u, dst, p->dim, L.n, L.P, L.logP, L.S, p->N, p->st);
    PT_CHECK_LAUNCH();
    if (tmp) {
      PT_CUDA(cudaMemcpyAsync(u_out, tmp, bytes, cudaMemcpyDeviceToHost, p->st));
      PT_CUDA(cudaFreeAsync(tmp, p->st));
    }
    PT_CUDA(cudaStreamSynchronize(p->st));
  }
  return st;
}

pt_status pt_solve_batch(pt_problem** ps, int count, const double* tol, const int* max_it, int* iters,
                         pt_status* status) {
  g_err.clear();
  if (!ps || count < 1 || !tol || !max_it) return fail(PT_EINVAL, "need problems, tol and max_it");
  int dev = -1;
  for (int i = 0; i < count; ++i) {
    if (!ps[i]) return fail(PT_EINVAL, "NULL problem in batch");
    if (max_it[i] < 0 || !(tol[i] >= 0.0)) return fail(PT_EINVAL, "need max_it >= 0 and tol >= 0");
    if (dev >= 0 && ps[i]->device != dev) return fail(PT_EINVAL, "all problems must be on one device");
    dev = ps[i]->device;
    for (int k = 0; k < i; ++k)
      if (ps[k] == ps[i]) return fail(PT_EINVAL, "a problem appears twice in the batch");
  }
  PT_CUDA(cudaSetDevice(dev));
  pt_status st;
  int max_rounds = 0;
  for (int i = 0; i < count; ++i) {
    pt_problem* p = ps[i];
    if ((st = ensure_hist(p, max_it[i])) != PT_OK) return st;
    if (p->opt.autotune > 0 && !p->tuned && (st = autotune(p)) != PT_OK) return st;
    if ((st = enqueue_reset(p, tol[i], max_it[i])) != PT_OK) return st;
    max_rounds = std::max(max_rounds, max_it[i] + 1);
  }
  for (int i = 0; i < count; ++i) PT_CUDA(cudaStreamSynchronize(ps[i]->st));
  const bool graphs = !profiling_enabled();
  if (graphs)
    for (int i = 0; i < count; ++i)
      if ((st = ensure_graph(ps[i], graph_iterations(ps[i]))) != PT_OK) return st;
  // device list of the solve states and a pinned copy of their done flags
  cudaStream_t bst = nullptr;
  cudaStream_t cst = nullptr;
  SolveState** dstates = nullptr;
  int* ddone = nullptr;
  int* hdone = nullptr;
  int* didx = nullptr;      // active problem indices (device loop)
  int* drounds = nullptr;   // rounds run by the device loop in the current launch
  int* hrounds = nullptr;
  cudaGraph_t parent = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (parent) cudaGraphDestroy(parent);
    if (dstates) cudaFree(dstates);
    if (ddone) cudaFree(ddone);
    if (didx) cudaFree(didx);
    if (drounds) cudaFree(drounds);
    if (hdone) cudaFreeHost(hdone);
    if (hrounds) cudaFreeHost(hrounds);
    if (bst) cudaStreamDestroy(bst);
    if (cst) cudaStreamDestroy(cst);
  };
#define PT_BATCH_CUDA(call)                                                          \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cleanup();                                                                     \
      return fail(PT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    }                                                                                \
  } while (0)
  PT_BATCH_CUDA(cudaStreamCreateWithFlags(&bst, cudaStreamNonBlocking));
  PT_BATCH_CUDA(cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking));
  std::vector<SolveState*> hstates(count);
  for (int i = 0; i < count; ++i) hstates[i] = ps[i]->state;
  PT_BATCH_CUDA(cudaMalloc(&dstates, sizeof(SolveState*) * count));
  PT_BATCH_CUDA(cudaMalloc(&ddone, sizeof(int) * count));
  PT_BATCH_CUDA(cudaMalloc(&didx, sizeof(int) * count));
  PT_BATCH_CUDA(cudaMalloc(&drounds, sizeof(int)));
  PT_BATCH_CUDA(cudaMallocHost(&hdone, sizeof(int) * count));
  PT_BATCH_CUDA(cudaMallocHost(&hrounds, sizeof(int)));
  PT_BATCH_CUDA(cudaMemcpyAsync(dstates, hstates.data(), sizeof(SolveState*) * count, cudaMemcpyHostToDevice, bst));
  std::vector<int> active(count);
  for (int i = 0; i < count; ++i) active[i] = i;
  unsigned long long kernels_per_round = 0;
  // Device-side loop: the parent graph is one conditional WHILE node whose body holds one
  // iteration of every active problem (each problem's captured iteration graph as a child node)
  // and the control kernel, so a whole run of rounds is a single graph launch; the loop ends on
  // the device once a quarter of the active set has finished (all of it when one is left), or
  // after the round limit.  Then the host drops the finished problems and launches again.  If
  // the CUDA driver cannot build conditional nodes, one plain graph launch per round is used instead.
  const int limit = max_rounds + 2;
  bool device_loop = graphs;
  auto rebuild = [&]() -> cudaError_t {
    if (exec) cudaGraphExecDestroy(exec);
    if (parent) cudaGraphDestroy(parent);
    exec = nullptr;
    parent = nullptr;
    kernels_per_round = 0;
    cudaError_t e = cudaGraphCreate(&parent, 0);
    if (e != cudaSuccess) return e;
    cudaGraph_t body = parent;
    cudaGraphConditionalHandle handle = 0;
    if (device_loop) {
      e = cudaGraphConditionalHandleCreate(&handle, parent, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode;
      if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, parent, nullptr, nullptr, 0, &cp);
      if (e != cudaSuccess) {  // no conditional nodes: per-round launches
        cudaGetLastError();
        device_loop = false;
        cudaGraphDestroy(parent);
        if ((e = cudaGraphCreate(&parent, 0)) != cudaSuccess) return e;
        body = parent;
      } else {
        body = cp.conditional.phGraph_out[0];
      }
    }
    std::vector<cudaGraphNode_t> nodes(active.size());
    for (size_t a = 0; e == cudaSuccess && a < active.size(); ++a) {
      e = cudaGraphAddChildGraphNode(&nodes[a], body, nullptr, 0, ps[active[a]]->graph);
      kernels_per_round += ps[active[a]]->graph_kernels;
    }
    if (e == cudaSuccess && device_loop) {
      std::vector<int> idx(active.begin(), active.end());
      e = cudaMemcpyAsync(didx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, bst);
      if (e == cudaSuccess) e = cudaStreamSynchronize(bst);
      const int n_act = (int)active.size();
      const int keep_above = n_act == 1 ? 0 : n_act - (n_act + 3) / 4;
      capture_begin();
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(cst, body, nodes.data(), nullptr, nodes.size(),
                                          cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        launch_batch_control(dstates, didx, n_act, keep_above, drounds, limit, handle, cst);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cst, &captured);
      }
      capture_end();
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, parent, 0);
    return e;
  };
  if (graphs) PT_BATCH_CUDA(rebuild());
  int check = ps[0]->opt.check_every > 0 ? ps[0]->opt.check_every : 4;
  int rounds = 0;
  while (!active.empty()) {
    if (graphs && device_loop) {
      PT_BATCH_CUDA(cudaMemsetAsync(drounds, 0, sizeof(int), bst));
      PT_BATCH_CUDA(cudaGraphLaunch(exec, bst));
      PT_BATCH_CUDA(cudaMemcpyAsync(hrounds, drounds, sizeof(int), cudaMemcpyDeviceToHost, bst));
    } else if (graphs) {
      PT_BATCH_CUDA(cudaGraphLaunch(exec, bst));
      note_launch((int)kernels_per_round);
    } else {
      for (int i : active) {
        cudaStream_t saved = ps[i]->st;
        ps[i]->st = bst;
        enqueue_iteration_any(ps[i]);
        ps[i]->st = saved;
      }
      PT_BATCH_CUDA(cudaGetLastError());
    }
    if (graphs && device_loop) {
      // the loop ran hrounds rounds on the device
      launch_gather_done(dstates, count, ddone, bst);
      PT_BATCH_CUDA(cudaMemcpyAsync(hdone, ddone, sizeof(int) * count, cudaMemcpyDeviceToHost, bst));
      PT_BATCH_CUDA(cudaStreamSynchronize(bst));
      rounds += *hrounds;
      note_launch((int)((kernels_per_round + 1) * (unsigned long long)*hrounds));
    } else {
      ++rounds;
      if (!(rounds % check == 0 || rounds > max_rounds)) continue;
      launch_gather_done(dstates, count, ddone, bst);
      PT_BATCH_CUDA(cudaMemcpyAsync(hdone, ddone, sizeof(int) * count, cudaMemcpyDeviceToHost, bst));
      PT_BATCH_CUDA(cudaStreamSynchronize(bst));
    }
    std::vector<int> still;
    for (int i : active)
      if (!hdone[i]) still.push_back(i);
    const size_t finished = active.size() - still.size();
    if (still.empty()) break;
    if (rounds > max_rounds + 2) {
      cleanup();
      return fail(PT_ECUDA, "batch did not stop at max_it");
    }
    if (finished > 0 && (device_loop || finished * 4 >= active.size())) {  // drop finished problems
      active.swap(still);
      if (graphs) PT_BATCH_CUDA(rebuild());
    }
  }
  PT_BATCH_CUDA(cudaStreamSynchronize(bst));
  cleanup();
#undef PT_BATCH_CUDA
  for (int i = 0; i < count; ++i) {
    SolveState hs;
    if ((st = read_state(ps[i], &hs)) != PT_OK) return st;
    if (iters) iters[i] = hs.iters;
    if (status) status[i] = (pt_status)hs.status;
  }
  return PT_OK;
}

pt_status pt_problem_estimate_bytes(const pt_grid* grid, int N_t, const pt_options* opts, size_t* bytes_out) {
  g_err.clear();
  if (!grid || !bytes_out) return fail(PT_EINVAL, "grid and bytes_out are required");
  if (grid->dim < 1 || grid->dim > 3 || N_t < 1) return fail(PT_EINVAL, "bad grid or N_t");
  *bytes_out = pt::estimate_problem_bytes(grid, N_t, opts);
  return PT_OK;
}

pt_status pt_problem_device_bytes(const pt_problem* p, size_t* bytes_out) {
  g_err.clear();
  if (!p || !bytes_out) return fail(PT_EINVAL, "problem and bytes_out are required");
  *bytes_out = pt::problem_bytes(p);
  return PT_OK;
}

pt_status pt_problem_get_state(pt_problem* p, double* u_out, double* p_out, int on_device) {
  g_err.clear();
  if (!p) return fail(PT_EINVAL, "problem is NULL");
  PT_CUDA(cudaSetDevice(p->device));
  const Level& L = p->lev[0];
  const size_t bytes = sizeof(double) * (size_t)p->ns * p->N;
  double* srcs[2] = {p->u, p->p};
  double* dsts[2] = {u_out, p_out};
  for (int k = 0; k < 2; ++k) {
    if (!dsts[k]) continue;
    double* dst = dsts[k];
    void* tmp = nullptr;
    if (!on_device) {
      PT_CUDA(cudaMallocAsync(&tmp, bytes, p->st));
      dst = (double*)tmp;
    }
    launch_unpack<double>(srcs[k], dst, p->dim, L.n, L.P, L.logP, L.S, p->N, p->st);
    PT_CHECK_LAUNCH();
    if (tmp) {
      PT_CUDA(cudaMemcpyAsync(dsts[k], tmp, bytes, cudaMemcpyDeviceToHost, p->st));
      PT_CUDA(cudaFreeAsync(tmp, p->st));
    }
  }
  PT_CUDA(cudaStreamSynchronize(p->st));
  return PT_OK;
}

void pt_problem_destroy(pt_problem* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->st);
  drop_graph(p);
  if (p->cap) cudaStreamDestroy(p->cap);
  for (void* a : p->allocs) cudaFree(a);
  if (p->host_state) cudaFreeHost(p->host_state);
  delete p;
}

pt_status pt_apply_B(pt_problem* p, const double* u_dev, double* out_dev) {
  g_err.clear();
  if (!p || !u_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  PT_CUDA(cudaSetDevice(p->device));
  pt_status st = ensure_tmp(p);
  if (st != PT_OK) return st;
  if ((st = pack_into<double>(p, u_dev, p->tmpA)) != PT_OK) return st;
  launch_apply_B(p->tmpA, p->tmpB, geom<double>(p, 0), p->cth_d, steps_d(p), p->N, p->st);
  PT_CHECK_LAUNCH();
  return unpack_from<double>(p, p->tmpB, out_dev);
}

pt_status pt_apply_S(pt_problem* p, const double* u_dev, double* out_dev) {
  g_err.clear();
  if (!p || !u_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  if (p->mixed) return fail(PT_EINVAL, "pt_apply_S needs an FP64 problem");
  PT_CUDA(cudaSetDevice(p->device));
  pt_status st = ensure_tmp(p);
  if (st != PT_OK) return st;
  if ((st = pack_into<double>(p, u_dev, p->tmpA)) != PT_OK) return st;
  const StencilGeom<double> g = geom<double>(p, 0);
  // S u = K^T A~^-1 K u + (K + K^T + A) u = K^T (A~^-1 K u + u) + B u
  launch_apply_K(p->tmpA, (double*)p->W1, g, steps_d(p).rho, p->N, p->st);
  apply_precond_A<double>(p, (const double*)p->W1, p->W2, 0, 0, nullptr);
  launch_apply_B(p->tmpA, p->tmpB, g, p->cth_d, steps_d(p), p->N, p->st);
  launch_add_KT(p->tmpB, (const double*)p->W2, p->tmpA, g, p->N, p->st);
  PT_CHECK_LAUNCH();
  return unpack_from<double>(p, p->tmpB, out_dev);
}

pt_status pt_dst_forward(pt_problem* p, const double* r_dev, double* out_dev) {
  g_err.clear();
  if (!p || !r_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  PT_CUDA(cudaSetDevice(p->device));
  return p->mixed ? comp_dst_forward<float>(p, r_dev, out_dev) : comp_dst_forward<double>(p, r_dev, out_dev);
}

pt_status pt_dst_inverse(pt_problem* p, const double* y_dev, double* out_dev) {
  g_err.clear();
  if (!p || !y_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  PT_CUDA(cudaSetDevice(p->device));
  return p->mixed ? comp_dst_inverse<float>(p, y_dev, out_dev) : comp_dst_inverse<double>(p, y_dev, out_dev);
}

pt_status pt_precond_A(pt_problem* p, const double* r_dev, double* out_dev) {
  g_err.clear();
  if (!p || !r_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  PT_CUDA(cudaSetDevice(p->device));
  return take_fault(p, p->mixed ? comp_precond_A<float>(p, r_dev, out_dev) : comp_precond_A<double>(p, r_dev, out_dev));
}

pt_status pt_precond_H(pt_problem* p, const double* r_dev, double* out_dev) {
  g_err.clear();
  if (!p || !r_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  PT_CUDA(cudaSetDevice(p->device));
  return take_fault(p, p->mixed ? comp_precond_H<float>(p, r_dev, out_dev) : comp_precond_H<double>(p, r_dev, out_dev));
}

}  // extern "C"
