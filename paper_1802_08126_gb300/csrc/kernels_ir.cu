// Mixed precision as iterative refinement of the Uzawa iteration (§3, eq. 3.1).
//
// The inexact Uzawa method is a stationary linear iteration x <- x + M^-1 (b - K x) for the
// saddle-point system of eq. 2.7 written as
//     -tau A p + K u = F,     K^T p + (K^T + B) u = F,      B = K + tau A,
// with M block lower triangular (A~ on the first block, omega^-1 H~ on the second).  Run on the
// correction equation K dx = b - K x from dx = 0, it produces the same iterates as when run on x
// itself.  So the iterate is kept in FP64 (u, p), and every few iterations its residual is formed
// in FP64 and rounded to FP32:
//     R1 = F - (K u - tau A p) = bres + tau A w,    R2 = F - K^T p - (K^T + B) u = bres - K^T w,
//     bres = F - B u,  w = p + u;
// the iterations in between run entirely in FP32 on the corrections (du, dp) with right-hand side
// (R1, R2):
//     b'   = R2 - B du                     (estimate of the outer residual F - B (u + du))
//     r_p' = K du - tau A dp - R1,         dp += A~^-1 r_p'
//     r_u' = b' - K^T (dp + du),           du += omega H~^-1 r_u'
// and the next FP64 step folds them in: u += du, p += dp.  With non-uniform steps tau A stands for
// diag(tau_n A_n) and the A~ inputs are scaled by rho_n = tau / tau_n (the V-cycles are formed for
// the reference step tau).  The FP64 step comes every kOuter
// iterations, and at once when the FP32 estimate ||b'|| reaches the tolerance or the iteration
// limit: the solve only ends on an FP64 residual of the FP64 iterate it returns.
//
// Device control (SolveState): `outer` marks an iteration that starts with the FP64 step;
// done == 2 skips the rest of an iteration (the FP32 estimate asked for confirmation), and the
// begin kernel of the next iteration turns it into an FP64 step for the same index j.
#include "stencil_common.cuh"

namespace pt {
namespace {

__device__ __forceinline__ int vload(const int* p) { return *((volatile const int*)p); }

__global__ void k_ir_begin(SolveState* st, int kouter) {
  if (vload(&st->done) == 1) return;
  const int confirm = vload(&st->done) == 2;
  st->done = 0;
  st->outer = (confirm || st->j % kouter == 0) ? 1 : 0;
}

// FP64 step, part 1: u += du, p += dp, du = dp = 0 (every padded element; ghosts stay zero)
__global__ void k_ir_fold(double* __restrict__ u, double* __restrict__ p, float* __restrict__ du,
                          float* __restrict__ dp, long long total, const SolveState* st) {
  if (vload(&st->done) != 0 || !vload(&st->outer)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    u[i] += (double)du[i];
    p[i] += (double)dp[i];
    du[i] = 0.f;
    dp[i] = 0.f;
  }
}

// FP64 step, part 2: bres = F - B u (FP64, norm partials), w = p + u; R1, R2 in FP32 and the
// first A~ input rho_t r_p' = -rho_t R1 into rp.  tau A w in FP32 (w -> 0 at the solution, it only enters the
// FP32 right-hand sides).
template <int DIM>
__global__ void k_ir_outer(const double* __restrict__ u, const double* __restrict__ p,
                           const double* __restrict__ F, float* __restrict__ R1, float* __restrict__ R2,
                           float* __restrict__ rp, double* __restrict__ partials, StencilGeom<double> g,
                           const double* __restrict__ cth, Steps<double> sp, int N, long long total,
                           const SolveState* st) {
  if (vload(&st->done) != 0 || !vload(&st->outer)) return;
  double acc = 0.0;
  const float h2f = (float)g.h2inv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    float r1 = 0.f, r2 = 0.f, rho = 1.f;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      double am[3], ap[3];
      face_coefs<DIM, double>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const double uc = u[i];
      const double Au = stencil_sum<DIM, double>(u, i, uc, am, ap, g.P) * g.h2inv;
      const double um = t > 0 ? u[i - g.S] : 0.0;
      const double tau = sp.tau[t];
      const float tauf = (float)tau;
      rho = (float)sp.rho[t];
      const double b = F[i] - (uc - um) - tau * Au;
      acc += b * b;
      const double wc = p[i] + uc;
      const double wn = t + 1 < N ? p[i + g.S] + u[i + g.S] : 0.0;
      const long long off[3] = {1, g.P, (long long)g.P * g.P};
      float aw = 0.f;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const float wm = (float)(p[i - off[d]] + u[i - off[d]]);
        const float wp = (float)(p[i + off[d]] + u[i + off[d]]);
        aw += (float)am[d] * ((float)wc - wm) + (float)ap[d] * ((float)wc - wp);
      }
      r1 = (float)b + tauf * h2f * aw;
      r2 = (float)(b - (wc - wn));
    }
    R1[i] = r1;
    R2[i] = r2;
    rp[i] = -(rho * r1);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// FP32 step: b' = R2 - B du (norm partials in FP64), A~ input rho_t r_p', r_p' = K du - tau_t A dp - R1
template <int DIM>
__global__ void k_ir_inner(const float* __restrict__ du, const float* __restrict__ dp,
                           const float* __restrict__ R1, const float* __restrict__ R2, float* __restrict__ bp,
                           float* __restrict__ rp, double* __restrict__ partials, StencilGeom<float> g,
                           const float* __restrict__ cth, Steps<float> sp, long long total, const SolveState* st) {
  if (vload(&st->done) != 0 || vload(&st->outer)) return;
  float acc = 0.f;  // per-thread sum in FP32 (an estimate), block sum in FP64
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    float b = 0.f, r = 0.f;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      float am[3], ap[3];
      face_coefs<DIM, float>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const float dc = du[i];
      const float Kd = dc - (t > 0 ? du[i - g.S] : 0.f);
      const float Ad = stencil_sum<DIM, float>(du, i, dc, am, ap, g.P);
      const float pc = dp[i];
      const float Ap = stencil_sum<DIM, float>(dp, i, pc, am, ap, g.P);
      const float sc = sp.tau[t] * g.h2inv;
      b = R2[i] - Kd - sc * Ad;
      r = (Kd - sc * Ap - R1[i]) * sp.rho[t];
      acc = fmaf(b, b, acc);
    }
    bp[i] = b;
    rp[i] = r;
  }
  const double sum = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

// r_u' = b' - K^T (dp + du); b' is R2 on the FP64-step iteration (du = 0 there)
__global__ void k_ir_resid_u(const float* __restrict__ bp, const float* __restrict__ R2,
                             const float* __restrict__ du, const float* __restrict__ dp, float* __restrict__ ru,
                             long long S, long long total, const SolveState* st) {
  if (vload(&st->done) != 0) return;
  const float* b = vload(&st->outer) ? R2 : bp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float wn = i + S < total ? dp[i + S] + du[i + S] : 0.f;
    ru[i] = b[i] - (dp[i] + du[i]) + wn;
  }
}

// Residual bookkeeping of one iteration: the FP64 step decides convergence, an FP32 estimate
// at or below the tolerance (or the iteration limit) asks for an FP64 step at the same index.
__global__ void k_ir_finalize(const double* __restrict__ partials, SolveState* state, double* __restrict__ hist) {
  if (vload(&state->done) != 0) return;
  if (vload(&state->fault) != 0) {
    if (threadIdx.x == 0) {
      state->status = PT_ETIMEOUT;
      state->done = 1;
    }
    return;
  }
  double v = partials[threadIdx.x];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    const int j = state->j;
    const double res = sqrt(v / state->fnorm2);
    hist[j] = res;
    state->last_res = res;
    state->iters = j;
    if (state->outer) {
      if (!(res <= 1e30)) {
        state->status = PT_EDIVERGED;
        state->done = 1;
      } else if (res <= state->tol) {
        state->status = PT_OK;
        state->done = 1;
      } else if (j >= state->max_it) {
        state->status = PT_ENOTCONV;
        state->done = 1;
      } else {
        state->j = j + 1;
      }
    } else if (!(res <= 1e30) || res <= state->tol || j >= state->max_it) {
      state->done = 2;
    } else {
      state->j = j + 1;
    }
  }
}

}  // namespace

#define PT_IR_DIM(dim, ...)   \
  switch (dim) {              \
    case 1: {                 \
      constexpr int D = 1;    \
      __VA_ARGS__;            \
    } break;                  \
    case 2: {                 \
      constexpr int D = 2;    \
      __VA_ARGS__;            \
    } break;                  \
    default: {                \
      constexpr int D = 3;    \
      __VA_ARGS__;            \
    } break;                  \
  }

void launch_ir_begin(SolveState* st, int kouter, cudaStream_t s) {
  LaunchScope ls("ir_begin", s, 0.0);
  k_ir_begin<<<1, 1, 0, s>>>(st, kouter);
}

void launch_ir_fold(double* u, double* p, float* du, float* dp, long long total, const SolveState* st,
                    cudaStream_t s) {
  LaunchScope ls("ir_fold", s, 40.0 * (double)total, 0.0, kOuterStep);
  k_ir_fold<<<grid_for(total), kThreads, 0, s>>>(u, p, du, dp, total, st);
}

void launch_ir_outer(const double* u, const double* p, const double* F, float* R1, float* R2, float* rp,
                     double* partials, StencilGeom<double> g, const double* cth, Steps<double> sp, int N,
                     const SolveState* st, cudaStream_t s) {
  const long long total = g.S * N;
  LaunchScope ls("ir_outer", s, (24.0 + 12.0) * (double)total, 0.0, kOuterStep);
  PT_IR_DIM(g.dim, k_ir_outer<D><<<kReduceBlocks, kThreads, 0, s>>>(u, p, F, R1, R2, rp, partials, g, cth, sp, N,
                                                                    total, st));
}

void launch_ir_inner(const float* du, const float* dp, const float* R1, const float* R2, float* bp, float* rp,
                     double* partials, StencilGeom<float> g, const float* cth, Steps<float> sp, int N,
                     const SolveState* st, cudaStream_t s) {
  const long long total = g.S * N;
  LaunchScope ls("ir_inner", s, 24.0 * (double)total, 0.0, kInnerStep);
  PT_IR_DIM(g.dim, k_ir_inner<D><<<kReduceBlocks, kThreads, 0, s>>>(du, dp, R1, R2, bp, rp, partials, g, cth, sp,
                                                                    total, st));
}

void launch_ir_resid_u(const float* bp, const float* R2, const float* du, const float* dp, float* ru, long long S,
                       int N, const SolveState* st, cudaStream_t s) {
  const long long total = S * N;
  LaunchScope ls("ir_resid_u", s, 16.0 * (double)total);
  k_ir_resid_u<<<grid_for(total), kThreads, 0, s>>>(bp, R2, du, dp, ru, S, total, st);
}

void launch_ir_finalize(const double* partials, SolveState* state, double* hist, cudaStream_t s) {
  LaunchScope ls("finalize", s, 8.0 * kReduceBlocks);
  k_ir_finalize<<<1, kReduceBlocks, 0, s>>>(partials, state, hist);
}

}  // namespace pt
