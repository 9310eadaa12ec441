// 2-D residual kernels with a small FP64 instruction count (the FP64 rate of this GPU is 1/64 of
// its FP32 rate, so these kernels are bound by FP64 instruction issue, not by memory).
//
// One pass forms, for every interior point of every step t,
//   bres = F - (u_t - u_{t-1}) - tau_t A_t u_t        (outer residual F - B u, FP64, stored)
//   r_p  = -bres - tau_t A_t (p_t + u_t)               (= K u - tau_t A_t p - F, first line of eq. 3.1)
// and the squared norm of bres; the second residual r_u = bres - K^T (p + u) is then a
// stencil-free pass.  w = p + u tends to zero, so its stencil is taken in FP32 in the mixed-
// precision form (the A~ input is rounded to FP32 anyway) and in FP64 in the plain form.
//
// Each warp sweeps a strip of kRows rows for 32 consecutive columns: the rows above and below
// stay in registers, x-neighbours of w come from warp shuffles, and the face coefficients
// (tau/h^2)(a0 + c g_t(t) g_x g_y) are one FMA each from per-row / per-column factors.  They are
// formed for the reference step tau (the operator of the V-cycles); the step's own tau_t enters as
// sigma_t = tau_t / tau in the multiply-add that subtracts the stencil from the residual, and the A~
// input is written as rho_t r_p (rho_t = tau / tau_t), which is -rho_t bres - (tau A_t)(p + u): no
// FP64 operation more than for uniform steps.
#include "bulk_pipe.cuh"
#include "stencil_common.cuh"

namespace pt {
namespace {

constexpr int kRows = 16;

// IR = true: the FP64 step of the mixed-precision refinement -- instead of bres and r_p it writes
// the FP32 right-hand sides R1 = bres + tau_t A w, R2 = bres - K^T w and rho_t r_p' = -rho_t R1, and
// runs only on refinement iterations (state flags).
// DG = true (FP64 path): the cached pairs (w/D, D) of tau A_n give the diagonal, and both
// stencils are D x_c - sum_f a_f x_f (six fewer FP64 operations per point).
// SC: 0 uniform steps (sigma = rho = 1, no factors), 1 sigma_t and rho_t, 2 sigma_t only and r_p
// itself (not with IR: the Krylov path's operator).  The FP64 form with both factors is held to 64
// registers (4 CTAs per SM, no spills), as the uniform one is.
template <typename W, bool IR, bool DG = false, int SC = 0>
__global__ void __launch_bounds__(256, (SC == 1 && DG && sizeof(W) == 8) ? 4 : 1) k_resid_bres_2d(
    const double* __restrict__ u, const double* __restrict__ p, const double* __restrict__ F,
    double* __restrict__ bres, W* __restrict__ rp, double* __restrict__ partials,
    const double* __restrict__ tab, const float* __restrict__ tabf, const double* __restrict__ cth,
    double a0s, double s_h2, int n, int logP, long long S, int N, long long nwarps, const int* done,
    float* __restrict__ R1, float* __restrict__ R2, const SolveState* st, Steps<double> sp,
    const double* __restrict__ jd = nullptr) {
  if (IR) {
    if (*((volatile const int*)&st->done) != 0 || !*((volatile const int*)&st->outer)) return;
  } else if (stop_requested(done)) {
    return;
  }
  const int P = 1 << logP;
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  // fixed grid (deterministic partial sums): each warp takes strips wg, wg + gridDim*8, ...
  for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wg < nwarps;
       wg += (long long)gridDim.x * (blockDim.x >> 5)) {
    const int wx_count = P >> 5, strips = P / kRows;
    const int wx = (int)(wg % wx_count);
    const long long rest = wg / wx_count;
    const int strip = (int)(rest % strips);
    const int t = (int)(rest / strips);
    const int x = (wx << 5) + lane;
    const int y0 = strip * kRows;
    const double* nx = tab;
    const double* fx = tab + P;
    const double* ny = tab + 2 * P;
    const double* fy = tab + 3 * P;
    const double ct = s_h2 * cth[t];  // (tau/h^2) c g_t(t_t)
    double sg = 1.0, rh = 1.0;
    if constexpr (SC >= 1) sg = sp.sig[t];
    if constexpr (SC == 1) rh = sp.rho[t];
    const float a0f = (float)a0s, ctf = (float)ct;
    const float* nxf = tabf;
    const float* fxf = tabf + P;
    const float* nyf = tabf + 2 * P;
    const float* fyf = tabf + 3 * P;
    const bool xin = x < n;
    const double fxl = fx[x], fxr = fx[x + 1 < P ? x + 1 : x];
    const double gxc = ct * nx[x];
    const float fxlf = fxf[x], fxrf = fxf[x + 1 < P ? x + 1 : x], gxcf = ctf * nxf[x];
    const long long base = (long long)t * S + x;
    auto at = [&](int y) { return base + (long long)y * P; };
    // rows y0-1 and y0 of u and w
    double u_m = u[at(y0) - P];
    double u_c = u[at(y0)];
    W w_m = (W)(p[at(y0) - P] + u_m);
    W w_c = (W)(p[at(y0)] + u_c);
    double ayl = fma(gxc, fy[y0], a0s);  // lower y-face of row y0
    float aylf = fmaf(gxcf, fyf[y0], a0f);
    for (int k = 0; k < kRows; ++k) {
      const int y = y0 + k;
      const bool yin = y < n;
      double u_p = 0.0;
      W w_p = (W)0;
      if (y + 1 < P) {
        u_p = u[at(y + 1)];
        w_p = (W)(p[at(y + 1)] + u_p);
      }
      // x-neighbours of w from the neighbouring lanes; the two edge lanes compute theirs
      W wW = __shfl_up_sync(0xffffffffu, w_c, 1);
      W wE = __shfl_down_sync(0xffffffffu, w_c, 1);
      if (lane == 0 && yin) wW = (W)(p[at(y) - 1] + u[at(y) - 1]);
      if (lane == 31 && yin && x + 1 < P) wE = (W)(p[at(y) + 1] + u[at(y) + 1]);
      const double ayu = fma(gxc, fy[y + 1 < P ? y + 1 : y], a0s);  // upper y-face
      const float ayuf = fmaf(gxcf, fyf[y + 1 < P ? y + 1 : y], a0f);
      double b = 0.0;
      W r = (W)0;
      float r1 = 0.f, r2 = 0.f;
      if (xin && yin) {
        const long long i = at(y);
        const double gy = ct * ny[y];
        const double axl = fma(gy, fxl, a0s), axr = fma(gy, fxr, a0s);
        const double uW = u[i - 1], uE = u[i + 1];
        const double um = t > 0 ? u[i - S] : 0.0;
        double D = 0.0;
        if constexpr (DG) D = ((const double2*)jd)[i].y;
        const double su = DG ? D * u_c - (axl * uW + axr * uE + ayl * u_m + ayu * u_p)
                             : axl * (u_c - uW) + axr * (u_c - uE) + ayl * (u_c - u_m) + ayu * (u_c - u_p);
        if constexpr (SC == 0)
          b = F[i] - (u_c - um) - su;
        else
          b = fma(-sg, su, F[i] - (u_c - um));
        acc = fma(b, b, acc);
        W sw;
        if (sizeof(W) == 4) {
          const float gyf = ctf * nyf[y];
          const float axlf = fmaf(gyf, fxlf, a0f), axrf = fmaf(gyf, fxrf, a0f);
          sw = (W)(axlf * ((float)w_c - (float)wW) + axrf * ((float)w_c - (float)wE) +
                   aylf * ((float)w_c - (float)w_m) + ayuf * ((float)w_c - (float)w_p));
        } else if constexpr (DG) {
          sw = (W)(D * (double)w_c - (axl * (double)wW + axr * (double)wE + ayl * (double)w_m + ayu * (double)w_p));
        } else {
          sw = (W)(axl * ((double)w_c - (double)wW) + axr * ((double)w_c - (double)wE) +
                   ayl * ((double)w_c - (double)w_m) + ayu * ((double)w_c - (double)w_p));
        }
        if (IR) {
          const long long in = i + S;
          const double wn = t + 1 < N ? p[in] + u[in] : 0.0;
          const double wc = p[i] + u_c;
          if constexpr (SC == 0)
            r1 = (float)b + (float)sw;
          else
            r1 = fmaf((float)sg, (float)sw, (float)b);
          r2 = (float)(b - (wc - wn));
        } else if constexpr (SC == 0) {
          r = (W)(-b) - sw;
        } else if constexpr (SC == 1) {  // rho_t r_p = -rho_t b - sw
          if constexpr (sizeof(W) == 8)
            r = (W)fma(-rh, b, -(double)sw);
          else
            r = (W)(-(rh * b)) - sw;
        } else {  // r_p = -b - sigma_t sw
          if constexpr (sizeof(W) == 8)
            r = (W)fma(-sg, (double)sw, -b);
          else
            r = (W)(-b) - (W)(sg * (double)sw);
        }
      }
      if (y < P) {
        if (IR) {
          R1[at(y)] = r1;
          R2[at(y)] = r2;
          if constexpr (SC == 0)
            rp[at(y)] = (W)(-r1);
          else
            rp[at(y)] = (W)(-((float)rh * r1));
        } else {
          bres[at(y)] = b;
          rp[at(y)] = r;
        }
      }
      u_m = u_c;
      u_c = u_p;
      w_m = w_c;
      w_c = w_p;
      ayl = ayu;
      aylf = ayuf;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

}  // namespace

template <typename W>
void launch_resid_bres_2d(const double* u, const double* p, const double* F, double* bres, W* rp,
                          double* partials, const double* tab, const float* tabf, const double* cth, double a0,
                          double tau, double h, int n, int logP, long long S, int N, const int* done,
                          const double* jd, Steps<double> sp, cudaStream_t st) {
  const int P = 1 << logP;
  const long long nwarps = (long long)(P / 32) * (P / kRows) * N;
  const double s_h2 = tau / (h * h);
  LaunchScope ls("resid_bres", st, (24.0 + 8.0 + sizeof(W)) * (double)n * n * N);
  const int sc = sp.uniform ? 0 : (sp.rho ? 1 : 2);
#define PT_RESID_BRES(DGV, SCV)                                                                                   \
  k_resid_bres_2d<W, false, DGV, SCV><<<kReduceBlocks, 256, 0, st>>>(u, p, F, bres, rp, partials, tab, tabf, cth, \
                                                                     s_h2 * a0, s_h2, n, logP, S, N, nwarps,    \
                                                                     done, nullptr, nullptr, nullptr, sp, jd)
  if (sizeof(W) == 8 && jd) {
    if (sc == 0) PT_RESID_BRES(true, 0);
    else if (sc == 1) PT_RESID_BRES(true, 1);
    else PT_RESID_BRES(true, 2);
  } else {
    if (sc == 0) PT_RESID_BRES(false, 0);
    else if (sc == 1) PT_RESID_BRES(false, 1);
    else PT_RESID_BRES(false, 2);
  }
#undef PT_RESID_BRES
}

void launch_ir_outer_2d(const double* u, const double* p, const double* F, float* R1, float* R2, float* rp,
                        double* partials, const double* tab, const float* tabf, const double* cth, double a0,
                        double tau, double h, int n, int logP, long long S, int N, Steps<double> sp,
                        const SolveState* st, cudaStream_t s) {
  const int P = 1 << logP;
  const long long nwarps = (long long)(P / 32) * (P / kRows) * N;
  const double s_h2 = tau / (h * h);
  LaunchScope ls("ir_outer", s, (24.0 + 12.0) * (double)n * n * N, 0.0, kOuterStep);
  if (sp.uniform)
    k_resid_bres_2d<float, true, false, 0><<<kReduceBlocks, 256, 0, s>>>(u, p, F, nullptr, rp, partials, tab, tabf,
                                                                         cth, s_h2 * a0, s_h2, n, logP, S, N, nwarps,
                                                                         nullptr, R1, R2, st, sp);
  else
    k_resid_bres_2d<float, true, false, 1><<<kReduceBlocks, 256, 0, s>>>(u, p, F, nullptr, rp, partials, tab, tabf,
                                                                         cth, s_h2 * a0, s_h2, n, logP, S, N, nwarps,
                                                                         nullptr, R1, R2, st, sp);
}

template void launch_resid_bres_2d<float>(const double*, const double*, const double*, double*, float*, double*,
                                          const double*, const float*, const double*, double, double, double, int,
                                          int, long long, int, const int*, const double*, Steps<double>,
                                          cudaStream_t);
template void launch_resid_bres_2d<double>(const double*, const double*, const double*, double*, double*, double*,
                                           const double*, const float*, const double*, double, double, double, int,
                                           int, long long, int, const int*, const double*, Steps<double>,
                                           cudaStream_t);

}  // namespace pt

// ---- FP32 inner step of the mixed-precision refinement, 2-D (n + 1 >= 32) ----
//   b'   = R2 - K du - tau_t A du,    rho_t r_p',  r_p' = K du - tau_t A dp - R1,    partials of ||b'||^2
// (stencils for the reference step tau, times sigma_t = tau_t / tau)
// with the same warp-strip sweep; the per-thread norm is accumulated in FP32 (it only decides
// when the FP64 step is due) and summed in FP64 across the block.
namespace pt {
namespace {

__global__ void __launch_bounds__(256) k_ir_inner_2d(
    const float* __restrict__ du, const float* __restrict__ dp, const float* __restrict__ R1,
    const float* __restrict__ R2, float* __restrict__ bp, float* __restrict__ rp, double* __restrict__ partials,
    const float* __restrict__ tabf, const float* __restrict__ cthf, float a0s, float s_h2, int n, int logP,
    long long S, long long nwarps, Steps<float> sp, const SolveState* st) {
  if (*((volatile const int*)&st->done) != 0 || *((volatile const int*)&st->outer) != 0) return;
  const int P = 1 << logP;
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wg < nwarps;
       wg += (long long)gridDim.x * (blockDim.x >> 5)) {
    const int wx_count = P >> 5, strips = P / kRows;
    const int wx = (int)(wg % wx_count);
    const long long rest = wg / wx_count;
    const int strip = (int)(rest % strips);
    const int t = (int)(rest / strips);
    const int x = (wx << 5) + lane;
    const int y0 = strip * kRows;
    const float* nx = tabf;
    const float* fx = tabf + P;
    const float* ny = tabf + 2 * P;
    const float* fy = tabf + 3 * P;
    const float ct = s_h2 * cthf[t];
    const float sg = sp.sig[t], rh = sp.rho[t];
    const bool xin = x < n;
    const float fxl = fx[x], fxr = fx[x + 1 < P ? x + 1 : x];
    const float gxc = ct * nx[x];
    const long long base = (long long)t * S + x;
    auto at = [&](int y) { return base + (long long)y * P; };
    float d_m = du[at(y0) - P], d_c = du[at(y0)];
    float q_m = dp[at(y0) - P], q_c = dp[at(y0)];
    float ayl = fmaf(gxc, fy[y0], a0s);
    // operands of the next row are loaded one iteration ahead (latency)
    auto ld_row = [&](int y, float& dv, float& qv) {
      dv = 0.f;
      qv = 0.f;
      if (y < P) {
        dv = du[at(y)];
        qv = dp[at(y)];
      }
    };
    auto ld_ctr = [&](int y, float& r1, float& r2, float& dt) {
      r1 = r2 = dt = 0.f;
      if (xin && y < n) {
        const long long i = at(y);
        r1 = R1[i];
        r2 = R2[i];
        dt = t > 0 ? du[i - S] : 0.f;
      }
    };
    float dpn, qpn, r1c, r2c, dtc;
    ld_row(y0 + 1, dpn, qpn);
    ld_ctr(y0, r1c, r2c, dtc);
    for (int k = 0; k < kRows; ++k) {
      const int y = y0 + k;
      const bool yin = y < n;
      const float d_p = dpn, q_p = qpn;
      const float r1 = r1c, r2 = r2c, dtm = dtc;
      ld_row(y + 2, dpn, qpn);
      ld_ctr(y + 1, r1c, r2c, dtc);
      float dW = __shfl_up_sync(0xffffffffu, d_c, 1), dE = __shfl_down_sync(0xffffffffu, d_c, 1);
      float qW = __shfl_up_sync(0xffffffffu, q_c, 1), qE = __shfl_down_sync(0xffffffffu, q_c, 1);
      if (lane == 0 && yin) {
        dW = du[at(y) - 1];
        qW = dp[at(y) - 1];
      }
      if (lane == 31 && yin && x + 1 < P) {
        dE = du[at(y) + 1];
        qE = dp[at(y) + 1];
      }
      const float ayu = fmaf(gxc, fy[y + 1 < P ? y + 1 : y], a0s);
      float b = 0.f, r = 0.f;
      if (xin && yin) {
        const long long i = at(y);
        const float gy = ct * ny[y];
        const float axl = fmaf(gy, fxl, a0s), axr = fmaf(gy, fxr, a0s);
        (void)i;
        const float Kd = d_c - dtm;
        const float sd = axl * (d_c - dW) + axr * (d_c - dE) + ayl * (d_c - d_m) + ayu * (d_c - d_p);
        const float sq = axl * (q_c - qW) + axr * (q_c - qE) + ayl * (q_c - q_m) + ayu * (q_c - q_p);
        b = fmaf(-sg, sd, r2 - Kd);
        r = (fmaf(-sg, sq, Kd) - r1) * rh;
        acc = fmaf(b, b, acc);
      }
      if (y < P) {
        bp[at(y)] = b;
        rp[at(y)] = r;
      }
      d_m = d_c;
      d_c = d_p;
      q_m = q_c;
      q_c = q_p;
      ayl = ayu;
    }
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Streamed form for P >= 256.  A CTA owns a segment of kSegW columns and walks strips of R rows
// of one slot; a producer warp copies, row after row, the du and dp rows (with a 16-byte halo on
// each side) and the R1, R2 and previous-slot du rows into a ring of kStages shared-memory stages
// (one bulk copy per array and row), and eight consumer warps, one column per thread, take the
// x-neighbours from the stage and the y-neighbours from registers.  Stage j of a strip holds the
// du / dp row y0 - 1 + j and the R1 / R2 / du(t-1) row y0 - 2 + j, so the stage that completes the
// 5-point stencil of row y also brings that row's other operands.  The arithmetic is that of
// k_ir_inner_2d, term by term.  The grid is persistent (one wave) and every CTA takes the tasks
// blockIdx.x, blockIdx.x + gridDim.x, ... in order, so the producer runs ahead across strips.
constexpr int kSegW = 256;
constexpr int kStages = 8;
constexpr int kHaloF = 4;
constexpr int kRowDU = kSegW + 2 * kHaloF;

struct IrStage {
  float du[kRowDU];
  float dp[kRowDU];
  float r1[kSegW];
  float r2[kSegW];
  float dt[kSegW];
};
static_assert(sizeof(IrStage) % 16 == 0, "bulk copies need 16-byte aligned stage buffers");

__device__ __forceinline__ void report_timeout(SolveState* st) { *(volatile int*)&st->fault = 1; }

__global__ void __launch_bounds__(kSegW + 32, 4) k_ir_inner_2d_rows(
    const float* __restrict__ du, const float* __restrict__ dp, const float* __restrict__ R1,
    const float* __restrict__ R2, float* __restrict__ bp, float* __restrict__ rp, double* __restrict__ partials,
    const float* __restrict__ tabf, const float* __restrict__ cthf, float a0s, float s_h2, int n, int logP,
    int logR, long long S, int N, Steps<float> sp, SolveState* st) {
  if (*((volatile const int*)&st->done) != 0 || *((volatile const int*)&st->outer) != 0) return;
  __shared__ __align__(128) IrStage stage[kStages];
  __shared__ __align__(8) RowRing<kStages> ring;
  const int P = 1 << logP, R = 1 << logR;
  const int logSeg = logP - 8, logStrips = logP - logR;
  const long long ntasks = (long long)N << (logSeg + logStrips);
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) ring.init(kSegW / 32);
  if (blockIdx.x == 0)
    for (int i = gridDim.x + tid; i < kReduceBlocks; i += blockDim.x) partials[i] = 0.0;
  __syncthreads();
  float acc = 0.f;
  if (tid >= kSegW) {
    // producer warp: one lane issues the copies
    if (lane == 0) {
      bool ok = true;
      unsigned c = 0;
      for (long long task = blockIdx.x; task < ntasks && ok; task += gridDim.x) {
        const int x0 = (int)(task & ((1 << logSeg) - 1)) << 8;
        const long long rest = task >> logSeg;
        const int y0 = (int)(rest & ((1 << logStrips) - 1)) << logR;
        const int t = (int)(rest >> logStrips);
        const long long slot = (long long)t * S;
        for (int j = 0; j < R + 2; ++j, ++c) {
          if (!ring.acquire(c)) {
            ok = false;
            break;
          }
          const int y = y0 - 1 + j, yr = y - 1;
          const bool cp_d = y <= P - 1, cp_r = j >= 2 && yr < n, cp_t = cp_r && t > 0;
          const unsigned bytes = (cp_d ? 2u * kRowDU * 4u : 0u) + (cp_r ? 2u * kSegW * 4u : 0u) +
                                 (cp_t ? (unsigned)kSegW * 4u : 0u);
          uint64_t* bar = ring.commit(c, bytes);
          IrStage& g = stage[c % kStages];
          if (cp_d) {
            const long long o = slot + (long long)y * P + x0 - kHaloF;
            bulk_g2s(g.du, du + o, kRowDU * 4u, bar);
            bulk_g2s(g.dp, dp + o, kRowDU * 4u, bar);
          }
          if (cp_r) {
            const long long o = slot + (long long)yr * P + x0;
            bulk_g2s(g.r1, R1 + o, kSegW * 4u, bar);
            bulk_g2s(g.r2, R2 + o, kSegW * 4u, bar);
            if (cp_t) bulk_g2s(g.dt, du + o - S, kSegW * 4u, bar);
          }
        }
      }
      if (!ok) ring.give_up();
      if (!ring.drain(c)) ok = false;
      if (!ok) report_timeout(st);
    }
    __syncwarp();  // the warp reaches the final block barrier converged
  } else {
    const float* nx = tabf;
    const float* fx = tabf + P;
    const float* ny = tabf + 2 * P;
    const float* fy = tabf + 3 * P;
    bool ok = true;
    unsigned c = 0;
    for (long long task = blockIdx.x; task < ntasks && ok; task += gridDim.x) {
      const int x0 = (int)(task & ((1 << logSeg) - 1)) << 8;
      const long long rest = task >> logSeg;
      const int y0 = (int)(rest & ((1 << logStrips) - 1)) << logR;
      const int t = (int)(rest >> logStrips);
      const int x = x0 + tid;
      const bool xin = x < n;
      const float ct = s_h2 * cthf[t];
      const float sg = sp.sig[t], rh = sp.rho[t];
      const float fxl = fx[x], fxr = fx[x + 1 < P ? x + 1 : x];
      const float gxc = ct * nx[x];
      float* bpt = bp + (long long)t * S + x;
      float* rpt = rp + (long long)t * S + x;
      float d_m = 0.f, d_c = 0.f, dW = 0.f, dE = 0.f, q_m = 0.f, q_c = 0.f, qW = 0.f, qE = 0.f;
      float ayl = fmaf(gxc, fy[y0], a0s);
      for (int j = 0; j < R + 2; ++j, ++c) {
        if (!ring.wait(c)) {
          ok = false;
          break;
        }
        const IrStage& g = stage[c % kStages];
        const float d_pW = g.du[kHaloF - 1 + tid], d_p = g.du[kHaloF + tid], d_pE = g.du[kHaloF + 1 + tid];
        const float q_pW = g.dp[kHaloF - 1 + tid], q_p = g.dp[kHaloF + tid], q_pE = g.dp[kHaloF + 1 + tid];
        const float r1 = g.r1[tid], r2 = g.r2[tid];
        const float dtm = t > 0 ? g.dt[tid] : 0.f;
        ring.release(c);
        if (j >= 2) {
          const int y = y0 + j - 2;
          const bool yin = y < n;
          const float ayu = fmaf(gxc, fy[y + 1 < P ? y + 1 : y], a0s);
          float b = 0.f, r = 0.f;
          if (xin && yin) {
            const float gy = ct * ny[y];
            const float axl = fmaf(gy, fxl, a0s), axr = fmaf(gy, fxr, a0s);
            const float Kd = d_c - dtm;
            const float sd = axl * (d_c - dW) + axr * (d_c - dE) + ayl * (d_c - d_m) + ayu * (d_c - d_p);
            const float sq = axl * (q_c - qW) + axr * (q_c - qE) + ayl * (q_c - q_m) + ayu * (q_c - q_p);
            b = fmaf(-sg, sd, r2 - Kd);
            r = (fmaf(-sg, sq, Kd) - r1) * rh;
            acc = fmaf(b, b, acc);
          }
          bpt[y * P] = b;
          rpt[y * P] = r;
          ayl = ayu;
        }
        d_m = d_c;
        d_c = d_p;
        dW = d_pW;
        dE = d_pE;
        q_m = q_c;
        q_c = q_p;
        qW = q_pW;
        qE = q_pE;
      }
    }
    if (!ok) {
      ring.give_up();
      if (lane == 0) report_timeout(st);
    }
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

void prepare_ir_inner_2d() { resident_grid((const void*)k_ir_inner_2d_rows, kSegW + 32, 0, kReduceBlocks); }

void launch_ir_inner_2d(const float* du, const float* dp, const float* R1, const float* R2, float* bp, float* rp,
                        double* partials, const float* tabf, const float* cthf, double a0, double tau, double h,
                        int n, int logP, long long S, int N, Steps<float> sp, SolveState* st, cudaStream_t s) {
  const int P = 1 << logP;
  const double s_h2 = tau / (h * h);
  LaunchScope ls("ir_inner", s, 24.0 * (double)n * n * N, 0.0, kInnerStep);
  if (P >= kSegW) {
    const int grid = resident_grid((const void*)k_ir_inner_2d_rows, kSegW + 32, 0, kReduceBlocks);
    // strips of 64 rows, shorter while there would be fewer than four tasks per CTA
    int logR = 6;
    while (logR > 4 && ((long long)N << (logP - 8 + logP - logR)) < 4LL * grid) --logR;
    k_ir_inner_2d_rows<<<grid, kSegW + 32, 0, s>>>(du, dp, R1, R2, bp, rp, partials, tabf, cthf,
                                                    (float)(s_h2 * a0), (float)s_h2, n, logP, logR, S, N, sp, st);
    return;
  }
  const long long nwarps = (long long)(P / 32) * (P / kRows) * N;
  k_ir_inner_2d<<<kReduceBlocks, 256, 0, s>>>(du, dp, R1, R2, bp, rp, partials, tabf, cthf, (float)(s_h2 * a0),
                                              (float)s_h2, n, logP, S, nwarps, sp, st);
}

}  // namespace pt

// ---- 3-D forms (n + 1 >= 32) of the two refinement residuals ----
// A warp owns 32 consecutive x of one (y, slot) line and sweeps a strip of kRows z-planes: the
// planes z-1, z, z+1 stay in registers, x-neighbours come from shuffles, y-neighbours are loads
// (the neighbouring warps read the same rows, so they hit in cache).
namespace pt {
namespace {

struct Sweep3 {
  int wx, y, z0, t;
};
__device__ __forceinline__ Sweep3 sweep3_decode(long long wg, int P) {
  const int wx_count = P >> 5, strips = P / kRows;
  Sweep3 s;
  s.wx = (int)(wg % wx_count);
  long long r = wg / wx_count;
  s.y = (int)(r % P);
  r /= P;
  s.z0 = (int)(r % strips) * kRows;
  s.t = (int)(r / strips);
  return s;
}

// FP32 inner step: b' = R2 - K du - tau_t A du, rho_t r_p', r_p' = K du - tau_t A dp - R1
__global__ void __launch_bounds__(256) k_ir_inner_3d(
    const float* __restrict__ du, const float* __restrict__ dp, const float* __restrict__ R1,
    const float* __restrict__ R2, float* __restrict__ bp, float* __restrict__ rp, double* __restrict__ partials,
    const float* __restrict__ tabf, const float* __restrict__ cthf, float a0s, float s_h2, int n, int logP,
    long long S, long long nwarps, Steps<float> sp, const SolveState* st) {
  if (*((volatile const int*)&st->done) != 0 || *((volatile const int*)&st->outer) != 0) return;
  const int P = 1 << logP;
  const long long P2 = (long long)P * P;
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  const float* nx = tabf;
  const float* fx = tabf + P;
  const float* ny = tabf + 2 * P;
  const float* fy = tabf + 3 * P;
  const float* nz = tabf + 4 * P;
  const float* fz = tabf + 5 * P;
  for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wg < nwarps;
       wg += (long long)gridDim.x * (blockDim.x >> 5)) {
    const Sweep3 w = sweep3_decode(wg, P);
    const int x = (w.wx << 5) + lane;
    const bool xyin = x < n && w.y < n;
    const float ct = s_h2 * cthf[w.t];
    const float sg = sp.sig[w.t], rh = sp.rho[w.t];
    const float gx = nx[x], gy = ny[w.y];
    const float fxl = fx[x], fxr = fx[x + 1 < P ? x + 1 : x];
    const float fyl = fy[w.y], fyu = fy[w.y + 1 < P ? w.y + 1 : w.y];
    const float gxy = ct * gx * gy;
    const long long base = (long long)w.t * S + (long long)w.y * P + x;
    auto at = [&](int z) { return base + (long long)z * P2; };
    float d_m = du[at(w.z0) - P2], d_c = du[at(w.z0)];
    float q_m = dp[at(w.z0) - P2], q_c = dp[at(w.z0)];
    float azl = fmaf(gxy, fz[w.z0], a0s);
    for (int k = 0; k < kRows; ++k) {
      const int z = w.z0 + k;
      const bool in = xyin && z < n;
      float d_p = 0.f, q_p = 0.f;
      if (z + 1 < P) {
        d_p = du[at(z + 1)];
        q_p = dp[at(z + 1)];
      }
      float dW = __shfl_up_sync(0xffffffffu, d_c, 1), dE = __shfl_down_sync(0xffffffffu, d_c, 1);
      float qW = __shfl_up_sync(0xffffffffu, q_c, 1), qE = __shfl_down_sync(0xffffffffu, q_c, 1);
      const float azu = fmaf(gxy, fz[z + 1 < P ? z + 1 : z], a0s);
      float b = 0.f, r = 0.f;
      if (in) {
        const long long i = at(z);
        if (lane == 0) {
          dW = du[i - 1];
          qW = dp[i - 1];
        }
        if (lane == 31) {
          dE = du[i + 1];
          qE = dp[i + 1];
        }
        const float dS = du[i - P], dN = du[i + P], qS = dp[i - P], qN = dp[i + P];
        const float gz = ct * nz[z];
        const float gyz = gz * gy, gxz = gz * gx;
        const float axl = fmaf(gyz, fxl, a0s), axr = fmaf(gyz, fxr, a0s);
        const float ayl = fmaf(gxz, fyl, a0s), ayu = fmaf(gxz, fyu, a0s);
        const float Kd = d_c - (w.t > 0 ? du[i - S] : 0.f);
        const float sd = axl * (d_c - dW) + axr * (d_c - dE) + ayl * (d_c - dS) + ayu * (d_c - dN) +
                         azl * (d_c - d_m) + azu * (d_c - d_p);
        const float sq = axl * (q_c - qW) + axr * (q_c - qE) + ayl * (q_c - qS) + ayu * (q_c - qN) +
                         azl * (q_c - q_m) + azu * (q_c - q_p);
        b = fmaf(-sg, sd, R2[i] - Kd);
        r = (fmaf(-sg, sq, Kd) - R1[i]) * rh;
        acc = fmaf(b, b, acc);
      }
      if (z < P) {
        bp[at(z)] = b;
        rp[at(z)] = r;
      }
      d_m = d_c;
      d_c = d_p;
      q_m = q_c;
      q_c = q_p;
      azl = azu;
    }
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// FP64 step: bres = F - K u - tau_t A u (FP64, norm), w = p + u; R1 = bres + tau_t A w (w-stencil in
// FP32), R2 = bres - K^T w, A~ input -rho_t R1
__global__ void __launch_bounds__(256) k_ir_outer_3d(
    const double* __restrict__ u, const double* __restrict__ p, const double* __restrict__ F,
    float* __restrict__ R1, float* __restrict__ R2, float* __restrict__ rp, double* __restrict__ partials,
    const double* __restrict__ tab, const float* __restrict__ tabf, const double* __restrict__ cth,
    double a0s, double s_h2, int n, int logP, long long S, int N, long long nwarps, Steps<double> sp,
    const SolveState* st) {
  if (*((volatile const int*)&st->done) != 0 || !*((volatile const int*)&st->outer)) return;
  const int P = 1 << logP;
  const long long P2 = (long long)P * P;
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  const double* nx = tab;
  const double* fx = tab + P;
  const double* ny = tab + 2 * P;
  const double* fy = tab + 3 * P;
  const double* nz = tab + 4 * P;
  const double* fz = tab + 5 * P;
  const float* fxf = tabf + P;
  const float* fyf = tabf + 3 * P;
  const float* nzf = tabf + 4 * P;
  const float* fzf = tabf + 5 * P;
  const float a0f = (float)a0s;
  for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wg < nwarps;
       wg += (long long)gridDim.x * (blockDim.x >> 5)) {
    const Sweep3 w = sweep3_decode(wg, P);
    const int x = (w.wx << 5) + lane;
    const bool xyin = x < n && w.y < n;
    const double ct = s_h2 * cth[w.t];
    const double sg = sp.sig[w.t];
    const float sgf = (float)sg, rhf = (float)sp.rho[w.t];
    const float ctf = (float)ct;
    const double gx = nx[x], gy = ny[w.y];
    const int xr = x + 1 < P ? x + 1 : x, yu = w.y + 1 < P ? w.y + 1 : w.y;
    const double gxy = ct * gx * gy;
    const float gxf = (float)gx, gyf = (float)gy, gxyf = (float)gxy;
    const long long base = (long long)w.t * S + (long long)w.y * P + x;
    auto at = [&](int z) { return base + (long long)z * P2; };
    auto wv = [&](long long i) { return p[i] + u[i]; };
    double u_m = u[at(w.z0) - P2], u_c = u[at(w.z0)];
    float w_m = (float)wv(at(w.z0) - P2), w_c = (float)wv(at(w.z0));
    double azl = fma(gxy, fz[w.z0], a0s);
    float azlf = fmaf(gxyf, fzf[w.z0], a0f);
    for (int k = 0; k < kRows; ++k) {
      const int z = w.z0 + k;
      const bool in = xyin && z < n;
      double u_p = 0.0;
      float w_p = 0.f;
      if (z + 1 < P) {
        u_p = u[at(z + 1)];
        w_p = (float)wv(at(z + 1));
      }
      double uW = __shfl_up_sync(0xffffffffu, u_c, 1), uE = __shfl_down_sync(0xffffffffu, u_c, 1);
      float wW = __shfl_up_sync(0xffffffffu, w_c, 1), wE = __shfl_down_sync(0xffffffffu, w_c, 1);
      const int zu = z + 1 < P ? z + 1 : z;
      const double azu = fma(gxy, fz[zu], a0s);
      const float azuf = fmaf(gxyf, fzf[zu], a0f);
      float r1 = 0.f, r2 = 0.f;
      if (in) {
        const long long i = at(z);
        if (lane == 0) {
          uW = u[i - 1];
          wW = (float)wv(i - 1);
        }
        if (lane == 31) {
          uE = u[i + 1];
          wE = (float)wv(i + 1);
        }
        const double uS = u[i - P], uN = u[i + P];
        const float wS = (float)wv(i - P), wN = (float)wv(i + P);
        const double gz = ct * nz[z];
        const double gyz = gz * gy, gxz = gz * gx;
        const double axl = fma(gyz, fx[x], a0s), axr = fma(gyz, fx[xr], a0s);
        const double ayl = fma(gxz, fy[w.y], a0s), ayu = fma(gxz, fy[yu], a0s);
        const double su = axl * (u_c - uW) + axr * (u_c - uE) + ayl * (u_c - uS) + ayu * (u_c - uN) +
                          azl * (u_c - u_m) + azu * (u_c - u_p);
        const double um = w.t > 0 ? u[i - S] : 0.0;
        const double b = fma(-sg, su, F[i] - (u_c - um));
        acc = fma(b, b, acc);
        const float gzf = ctf * nzf[z];
        const float gyzf = gzf * gyf, gxzf = gzf * gxf;
        const float axlf = fmaf(gyzf, fxf[x], a0f), axrf = fmaf(gyzf, fxf[xr], a0f);
        const float aylf = fmaf(gxzf, fyf[w.y], a0f), ayuf = fmaf(gxzf, fyf[yu], a0f);
        const float sw = axlf * (w_c - wW) + axrf * (w_c - wE) + aylf * (w_c - wS) + ayuf * (w_c - wN) +
                         azlf * (w_c - w_m) + azuf * (w_c - w_p);
        const double wc = p[i] + u_c;
        const double wn = w.t + 1 < N ? wv(i + S) : 0.0;
        r1 = fmaf(sgf, sw, (float)b);
        r2 = (float)(b - (wc - wn));
      }
      if (z < P) {
        R1[at(z)] = r1;
        R2[at(z)] = r2;
        rp[at(z)] = -(rhf * r1);
      }
      u_m = u_c;
      u_c = u_p;
      w_m = w_c;
      w_c = w_p;
      azl = azu;
      azlf = azuf;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

}  // namespace

namespace {

// Streamed form of the 3-D FP32 step for 32 <= P <= 128: a CTA owns a band of YB = 256 / P rows
// (all P columns) of one slot and walks a strip of R z-planes, one thread per (x, y) of the band.
// Stage j holds the du and dp rows y0 - 1 .. y0 + YB of plane z0 - 1 + j (the band's rows are
// contiguous: one bulk copy per array, with a 16-byte halo before and after) and the R1, R2 and
// previous-slot du rows of the band on plane z0 - 2 + j, so the stage that completes the 7-point
// stencil of plane z also brings that plane's other operands.  x- and y-neighbours come from the
// stage, z-neighbours from registers; the arithmetic is that of k_ir_inner_3d term by term.
constexpr int kBand = 256;
constexpr int kStages3 = 6;

template <int LOGP>
struct IrStage3 {
  static constexpr int P = 1 << LOGP, YB = kBand / P, DU = (YB + 2) * P + 2 * kHaloF;
  float du[DU];
  float dp[DU];
  float r1[kBand];
  float r2[kBand];
  float dt[kBand];
};

template <int LOGP>
__global__ void __launch_bounds__(kBand + 32, 4) k_ir_inner_3d_rows(
    const float* __restrict__ du, const float* __restrict__ dp, const float* __restrict__ R1,
    const float* __restrict__ R2, float* __restrict__ bp, float* __restrict__ rp, double* __restrict__ partials,
    const float* __restrict__ tabf, const float* __restrict__ cthf, float a0s, float s_h2, int n, int logR,
    long long S, int N, Steps<float> sp, SolveState* st) {
  using Stage = IrStage3<LOGP>;
  constexpr int P = Stage::P, YB = Stage::YB, DU = Stage::DU;
  static_assert(sizeof(Stage) % 16 == 0, "bulk copies need 16-byte aligned stage buffers");
  if (*((volatile const int*)&st->done) != 0 || *((volatile const int*)&st->outer) != 0) return;
  __shared__ __align__(128) Stage stage[kStages3];
  __shared__ __align__(8) RowRing<kStages3> ring;
  const int R = 1 << logR;
  constexpr int bands = P / YB;
  const int strips = P >> logR;
  const long long ntasks = (long long)N * bands * strips;
  const long long P2 = (long long)P * P;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) ring.init(kBand / 32);
  if (blockIdx.x == 0)
    for (int i = gridDim.x + tid; i < kReduceBlocks; i += blockDim.x) partials[i] = 0.0;
  __syncthreads();
  float acc = 0.f;
  if (tid >= kBand) {
    if (lane == 0) {
      bool ok = true;
      unsigned c = 0;
      for (long long task = blockIdx.x; task < ntasks && ok; task += gridDim.x) {
        const int y0 = (int)(task % bands) * YB;
        const long long rest = task / bands;
        const int z0 = (int)(rest % strips) << logR;
        const int t = (int)(rest / strips);
        const long long slot = (long long)t * S;
        for (int j = 0; j < R + 2; ++j, ++c) {
          if (!ring.acquire(c)) {
            ok = false;
            break;
          }
          const int z = z0 - 1 + j, zr = z - 1;
          // planes up to P - 1 (the ghost plane as the last z-neighbour); the row after the band
          // is left out when it would be row P (past the slot, past the array for the last slot)
          const bool cp_d = z <= P - 1;
          const unsigned dbytes = (unsigned)(y0 + YB < P ? DU : DU - P) * 4u;
          const bool cp_r = j >= 2 && zr < n, cp_t = cp_r && t > 0;
          const unsigned bytes = (cp_d ? 2u * dbytes : 0u) + (cp_r ? 2u * kBand * 4u : 0u) +
                                 (cp_t ? (unsigned)kBand * 4u : 0u);
          uint64_t* bar = ring.commit(c, bytes);
          Stage& g = stage[c % kStages3];
          if (cp_d) {
            const long long o = slot + ((long long)z * P + y0 - 1) * P - kHaloF;
            bulk_g2s(g.du, du + o, dbytes, bar);
            bulk_g2s(g.dp, dp + o, dbytes, bar);
          }
          if (cp_r) {
            const long long o = slot + ((long long)zr * P + y0) * P;
            bulk_g2s(g.r1, R1 + o, kBand * 4u, bar);
            bulk_g2s(g.r2, R2 + o, kBand * 4u, bar);
            if (cp_t) bulk_g2s(g.dt, du + o - S, kBand * 4u, bar);
          }
        }
      }
      if (!ok) ring.give_up();
      if (!ring.drain(c)) ok = false;
      if (!ok) report_timeout(st);
    }
    __syncwarp();
  } else {
    const float* nx = tabf;
    const float* fx = tabf + P;
    const float* ny = tabf + 2 * P;
    const float* fy = tabf + 3 * P;
    const float* nz = tabf + 4 * P;
    const float* fz = tabf + 5 * P;
    const int x = tid & (P - 1), yl = tid >> LOGP;
    const int sc = kHaloF + (yl + 1) * P + x;  // this thread's point in a stage's du / dp rows
    bool ok = true;
    unsigned c = 0;
    for (long long task = blockIdx.x; task < ntasks && ok; task += gridDim.x) {
      const int y0 = (int)(task % bands) * YB;
      const long long rest = task / bands;
      const int z0 = (int)(rest % strips) << logR;
      const int t = (int)(rest / strips);
      const int y = y0 + yl;
      const bool xyin = x < n && y < n;
      const float ct = s_h2 * cthf[t];
      const float sg = sp.sig[t], rh = sp.rho[t];
      const float gx = nx[x], gy = ny[y];
      const float fxl = fx[x], fxr = fx[x + 1 < P ? x + 1 : x];
      const float fyl = fy[y], fyu = fy[y + 1 < P ? y + 1 : y];
      const float gxy = ct * gx * gy;
      float* bpt = bp + (long long)t * S + (long long)y * P + x;
      float* rpt = rp + (long long)t * S + (long long)y * P + x;
      float d_m = 0.f, d_c = 0.f, dW = 0.f, dE = 0.f, dS = 0.f, dN = 0.f;
      float q_m = 0.f, q_c = 0.f, qW = 0.f, qE = 0.f, qS = 0.f, qN = 0.f;
      float azl = fmaf(gxy, fz[z0], a0s);
      for (int j = 0; j < R + 2; ++j, ++c) {
        if (!ring.wait(c)) {
          ok = false;
          break;
        }
        const Stage& g = stage[c % kStages3];
        const float d_p = g.du[sc], d_pW = g.du[sc - 1], d_pE = g.du[sc + 1], d_pS = g.du[sc - P],
                    d_pN = g.du[sc + P];
        const float q_p = g.dp[sc], q_pW = g.dp[sc - 1], q_pE = g.dp[sc + 1], q_pS = g.dp[sc - P],
                    q_pN = g.dp[sc + P];
        const float r1 = g.r1[tid], r2 = g.r2[tid];
        const float dtm = t > 0 ? g.dt[tid] : 0.f;
        ring.release(c);
        if (j >= 2) {
          const int z = z0 + j - 2;
          const bool in = xyin && z < n;
          const float azu = fmaf(gxy, fz[z + 1 < P ? z + 1 : z], a0s);
          float b = 0.f, r = 0.f;
          if (in) {
            const float gz = ct * nz[z];
            const float gyz = gz * gy, gxz = gz * gx;
            const float axl = fmaf(gyz, fxl, a0s), axr = fmaf(gyz, fxr, a0s);
            const float ayl = fmaf(gxz, fyl, a0s), ayu = fmaf(gxz, fyu, a0s);
            const float Kd = d_c - dtm;
            const float sd = axl * (d_c - dW) + axr * (d_c - dE) + ayl * (d_c - dS) + ayu * (d_c - dN) +
                             azl * (d_c - d_m) + azu * (d_c - d_p);
            const float sq = axl * (q_c - qW) + axr * (q_c - qE) + ayl * (q_c - qS) + ayu * (q_c - qN) +
                             azl * (q_c - q_m) + azu * (q_c - q_p);
            b = fmaf(-sg, sd, r2 - Kd);
            r = (fmaf(-sg, sq, Kd) - r1) * rh;
            acc = fmaf(b, b, acc);
          }
          bpt[z * P2] = b;
          rpt[z * P2] = r;
          azl = azu;
        }
        d_m = d_c;
        d_c = d_p;
        dW = d_pW;
        dE = d_pE;
        dS = d_pS;
        dN = d_pN;
        q_m = q_c;
        q_c = q_p;
        qW = q_pW;
        qE = q_pE;
        qS = q_pS;
        qN = q_pN;
      }
    }
    if (!ok) {
      ring.give_up();
      if (lane == 0) report_timeout(st);
    }
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <int LOGP>
void launch_ir_inner_3d_rows(const float* du, const float* dp, const float* R1, const float* R2, float* bp,
                             float* rp, double* partials, const float* tabf, const float* cthf, float a0s,
                             float s_h2, int n, long long S, int N, Steps<float> sp, SolveState* st, cudaStream_t s) {
  constexpr int P = 1 << LOGP;
  const int grid = resident_grid((const void*)k_ir_inner_3d_rows<LOGP>, kBand + 32, 0, kReduceBlocks);
  // strips of 32 planes, shorter while there would be fewer than four tasks per CTA
  int logR = 5;
  while (logR > 3 && (long long)N * (P / (kBand / P)) * (P >> logR) < 4LL * grid) --logR;
  k_ir_inner_3d_rows<LOGP><<<grid, kBand + 32, 0, s>>>(du, dp, R1, R2, bp, rp, partials, tabf, cthf, a0s, s_h2, n,
                                                      logR, S, N, sp, st);
}

}  // namespace

void prepare_ir_inner_3d() {
  resident_grid((const void*)k_ir_inner_3d_rows<5>, kBand + 32, 0, kReduceBlocks);
  resident_grid((const void*)k_ir_inner_3d_rows<6>, kBand + 32, 0, kReduceBlocks);
  resident_grid((const void*)k_ir_inner_3d_rows<7>, kBand + 32, 0, kReduceBlocks);
}

void launch_ir_inner_3d(const float* du, const float* dp, const float* R1, const float* R2, float* bp, float* rp,
                        double* partials, const float* tabf, const float* cthf, double a0, double tau, double h,
                        int n, int logP, long long S, int N, Steps<float> sp, SolveState* st, cudaStream_t s) {
  const int P = 1 << logP;
  const long long nwarps = (long long)(P / 32) * P * (P / kRows) * N;
  const double s_h2 = tau / (h * h);
  LaunchScope ls("ir_inner", s, 24.0 * (double)n * n * n * N, 0.0, kInnerStep);
  const float a0s = (float)(s_h2 * a0), sh = (float)s_h2;
  if (logP == 5)
    launch_ir_inner_3d_rows<5>(du, dp, R1, R2, bp, rp, partials, tabf, cthf, a0s, sh, n, S, N, sp, st, s);
  else if (logP == 6)
    launch_ir_inner_3d_rows<6>(du, dp, R1, R2, bp, rp, partials, tabf, cthf, a0s, sh, n, S, N, sp, st, s);
  else if (logP == 7)
    launch_ir_inner_3d_rows<7>(du, dp, R1, R2, bp, rp, partials, tabf, cthf, a0s, sh, n, S, N, sp, st, s);
  else
    k_ir_inner_3d<<<kReduceBlocks, 256, 0, s>>>(du, dp, R1, R2, bp, rp, partials, tabf, cthf, a0s, sh, n, logP, S,
                                                nwarps, sp, st);
}

void launch_ir_outer_3d(const double* u, const double* p, const double* F, float* R1, float* R2, float* rp,
                        double* partials, const double* tab, const float* tabf, const double* cth, double a0,
                        double tau, double h, int n, int logP, long long S, int N, Steps<double> sp,
                        const SolveState* st, cudaStream_t s) {
  const int P = 1 << logP;
  const long long nwarps = (long long)(P / 32) * P * (P / kRows) * N;
  const double s_h2 = tau / (h * h);
  LaunchScope ls("ir_outer", s, 36.0 * (double)n * n * n * N, 0.0, kOuterStep);
  k_ir_outer_3d<<<kReduceBlocks, 256, 0, s>>>(u, p, F, R1, R2, rp, partials, tab, tabf, cth, s_h2 * a0, s_h2, n,
                                              logP, S, N, nwarps, sp, st);
}

}  // namespace pt
