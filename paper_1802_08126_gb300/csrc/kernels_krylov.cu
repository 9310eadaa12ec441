// Kernels of the Krylov-accelerated form of the method (flexible GMRES(m) right-preconditioned by
// one inexact Uzawa step; the Krylov acceleration the paper applies in its 3-D experiments, §8.3).
// Every vector is a pair (p, u) of padded FP64 space-time vectors; the saddle-point operator of
// eq. 2.7 in the form the Uzawa iteration solves is
//     Sad (p, u) = ( -tau A p + K u ,  K^T p + (K^T + B) u ),   B = K + tau A,
// with tau A = diag(tau_n A_n).
#include "stencil_common.cuh"

namespace pt {
namespace {

template <int DIM>
__global__ void k_apply_saddle(const double* __restrict__ zp, const double* __restrict__ zu,
                               double* __restrict__ op, double* __restrict__ ou, StencilGeom<double> g,
                               const double* __restrict__ cth, Steps<double> sp, int N, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double r1 = 0.0, r2 = 0.0;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      double am[3], ap[3];
      face_coefs<DIM, double>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const double pc = zp[i], uc = zu[i];
      const double tau = sp.tau[t];
      const double Ap = tau * g.h2inv * stencil_sum<DIM, double>(zp, i, pc, am, ap, g.P);
      const double Au = tau * g.h2inv * stencil_sum<DIM, double>(zu, i, uc, am, ap, g.P);
      const double Ku = uc - (t > 0 ? zu[i - g.S] : 0.0);
      const double wc = pc + uc;
      const double wn = t + 1 < N ? zp[i + g.S] + zu[i + g.S] : 0.0;
      r1 = Ku - Ap;
      r2 = (wc - wn) + Ku + Au;
    }
    op[i] = r1;
    ou[i] = r2;
  }
}

// partials[k][block] of <w, v_k> over both halves of the pairs, k < nv, and (self) of <w, w> in
// row nv.  w is read once per chunk of kChunk vectors (blockIdx.y picks the chunk).  On this GPU
// the two FP64 multiply-adds per element and vector bound the kernel, not the bytes.
constexpr int kChunk = 8;
__global__ void __launch_bounds__(256) k_multidot(const double* const* __restrict__ vp,
                                                  const double* const* __restrict__ vu,
                                                  const double* __restrict__ wp, const double* __restrict__ wu,
                                                  int nv, int self, long long total, double* __restrict__ partials) {
  __shared__ double red[kChunk + 1][8];
  const int k0 = blockIdx.y * kChunk;
  const int nk = min(kChunk, nv - k0);
  const bool do_self = self && blockIdx.y == 0;
  double acc[kChunk + 1];
  const double* pp[kChunk];
  const double* pu[kChunk];
#pragma unroll
  for (int q = 0; q <= kChunk; ++q) acc[q] = 0.0;
#pragma unroll
  for (int q = 0; q < kChunk; ++q) {
    pp[q] = q < nk ? vp[k0 + q] : wp;
    pu[q] = q < nk ? vu[k0 + q] : wu;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = wp[i], b = wu[i];
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nk) acc[q] = fma(pp[q][i], a, fma(pu[q][i], b, acc[q]));
    if (do_self) acc[kChunk] = fma(a, a, fma(b, b, acc[kChunk]));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q <= kChunk; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x <= kChunk) {
    const int q = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[q][w];
    if (q < nk) partials[(long long)(k0 + q) * gridDim.x + blockIdx.x] = v;
    if (q == kChunk && do_self) partials[(long long)nv * gridDim.x + blockIdx.x] = v;
  }
}

// (wp, wu) += sum_k c_k (vp_k, vu_k)
__global__ void k_multiaxpy(const double* const* __restrict__ vp, const double* const* __restrict__ vu,
                            const double* __restrict__ c, int nv, double* __restrict__ wp, double* __restrict__ wu,
                            long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    double sp = wp[i], su = wu[i];
    for (int k = 0; k < nv; ++k) {
      sp = fma(c[k], vp[k][i], sp);
      su = fma(c[k], vu[k][i], su);
    }
    wp[i] = sp;
    wu[i] = su;
  }
}

// (yp, yu) = s (xp, xu), times rho[i >> logS] when rho is not null
__global__ void k_scale_pair(const double* __restrict__ xp, const double* __restrict__ xu, double s,
                             double* __restrict__ yp, double* __restrict__ yu, long long total,
                             const double* __restrict__ rho, int logS) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double f = rho ? s * rho[i >> logS] : s;
    yp[i] = f * xp[i];
    yu[i] = f * xu[i];
  }
}

// ru = vu - K^T zp  (the second block of the Uzawa step's right-hand side), zp = -A~^-1 vp given
__global__ void k_uzawa_ru(const double* __restrict__ vu, const double* __restrict__ zp, double* __restrict__ ru,
                           long long S, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double next = i + S < total ? zp[i + S] : 0.0;
    ru[i] = vu[i] - (zp[i] - next);
  }
}

}  // namespace

void launch_apply_saddle(const double* zp, const double* zu, double* op, double* ou, StencilGeom<double> g,
                         const double* cth, Steps<double> sp, int N, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("krylov_apply", st, 48.0 * (double)total);
  switch (g.dim) {
    case 1: k_apply_saddle<1><<<grid_for(total), kThreads, 0, st>>>(zp, zu, op, ou, g, cth, sp, N, total); break;
    case 2: k_apply_saddle<2><<<grid_for(total), kThreads, 0, st>>>(zp, zu, op, ou, g, cth, sp, N, total); break;
    default: k_apply_saddle<3><<<grid_for(total), kThreads, 0, st>>>(zp, zu, op, ou, g, cth, sp, N, total); break;
  }
}

void launch_multidot(const double* const* vp, const double* const* vu, const double* wp, const double* wu, int nv,
                     int self, long long total, double* partials, cudaStream_t st) {
  LaunchScope ls("krylov_dot", st, 16.0 * (nv + 1) * (double)total);
  const dim3 grid(kReduceBlocks, (unsigned)((nv + kChunk - 1) / kChunk > 0 ? (nv + kChunk - 1) / kChunk : 1));
  k_multidot<<<grid, 256, 0, st>>>(vp, vu, wp, wu, nv, self, total, partials);
}

void launch_multiaxpy(const double* const* vp, const double* const* vu, const double* c, int nv, double* wp,
                      double* wu, long long total, cudaStream_t st) {
  LaunchScope ls("krylov_axpy", st, 16.0 * (nv + 2) * (double)total);
  k_multiaxpy<<<grid_for(total), kThreads, 0, st>>>(vp, vu, c, nv, wp, wu, total);
}

void launch_scale_pair(const double* xp, const double* xu, double s, double* yp, double* yu, long long total,
                       cudaStream_t st, const double* rho, int logS) {
  LaunchScope ls("krylov_scale", st, 32.0 * (double)total);
  k_scale_pair<<<grid_for(total), kThreads, 0, st>>>(xp, xu, s, yp, yu, total, rho, logS);
}

void launch_uzawa_ru(const double* vu, const double* zp, double* ru, long long S, int N, cudaStream_t st) {
  const long long total = S * N;
  LaunchScope ls("krylov_ru", st, 24.0 * (double)total);
  k_uzawa_ru<<<grid_for(total), kThreads, 0, st>>>(vu, zp, ru, S, total);
}

}  // namespace pt
