// Space-time stencil kernels: layout conversion, the two Uzawa residuals (§3, eq. 3.1), the
// time-global operator B (§2, eq. 2.3-2.4), the Abar apply of the block solve (§4, eq. 4.4)
// and the deterministic FP64 reductions.
#include <cmath>

#include "stencil_common.cuh"

namespace pt {

namespace {

// (K (x) M) u at padded index i of slot t: M (u_t - u_{t-1}), u_{-1} := 0 (§2, eq. 2.3-2.4),
// M the identity or the P1 mass (g.mass)
template <int DIM>
__device__ __forceinline__ double kdiff(const StencilGeom<double>& g, const double* __restrict__ u,
                                        long long i, long long t, double uc) {
  if (g.mass == 0) return uc - (t > 0 ? u[i - g.S] : 0.0);
  double v = mass_p1<DIM, double>(u, i, uc, g.P);
  if (t > 0) v -= mass_p1<DIM, double>(u, i - g.S, u[i - g.S], g.P);
  return v;
}

// out = M v slice by slice (interior points; ghosts written zero)
template <int DIM>
__global__ void k_apply_mass(const double* __restrict__ v, double* __restrict__ out, StencilGeom<double> g,
                             long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    out[i] = decode<DIM>(i, g.logP, g.n, t, x, y, z) ? mass_apply<DIM, double>(g.mass, v, i, v[i], g.P) : 0.0;
  }
}

// out = rho_t M (u_t - u_{t-1}): the A~ input rho_t (K u)_t of the Schur complement apply
template <int DIM>
__global__ void k_apply_K(const double* __restrict__ u, double* __restrict__ out, StencilGeom<double> g,
                          const double* __restrict__ rho, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    out[i] = decode<DIM>(i, g.logP, g.n, t, x, y, z) ? rho[t] * kdiff<DIM>(g, u, i, t, u[i]) : 0.0;
  }
}

// acc += (K^T (x) M)(z + u): M (w_t - w_{t+1}), w = z + u, w_{N} := 0
template <int DIM>
__global__ void k_add_KT(double* __restrict__ acc, const double* __restrict__ zv, const double* __restrict__ u,
                         StencilGeom<double> g, int N, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    if (!decode<DIM>(i, g.logP, g.n, t, x, y, z)) continue;
    double w = mass_apply<DIM, double>(g.mass, zv, i, zv[i], g.P) + mass_apply<DIM, double>(g.mass, u, i, u[i], g.P);
    if (t + 1 < N) {
      const long long j = i + g.S;
      w -= mass_apply<DIM, double>(g.mass, zv, j, zv[j], g.P) + mass_apply<DIM, double>(g.mass, u, j, u[j], g.P);
    }
    acc[i] += w;
  }
}

// x = a x
__global__ void k_scale(double* __restrict__ x, double a, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= a;
}

template <int DIM>
__global__ void k_pack(const double* __restrict__ src, const double* __restrict__ u0,
                       double* __restrict__ dst, double scale, const double* __restrict__ scale_t, int n,
                       int logP, long long total) {
  const long long ns = DIM == 1 ? n : (DIM == 2 ? (long long)n * n : (long long)n * n * n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double v = 0.0;
    if (decode<DIM>(i, logP, n, t, x, y, z)) {
      const long long q = ((long long)z * n + y) * n + x;
      v = (scale_t ? scale_t[t] : scale) * src[t * ns + q];
      if (u0 != nullptr && t == 0) v += u0[q];
    }
    dst[i] = v;
  }
}

// F = scale * (2 U - 1) (+ u0 on slot 0) with U the top 53 bits of SplitMix64 draw q of stream
// `seed`, q the packed index (t * ns + spatial index) of the point: the generator of Steele, Lea &
// Flood (2014) used as a counter-based generator.
template <int DIM>
__global__ void k_pack_uniform(unsigned long long seed, const double* __restrict__ u0,
                               double* __restrict__ dst, double scale, const double* __restrict__ scale_t, int n,
                               int logP, long long total) {
  const long long ns = DIM == 1 ? n : (DIM == 2 ? (long long)n * n : (long long)n * n * n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double v = 0.0;
    if (decode<DIM>(i, logP, n, t, x, y, z)) {
      const long long q = ((long long)z * n + y) * n + x;
      unsigned long long h = seed + ((unsigned long long)(t * ns + q) + 1ull) * 0x9E3779B97F4A7C15ull;
      h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
      h = (h ^ (h >> 27)) * 0x94D049BB133111EBull;
      h ^= h >> 31;
      const double uni = (double)(h >> 11) * (1.0 / 9007199254740992.0);
      v = (scale_t ? scale_t[t] : scale) * (2.0 * uni - 1.0);
      if (u0 != nullptr && t == 0) v += u0[q];
    }
    dst[i] = v;
  }
}

template <int DIM, typename T>
__global__ void k_pack_typed(const double* __restrict__ src, T* __restrict__ dst, int n, int logP,
                             long long total) {
  const long long ns = DIM == 1 ? n : (DIM == 2 ? (long long)n * n : (long long)n * n * n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    T v = (T)0;
    if (decode<DIM>(i, logP, n, t, x, y, z)) v = (T)src[t * ns + ((long long)z * n + y) * n + x];
    dst[i] = v;
  }
}

template <int DIM, typename T>
__global__ void k_unpack(const T* __restrict__ src, double* __restrict__ dst, int n, int logP,
                         long long S, long long total_packed) {
  const long long ns = DIM == 1 ? n : (DIM == 2 ? (long long)n * n : (long long)n * n * n);
  const int P = 1 << logP;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total_packed;
       q += (long long)gridDim.x * blockDim.x) {
    const long long t = q / ns;
    long long r = q - t * ns;
    const int x = (int)(r % n);
    r /= n;
    const int y = DIM >= 2 ? (int)(r % n) : 0;
    const int z = DIM >= 3 ? (int)(r / n) : 0;
    dst[q] = (double)src[t * S + ((long long)z * P + y) * P + x];
  }
}

template <int DIM>
__global__ void k_apply_B(const double* __restrict__ u, double* __restrict__ out,
                          StencilGeom<double> g, const double* __restrict__ cth, Steps<double> sp,
                          long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double v = 0.0;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      double am[3], ap[3];
      face_coefs<DIM, double>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const double uc = u[i];
      const double Au = stencil_sum<DIM, double>(u, i, uc, am, ap, g.P) * g.h2inv;
      v = kdiff<DIM>(g, u, i, t, uc) + sp.tau[t] * Au;
    }
    out[i] = v;
  }
}

// rho_t r_p, r_p = K u - tau_t A_t p - F  (first line of eq. 3.1; rho_t makes the A~ input of
// the V-cycle for tau A_t that of tau_t A_t)
template <int DIM, typename Tp>
__global__ void k_resid_p(const double* __restrict__ u, const double* __restrict__ p,
                          const double* __restrict__ F, Tp* __restrict__ rp, StencilGeom<double> g,
                          const double* __restrict__ cth, Steps<double> sp, long long total,
                          const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double v = 0.0;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      double am[3], ap[3];
      face_coefs<DIM, double>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const double pc = p[i];
      const double Ap = stencil_sum<DIM, double>(p, i, pc, am, ap, g.P) * g.h2inv;
      v = (kdiff<DIM>(g, u, i, t, u[i]) - sp.tau[t] * Ap - F[i]) * sp.rho[t];
    }
    rp[i] = (Tp)v;
  }
}

// r_u = F - K^T p - (K + K^T + A) u = (F - B u) - K^T (p + u)  (second line of eq. 3.1),
// plus per-block partial sums of ||F - B u||^2.
template <int DIM, typename Tp>
__global__ void k_resid_u(const double* __restrict__ u, const double* __restrict__ p,
                          const double* __restrict__ F, Tp* __restrict__ ru,
                          double* __restrict__ partials, StencilGeom<double> g,
                          const double* __restrict__ cth, Steps<double> sp, int N, long long total,
                          const int* done) {
  if (stop_requested(done)) return;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double v = 0.0;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      double am[3], ap[3];
      face_coefs<DIM, double>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const double uc = u[i];
      const double Au = stencil_sum<DIM, double>(u, i, uc, am, ap, g.P) * g.h2inv;
      const double bres = F[i] - kdiff<DIM>(g, u, i, t, uc) - sp.tau[t] * Au;
      acc += bres * bres;
      if (g.mass == 0) {
        const double next = t + 1 < N ? p[i + g.S] + u[i + g.S] : 0.0;
        v = bres - (p[i] + uc) + next;
      } else {  // M (w_t - w_{t+1}), w = p + u
        double mw = mass_p1<DIM, double>(p, i, p[i], g.P) + mass_p1<DIM, double>(u, i, uc, g.P);
        if (t + 1 < N) {
          const long long j = i + g.S;
          mw -= mass_p1<DIM, double>(p, j, p[j], g.P) + mass_p1<DIM, double>(u, j, u[j], g.P);
        }
        v = bres - mw;
      }
    }
    ru[i] = (Tp)v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Mixed precision, first half of an iteration: the outer residual bres = F - K u - tau_t A_t u in
// FP64 (stored, with its squared-norm partials), and the A~ input rho_t r_p,
//   r_p = K u - tau_t A_t p - F = -bres - tau_t A_t (p + u)
// whose second term is a stencil on w = p + u, a quantity that tends to zero, taken in FP32.
template <int DIM>
__global__ void k_resid_bres_mixed(const double* __restrict__ u, const double* __restrict__ p,
                                   const double* __restrict__ F, double* __restrict__ bres,
                                   float* __restrict__ rp, double* __restrict__ partials,
                                   StencilGeom<double> g, const double* __restrict__ cth, Steps<double> sp,
                                   long long total, const int* done) {
  if (stop_requested(done)) return;
  double acc = 0.0;
  const float h2f = (float)g.h2inv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    double b = 0.0;
    float r = 0.f;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, z)) {
      double am[3], ap[3];
      face_coefs<DIM, double>(g.tab, g.P, x, y, z, cth[t], g.a0, am, ap);
      const double uc = u[i];
      const double Au = stencil_sum<DIM, double>(u, i, uc, am, ap, g.P) * g.h2inv;
      const double um = t > 0 ? u[i - g.S] : 0.0;
      const double tau = sp.tau[t];
      b = F[i] - (uc - um) - tau * Au;
      acc += b * b;
      const float tauf = (float)tau;
      const float wc = (float)(p[i] + uc);
      long long off[3] = {1, g.P, (long long)g.P * g.P};
      float aw = 0.f;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const float wm = (float)(p[i - off[d]] + u[i - off[d]]);
        const float wp = (float)(p[i + off[d]] + u[i + off[d]]);
        aw += (float)am[d] * (wc - wm) + (float)ap[d] * (wc - wp);
      }
      r = ((float)(-b) - tauf * h2f * aw) * (float)sp.rho[t];
    }
    bres[i] = b;
    rp[i] = r;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Second residual without a stencil: r_u = bres - K^T (p + u), or its negative (NEG; the Krylov
// path's saddle operator).  The sign is a template parameter: a run-time factor would cost an
// FP64 multiply per point.
template <typename Tp, bool NEG>
__global__ void k_resid_u_from_bres(const double* __restrict__ bres, const double* __restrict__ u,
                                    const double* __restrict__ p, Tp* __restrict__ ru, long long S,
                                    long long total, const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double next = i + S < total ? p[i + S] + u[i + S] : 0.0;
    const double v = NEG ? (p[i] + u[i]) - next - bres[i] : bres[i] - (p[i] + u[i]) + next;
    ru[i] = (Tp)v;
  }
}

template <int DIM, typename T>
__global__ void k_apply_A_scaled(const T* __restrict__ z, T* __restrict__ out, StencilGeom<T> g,
                                 T cth, T scale, long long total, const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, zz;
    T v = (T)0;
    if (decode<DIM>(i, g.logP, g.n, t, x, y, zz)) {
      T am[3], ap[3];
      face_coefs<DIM, T>(g.tab, g.P, x, y, zz, cth, g.a0, am, ap);
      const T zc = z[i];
      v = scale * g.h2inv * stencil_sum<DIM, T>(z, i, zc, am, ap, g.P);
    }
    out[i] = v;
  }
}

__global__ void k_norm2_partials(const double* __restrict__ v, long long count,
                                 double* __restrict__ partials) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    acc += v[i] * v[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// One block of kReduceBlocks threads sums the partials in a fixed order; the iteration index,
// tolerance and iteration limit live in the state, so the launch is the same every iteration.
__global__ void k_finalize_residual(const double* __restrict__ partials, SolveState* state,
                                    double* __restrict__ hist) {
  if (state->done) return;
  if (state->fault) {
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
    if (!(res <= 1e30)) {  // NaN or overflow
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
  }
}

// start of a solve: ||F||^2 from the partials, counters reset
__global__ void k_finalize_fnorm(const double* __restrict__ partials, SolveState* state, double tol,
                                 int max_it) {
  double v = partials[threadIdx.x];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    state->fnorm2 = v > 0.0 ? v : 1.0;
    state->done = 0;
    state->status = PT_ENOTCONV;
    state->iters = 0;
    state->j = 0;
    state->tol = tol;
    state->max_it = max_it;
    state->last_res = 1.0;
    state->fault = 0;
  }
}

__global__ void k_gather_done(SolveState* const* __restrict__ states, int count, int* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = states[i]->done == 1;
}

// Control of the device-side batch loop (the body of a conditional WHILE graph node holds one
// iteration of every active problem and this kernel): counts the active problems that have not
// finished, advances the round counter, and keeps the loop going while more than `keep_above`
// are unfinished and fewer than `limit` rounds have run (the limit bounds the loop on the device
// whatever the states say).  One block.
__global__ void k_batch_control(SolveState* const* __restrict__ states, const int* __restrict__ idx, int count,
                                int keep_above, int* __restrict__ rounds, int limit,
                                cudaGraphConditionalHandle handle) {
  int open = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) open += states[idx[i]]->done != 1;
  const double total = block_sum((double)open);
  if (threadIdx.x == 0) {
    const int r = ++(*rounds);
    cudaGraphSetConditional(handle, ((int)total > keep_above && r < limit) ? 1u : 0u);
  }
}

// x[i] *= f[i >> logS]: one factor per slot of 2^logS elements
template <typename T>
__global__ void k_scale_slices(T* __restrict__ x, const T* __restrict__ f, int logS, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= f[i >> logS];
}

template <typename Tp>
__global__ void k_axpy(double* __restrict__ y, const Tp* __restrict__ x, double a, long long count,
                       const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += a * (double)x[i];
}

}  // namespace

#define PT_DISPATCH_DIM(dim, ...)                 \
  switch (dim) {                                  \
    case 1: {                                     \
      constexpr int D = 1;                        \
      __VA_ARGS__;                                \
    } break;                                      \
    case 2: {                                     \
      constexpr int D = 2;                        \
      __VA_ARGS__;                                \
    } break;                                      \
    default: {                                    \
      constexpr int D = 3;                        \
      __VA_ARGS__;                                \
    } break;                                      \
  }

inline double dofs(int dim, int n, int N) {
  double d = N;
  for (int k = 0; k < dim; ++k) d *= n;
  return d;
}

void launch_pack(const double* src, const double* u0, double* dst, double scale, const double* scale_t, int dim,
                 int n, int P, int logP, long long S, int N, cudaStream_t st) {
  (void)P;
  const long long total = S * N;
  LaunchScope ls("pack", st, 16.0 * dofs(dim, n, N));
  PT_DISPATCH_DIM(dim, k_pack<D><<<grid_for(total), kThreads, 0, st>>>(src, u0, dst, scale, scale_t, n, logP, total));
}

void launch_pack_uniform(unsigned long long seed, const double* u0, double* dst, double scale,
                         const double* scale_t, int dim, int n, int logP, long long S, int N, cudaStream_t st) {
  const long long total = S * N;
  LaunchScope ls("pack", st, 8.0 * dofs(dim, n, N));
  PT_DISPATCH_DIM(dim, k_pack_uniform<D><<<grid_for(total), kThreads, 0, st>>>(seed, u0, dst, scale, scale_t, n,
                                                                               logP, total));
}

template <typename T>
void launch_pack_typed(const double* src, T* dst, int dim, int n, int P, int logP, long long S,
                       int N, cudaStream_t st) {
  (void)P;
  const long long total = S * N;
  LaunchScope ls("pack", st, (8.0 + sizeof(T)) * dofs(dim, n, N));
  PT_DISPATCH_DIM(dim, k_pack_typed<D, T><<<grid_for(total), kThreads, 0, st>>>(src, dst, n, logP, total));
}

template <typename T>
void launch_unpack(const T* src, double* dst, int dim, int n, int P, int logP, long long S, int N,
                   cudaStream_t st) {
  (void)P;
  long long ns = n;
  for (int d = 1; d < dim; ++d) ns *= n;
  const long long total = ns * N;
  LaunchScope ls("unpack", st, (8.0 + sizeof(T)) * (double)total);
  PT_DISPATCH_DIM(dim, k_unpack<D, T><<<grid_for(total), kThreads, 0, st>>>(src, dst, n, logP, S, total));
}

void launch_apply_B(const double* u, double* out, StencilGeom<double> g, const double* cth, Steps<double> sp,
                    int N, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("apply_B", st, 16.0 * dofs(g.dim, g.n, N));
  PT_DISPATCH_DIM(g.dim, k_apply_B<D><<<grid_for(total), kThreads, 0, st>>>(u, out, g, cth, sp, total));
}

template <typename Tp>
void launch_resid_p(const double* u, const double* p, const double* F, Tp* rp, StencilGeom<double> g,
                    const double* cth, Steps<double> sp, int N, const int* done, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("resid_p", st, (24.0 + sizeof(Tp)) * dofs(g.dim, g.n, N));
  PT_DISPATCH_DIM(g.dim, k_resid_p<D, Tp><<<grid_for(total), kThreads, 0, st>>>(u, p, F, rp, g, cth, sp, total, done));
}

template <typename Tp>
void launch_resid_u(const double* u, const double* p, const double* F, Tp* ru, double* partials,
                    StencilGeom<double> g, const double* cth, Steps<double> sp, int N, const int* done,
                    cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("resid_u", st, (24.0 + sizeof(Tp)) * dofs(g.dim, g.n, N));
  PT_DISPATCH_DIM(g.dim, k_resid_u<D, Tp><<<kReduceBlocks, kThreads, 0, st>>>(u, p, F, ru, partials, g, cth, sp, N, total, done));
}

void launch_resid_bres_mixed(const double* u, const double* p, const double* F, double* bres, float* rp,
                             double* partials, StencilGeom<double> g, const double* cth, Steps<double> sp, int N,
                             const int* done, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("resid_bres", st, (24.0 + 8.0 + 4.0) * dofs(g.dim, g.n, N));
  PT_DISPATCH_DIM(g.dim, k_resid_bres_mixed<D><<<kReduceBlocks, kThreads, 0, st>>>(u, p, F, bres, rp, partials, g, cth, sp, total, done));
}

template <typename Tp>
void launch_resid_u_from_bres(const double* bres, const double* u, const double* p, Tp* ru, long long S,
                              int N, int dim, int n, const int* done, cudaStream_t st, double sgn) {
  const long long total = S * N;
  LaunchScope ls("resid_u_bres", st, (24.0 + sizeof(Tp)) * dofs(dim, n, N));
  if (sgn < 0.0)
    k_resid_u_from_bres<Tp, true><<<grid_for(total), kThreads, 0, st>>>(bres, u, p, ru, S, total, done);
  else
    k_resid_u_from_bres<Tp, false><<<grid_for(total), kThreads, 0, st>>>(bres, u, p, ru, S, total, done);
}
template void launch_resid_u_from_bres<float>(const double*, const double*, const double*, float*, long long, int,
                                              int, int, const int*, cudaStream_t, double);
template void launch_resid_u_from_bres<double>(const double*, const double*, const double*, double*, long long, int,
                                               int, int, const int*, cudaStream_t, double);

template <typename T>
void launch_apply_A_scaled(const T* z, T* out, StencilGeom<T> g, T cth, T scale, int N,
                           const int* done, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("apply_Abar", st, 2.0 * sizeof(T) * dofs(g.dim, g.n, N));
  PT_DISPATCH_DIM(g.dim, k_apply_A_scaled<D, T><<<grid_for(total), kThreads, 0, st>>>(z, out, g, cth, scale, total, done));
}

void launch_apply_mass(const double* v, double* out, StencilGeom<double> g, int N, cudaStream_t st) {
  const long long total = g.S * N;
  double d = N;
  for (int k = 0; k < g.dim; ++k) d *= g.n;
  LaunchScope ls("apply_mass", st, 16.0 * d);
  PT_DISPATCH_DIM(g.dim, k_apply_mass<D><<<grid_for(total), kThreads, 0, st>>>(v, out, g, total));
}

void launch_apply_K(const double* u, double* out, StencilGeom<double> g, const double* rho, int N, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("apply_K", st, 16.0 * (double)total);
  PT_DISPATCH_DIM(g.dim, k_apply_K<D><<<grid_for(total), kThreads, 0, st>>>(u, out, g, rho, total));
}

void launch_add_KT(double* acc, const double* z, const double* u, StencilGeom<double> g, int N, cudaStream_t st) {
  const long long total = g.S * N;
  LaunchScope ls("add_KT", st, 32.0 * (double)total);
  PT_DISPATCH_DIM(g.dim, k_add_KT<D><<<grid_for(total), kThreads, 0, st>>>(acc, z, u, g, N, total));
}

void launch_scale(double* x, double a, long long total, cudaStream_t st) {
  LaunchScope ls("scale", st, 16.0 * (double)total);
  k_scale<<<grid_for(total), kThreads, 0, st>>>(x, a, total);
}

void launch_norm2_partials(const double* v, long long count, double* partials, cudaStream_t st) {
  LaunchScope ls("norm2", st, 8.0 * (double)count);
  k_norm2_partials<<<kReduceBlocks, kThreads, 0, st>>>(v, count, partials);
}

void launch_finalize_residual(const double* partials, SolveState* state, double* hist, cudaStream_t st) {
  LaunchScope ls("finalize", st, 8.0 * kReduceBlocks);
  k_finalize_residual<<<1, kReduceBlocks, 0, st>>>(partials, state, hist);
}

void launch_finalize_fnorm(const double* partials, SolveState* state, double tol, int max_it,
                           cudaStream_t st) {
  LaunchScope ls("finalize", st, 8.0 * kReduceBlocks);
  k_finalize_fnorm<<<1, kReduceBlocks, 0, st>>>(partials, state, tol, max_it);
}

void launch_batch_control(SolveState* const* states, const int* idx, int count, int keep_above, int* rounds,
                          int limit, cudaGraphConditionalHandle handle, cudaStream_t st) {
  LaunchScope ls("batch_control", st, 0.0);
  k_batch_control<<<1, 256, 0, st>>>(states, idx, count, keep_above, rounds, limit, handle);
}

void launch_gather_done(SolveState* const* states, int count, int* out, cudaStream_t st) {
  LaunchScope ls("gather_done", st, 12.0 * count);
  k_gather_done<<<(count + 255) / 256, 256, 0, st>>>(states, count, out);
}

template <typename T>
void launch_scale_slices(T* x, const T* f, int logS, long long total, cudaStream_t st) {
  LaunchScope ls("scale_slices", st, 2.0 * sizeof(T) * (double)total);
  k_scale_slices<T><<<grid_for(total), kThreads, 0, st>>>(x, f, logS, total);
}
template void launch_scale_slices<float>(float*, const float*, int, long long, cudaStream_t);
template void launch_scale_slices<double>(double*, const double*, int, long long, cudaStream_t);

template <typename Tp>
void launch_axpy(double* y, const Tp* x, double a, long long count, const int* done, cudaStream_t st) {
  LaunchScope ls("axpy", st, (16.0 + sizeof(Tp)) * (double)count);
  k_axpy<Tp><<<grid_for(count), kThreads, 0, st>>>(y, x, a, count, done);
}

template void launch_pack_typed<float>(const double*, float*, int, int, int, int, long long, int, cudaStream_t);
template void launch_pack_typed<double>(const double*, double*, int, int, int, int, long long, int, cudaStream_t);
template void launch_unpack<float>(const float*, double*, int, int, int, int, long long, int, cudaStream_t);
template void launch_unpack<double>(const double*, double*, int, int, int, int, long long, int, cudaStream_t);
template void launch_resid_p<float>(const double*, const double*, const double*, float*, StencilGeom<double>, const double*, Steps<double>, int, const int*, cudaStream_t);
template void launch_resid_p<double>(const double*, const double*, const double*, double*, StencilGeom<double>, const double*, Steps<double>, int, const int*, cudaStream_t);
template void launch_resid_u<float>(const double*, const double*, const double*, float*, double*, StencilGeom<double>, const double*, Steps<double>, int, const int*, cudaStream_t);
template void launch_resid_u<double>(const double*, const double*, const double*, double*, double*, StencilGeom<double>, const double*, Steps<double>, int, const int*, cudaStream_t);
template void launch_apply_A_scaled<float>(const float*, float*, StencilGeom<float>, float, float, int, const int*, cudaStream_t);
template void launch_apply_A_scaled<double>(const double*, double*, StencilGeom<double>, double, double, int, const int*, cudaStream_t);
template void launch_axpy<float>(double*, const float*, double, long long, const int*, cudaStream_t);
template void launch_axpy<double>(double*, const double*, double, long long, const int*, cudaStream_t);

}  // namespace pt
