// Temporal change of basis of the preconditioner (§4, eq. 4.2-4.4): for every spatial point,
//   forward  (Phi^-T):  rhat_k = sum_{n=1}^N r_n sin((2k-1) n pi / (2N)),   k = 1..N,
//   inverse  (Phi^-1):  u_n    = sum_{k=1}^N y_k sin((2k-1) n pi / (2N)),   n = 1..N,
// computed with an N-point complex FFT (the fast splitting §5 refers to), not as sums.
//
// Both are reduced to cosine transforms by reflecting the time index (n' = N - n):
//   inverse: u_{N-m} = sum_j z_j cos(pi (2j+1) m / (2N)) with z_j = (-1)^j y_{j+1}   (DCT-II of z)
//   forward: rhat_{j+1} = (-1)^j sum_m w_m cos(pi (2j+1) m / (2N)), w_m = r_{N-m}     (DCT-III of w)
// and the cosine transforms are computed through one complex FFT of length N (Makhoul, IEEE
// Trans. ASSP 28, 1980): the DCT-II permutes v_j = z_{2j}, v_{N-1-j} = z_{2j+1}, transforms,
// and takes Re(e^{-i pi m/(2N)} V_m); the DCT-III runs those steps backwards.  Two real columns
// share one complex FFT (real and imaginary parts).  The FFT is a radix-2 decimation-in-
// frequency transform in shared memory (natural order in, bit-reversed order out).
//
// A CTA owns W = 2C consecutive padded spatial columns for all N time slots, so the transform
// is done in place with no inter-CTA dependency.  N must be a power of two.
#include <algorithm>
#include <cmath>

#include "fft_common.cuh"

namespace pt {

namespace {

// Geometry of the padded columns: a column whose spatial coordinates include the ghost index n
// must stay exactly zero.  (Two real columns share one complex FFT; rounding would otherwise
// leak a few ulps of the interior partner into a ghost column.)
struct ColGeom {
  int dim, n, logP;
};

__device__ __forceinline__ bool ghost_col(ColGeom g, long long col) {
  const int P = 1 << g.logP;
  const int x = (int)(col & (P - 1));
  const int y = g.dim >= 2 ? (int)((col >> g.logP) & (P - 1)) : 0;
  const int z = g.dim >= 3 ? (int)((col >> (2 * g.logP)) & (P - 1)) : 0;
  return x == g.n || y == g.n || z == g.n;
}

// N-point DFT X_k = sum_n x_n e^{sgn 2 pi i n k / N} of C columns for any N (Bluestein's
// chirp-z): with c_m = e^{i pi m^2 / N} and w = conj(c) (sgn < 0) or c (sgn > 0),
// X_k = w_k sum_n (x_n w_n) conj(w)_{k-n}, the convolution done by two M-point FFTs
// (M a power of two >= 2N - 1) and the precomputed spectrum of the chirp, stored in
// bit-reversed order and divided by M.  In and out in natural order, columns of stride L.
template <typename T, typename T2>
__device__ __forceinline__ void bluestein(T2* buf, int C, int L, const DstPlan<T>& p, T sgn) {
  const T2* chirp = (const T2*)p.chirp;
  const T2* filt = (const T2*)(sgn < (T)0 ? p.gfwd : p.ginv);
  const T2* twM = (const T2*)p.twM;
  for (int idx = threadIdx.x; idx < C * p.M; idx += blockDim.x) {
    const int c = idx / p.M, m = idx - c * p.M;
    T2* col = buf + (size_t)c * L;
    T2 v;
    if (m < p.N) {
      const T2 x = col[m];
      const T2 w = chirp[m];
      const T wi = sgn < (T)0 ? -w.y : w.y;
      v.x = x.x * w.x - x.y * wi;
      v.y = x.x * wi + x.y * w.x;
    } else {
      v.x = (T)0;
      v.y = (T)0;
    }
    col[m] = v;
  }
  __syncthreads();
  dif_fft<T, T2>(buf, C, L, p.M, p.logM, twM, (T)-1);
  for (int idx = threadIdx.x; idx < C * p.M; idx += blockDim.x) {
    const int c = idx / p.M, m = idx - c * p.M;
    T2* col = buf + (size_t)c * L;
    const T2 x = col[m], g = filt[m];
    T2 v;
    v.x = x.x * g.x - x.y * g.y;
    v.y = x.x * g.y + x.y * g.x;
    col[m] = v;
  }
  __syncthreads();
  dit_fft<T, T2>(buf, C, L, p.M, p.logM, twM, (T)1);
  for (int idx = threadIdx.x; idx < C * p.N; idx += blockDim.x) {
    const int c = idx / p.N, k = idx - c * p.N;
    T2* col = buf + (size_t)c * L;
    const T2 x = col[k];
    const T2 w = chirp[k];
    const T wi = sgn < (T)0 ? -w.y : w.y;
    T2 v;
    v.x = x.x * w.x - x.y * wi;
    v.y = x.x * wi + x.y * w.x;
    col[k] = v;
  }
  __syncthreads();
}

// the N-point transform of the C columns; returns through `slot` where output k lives
template <typename T, typename T2, bool BLUE>
__device__ __forceinline__ void fft_any(T2* buf, int C, int L, const DstPlan<T>& p, T sgn) {
  if (BLUE)
    bluestein<T, T2>(buf, C, L, p, sgn);
  else
    dif_fft<T, T2>(buf, C, L, p.N, p.logN, (const T2*)p.tw, sgn);
}

template <bool BLUE>
__device__ __forceinline__ int out_slot(int k, int logN) {
  return BLUE ? k : bitrev(k, logN);
}

template <typename T, bool BLUE>
__global__ void k_dst_forward(T* x, long long S, ColGeom cg, DstPlan<T> plan, int C, const int* done) {
  using T2 = typename Vec2<T>::type;
  if (stop_requested(done)) return;
  const int N = plan.N, logN = plan.logN;
  const int L = BLUE ? plan.M + 1 : N + 1;  // column stride in shared memory
  const T2* __restrict__ pre = (const T2*)plan.pre;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* buf = (T2*)smem_raw;
  const long long c0 = (long long)blockIdx.x * 2 * C;
  // load: slot m = N-1-t holds (w_a, w_b); the m = 0 entry is doubled
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int c = idx % C;
    const int t = idx / C;
    T2 v = *(const T2*)(x + (long long)t * S + c0 + 2 * c);
    const int m = N - 1 - t;
    if (m == 0) {
      v.x *= (T)2;
      v.y *= (T)2;
    }
    buf[(size_t)c * L + m] = v;
  }
  __syncthreads();
  // pre-twiddle in pairs (m, N-m):  V[m] = e^{i pi m/(2N)} (w_m - i w_{N-m});  Z = V_a + i V_b
  const int halfp = (N >> 1) + 1;
  for (int idx = threadIdx.x; idx < C * halfp; idx += blockDim.x) {
    const int c = idx / halfp;
    const int m = idx - c * halfp;
    if (m == 0 || N == 1) continue;
    const int q = N - m;
    T2* col = buf + (size_t)c * L;
    const T2 A = col[m], Bq = col[q];
    const T2 em = pre[m], eq = pre[q];
    // column a: w_a = A.x (at m), Bq.x (at q); column b: A.y, Bq.y
    const T vam_r = A.x * em.x + Bq.x * em.y, vam_i = A.x * em.y - Bq.x * em.x;
    const T vbm_r = A.y * em.x + Bq.y * em.y, vbm_i = A.y * em.y - Bq.y * em.x;
    T2 zm;
    zm.x = vam_r - vbm_i;
    zm.y = vam_i + vbm_r;
    if (q != m) {
      const T vaq_r = Bq.x * eq.x + A.x * eq.y, vaq_i = Bq.x * eq.y - A.x * eq.x;
      const T vbq_r = Bq.y * eq.x + A.y * eq.y, vbq_i = Bq.y * eq.y - A.y * eq.x;
      T2 zq;
      zq.x = vaq_r - vbq_i;
      zq.y = vaq_i + vbq_r;
      col[q] = zq;
    }
    col[m] = zm;
  }
  __syncthreads();
  fft_any<T, T2, BLUE>(buf, C, L, plan, (T)1);
  // output: rhat_{j+1} = (-1)^j C3_j / 2, C3_{2i} = v_i, C3_{2i+1} = v_{N-1-i}
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int c = idx % C;
    const int j = idx / C;
    const int vi = (j & 1) ? (N - 1 - (j >> 1)) : (j >> 1);
    T2 v = buf[(size_t)c * L + out_slot<BLUE>(vi, logN)];
    const T sc = (j & 1) ? (T)-0.5 : (T)0.5;
    v.x = ghost_col(cg, c0 + 2 * c) ? (T)0 : v.x * sc;
    v.y = ghost_col(cg, c0 + 2 * c + 1) ? (T)0 : v.y * sc;
    *(T2*)(x + (long long)j * S + c0 + 2 * c) = v;
  }
}

template <typename T, bool BLUE>
__global__ void k_dst_inverse(const T* __restrict__ y, void* out, int mode, double omega, long long S,
                              ColGeom cg, DstPlan<T> plan, int C, const int* done) {
  using T2 = typename Vec2<T>::type;
  if (stop_requested(done)) return;
  const int N = plan.N, logN = plan.logN;
  const int L = BLUE ? plan.M + 1 : N + 1;
  const T2* __restrict__ pre = (const T2*)plan.pre;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* buf = (T2*)smem_raw;
  const long long c0 = (long long)blockIdx.x * 2 * C;
  // load: z_j = (-1)^j y_{j+1};  v_{j/2} = z_j (j even), v_{N-1-(j-1)/2} = z_j (j odd)
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int c = idx % C;
    const int j = idx / C;
    T2 v = *(const T2*)(y + (long long)j * S + c0 + 2 * c);
    int s;
    if (j & 1) {
      s = N - 1 - (j >> 1);
      v.x = -v.x;
      v.y = -v.y;
    } else {
      s = j >> 1;
    }
    buf[(size_t)c * L + s] = v;
  }
  __syncthreads();
  fft_any<T, T2, BLUE>(buf, C, L, plan, (T)-1);
  // post: V_a[m] = (C_m + conj C_{N-m})/2, V_b[m] = (C_m - conj C_{N-m})/(2i);
  //       X[m] = Re(e^{-i pi m/(2N)} V[m]);  u_{N-m} = X[m]  (time slot N-1-m)
  const int halfp = (N >> 1) + 1;
  for (int idx = threadIdx.x; idx < C * halfp; idx += blockDim.x) {
    const int c = idx % C;
    const int m = idx / C;
    if (N == 1 && m > 0) continue;
    const bool ga = ghost_col(cg, c0 + 2 * c), gb = ghost_col(cg, c0 + 2 * c + 1);
    const int q = m == 0 ? 0 : N - m;
    const T2* col = buf + (size_t)c * L;
    const T2 Cm = col[out_slot<BLUE>(m, logN)];
    const T2 Cq = col[out_slot<BLUE>(q, logN)];
    // V_a[m] = ((Cm.x + Cq.x)/2, (Cm.y - Cq.y)/2); V_b[m] = ((Cm.y + Cq.y)/2, (Cq.x - Cm.x)/2)
    const T2 em = pre[m];
    const T var = (T)0.5 * (Cm.x + Cq.x), vai = (T)0.5 * (Cm.y - Cq.y);
    const T vbr = (T)0.5 * (Cm.y + Cq.y), vbi = (T)0.5 * (Cq.x - Cm.x);
    const T Xa = ga ? (T)0 : var * em.x + vai * em.y;
    const T Xb = gb ? (T)0 : vbr * em.x + vbi * em.y;
    const long long o1 = (long long)(N - 1 - m) * S + c0 + 2 * c;
    if (mode == 1) {
      double2* u = (double2*)((double*)out + o1);
      double2 cur = *u;
      cur.x += omega * (double)Xa;
      cur.y += omega * (double)Xb;
      *u = cur;
    } else if (mode == 2) {
      T2* o = (T2*)((T*)out + o1);
      T2 cur = *o;
      cur.x += (T)omega * Xa;
      cur.y += (T)omega * Xb;
      *o = cur;
    } else {
      T2 v;
      v.x = Xa;
      v.y = Xb;
      *(T2*)((T*)out + o1) = v;
    }
    if (m != 0 && q != m) {
      // X[q] with the roles of m and q exchanged -> time slot N-1-q = m-1
      const T2 eq = pre[q];
      const T var2 = (T)0.5 * (Cq.x + Cm.x), vai2 = (T)0.5 * (Cq.y - Cm.y);
      const T vbr2 = (T)0.5 * (Cq.y + Cm.y), vbi2 = (T)0.5 * (Cm.x - Cq.x);
      const T Xa2 = ga ? (T)0 : var2 * eq.x + vai2 * eq.y;
      const T Xb2 = gb ? (T)0 : vbr2 * eq.x + vbi2 * eq.y;
      const long long o2 = (long long)(m - 1) * S + c0 + 2 * c;
      if (mode == 1) {
        double2* u = (double2*)((double*)out + o2);
        double2 cur = *u;
        cur.x += omega * (double)Xa2;
        cur.y += omega * (double)Xb2;
        *u = cur;
      } else if (mode == 2) {
        T2* o = (T2*)((T*)out + o2);
        T2 cur = *o;
        cur.x += (T)omega * Xa2;
        cur.y += (T)omega * Xb2;
        *o = cur;
      } else {
        T2 v;
        v.x = Xa2;
        v.y = Xb2;
        *(T2*)((T*)out + o2) = v;
      }
    }
  }
}

// ---- power-of-two N, 2 <= N <= 2048: the same transforms with radix-8 Stockham passes ----
// A CTA owns F complex columns (2F real columns) for all N slots; each column's FFT is done by
// nthr = max(1, N/8) threads, in place in a padded shared-memory array.  The e^{+} transform of
// the forward direction is taken as the conjugate of the e^{-} transform of the conjugate.

constexpr int kStockMaxN = 2048;
constexpr int kStockThreads = 256;  // (FP32: 4 CTAs per SM, FP64: 2 -- the register budget)

// MINB: CTAs per SM the register budget is sized for (FP32: 3 for N >= 1024, where the unspilled
// 80-register form measured faster, 4 below; FP64: 2)
template <typename T, int MINB>
__global__ void __launch_bounds__(kStockThreads, MINB) k_dst_forward_s(T* x, long long S, ColGeom cg, DstPlan<T> plan,
                                                                 int F, const int* done) {
  using T2 = typename Vec2<T>::type;
  if (stop_requested(done)) return;
  const int N = plan.N, logN = plan.logN;
  const int nthr = N >= 8 ? N >> 3 : 1;
  const int Lp = padded_len(N);
  const int logF = __ffs(F) - 1;  // F is a power of two: shifts instead of divisions
  const T2* __restrict__ pre = (const T2*)plan.pre;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* sm = (T2*)smem_raw;
  const long long c0 = (long long)blockIdx.x * 2 * F;
  // load: slot m = N-1-t holds (w_a, w_b); the m = 0 entry is doubled.  Four loads in flight
  // per thread (the loads are latency-bound at this occupancy).
  for (int idx0 = threadIdx.x; idx0 < N * F; idx0 += 4 * blockDim.x) {
    T2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = idx0 + q * blockDim.x;
      if (idx < N * F) v[q] = *(const T2*)(x + (long long)(idx >> logF) * S + c0 + 2 * (idx & (F - 1)));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = idx0 + q * blockDim.x;
      if (idx < N * F) {
        const int f = idx & (F - 1), m = N - 1 - (idx >> logF);
        if (m == 0) {
          v[q].x *= (T)2;
          v[q].y *= (T)2;
        }
        sm[(size_t)f * Lp + pd(m)] = v[q];
      }
    }
  }
  __syncthreads();
  // pre-twiddle in pairs (m, N-m): V[m] = e^{i pi m/(2N)} (w_m - i w_{N-m}), Z = V_a + i V_b,
  // stored conjugated
  const int halfp = (N >> 1) + 1;
  for (int idx = threadIdx.x; idx < F * halfp; idx += blockDim.x) {
    const int f = idx & (F - 1), m = idx >> logF;
    T2* col = sm + (size_t)f * Lp;
    if (m == 0) {
      col[0].y = -col[0].y;
      continue;
    }
    const int q = N - m;
    const T2 A = col[pd(m)], Bq = col[pd(q)];
    const T2 em = pre[m], eq = pre[q];
    const T vam_r = A.x * em.x + Bq.x * em.y, vam_i = A.x * em.y - Bq.x * em.x;
    const T vbm_r = A.y * em.x + Bq.y * em.y, vbm_i = A.y * em.y - Bq.y * em.x;
    if (q != m) {
      const T vaq_r = Bq.x * eq.x + A.x * eq.y, vaq_i = Bq.x * eq.y - A.x * eq.x;
      const T vbq_r = Bq.y * eq.x + A.y * eq.y, vbq_i = Bq.y * eq.y - A.y * eq.x;
      col[pd(q)] = mk<T2>(vaq_r - vbq_i, -(vaq_i + vbq_r));
    }
    col[pd(m)] = mk<T2>(vam_r - vbm_i, -(vam_i + vbm_r));
  }
  __syncthreads();
  {
    const int f = threadIdx.x / nthr, tid = threadIdx.x - f * nthr;
    block_fft<T2>(sm + (size_t)f * Lp, logN, (const T2*)plan.twS, tid, nthr);
  }
  // output: rhat_{j+1} = (-1)^j C3_j / 2, C3_{2i} = v_i, C3_{2i+1} = v_{N-1-i}; v = conj(spectrum)
  for (int idx = threadIdx.x; idx < N * F; idx += blockDim.x) {
    const int f = idx & (F - 1), j = idx >> logF;
    const int vi = (j & 1) ? (N - 1 - (j >> 1)) : (j >> 1);
    const T2 r = sm[(size_t)f * Lp + pd(vi)];
    const T sc = (j & 1) ? (T)-0.5 : (T)0.5;
    T2 v;
    v.x = ghost_col(cg, c0 + 2 * f) ? (T)0 : r.x * sc;
    v.y = ghost_col(cg, c0 + 2 * f + 1) ? (T)0 : -r.y * sc;
    *(T2*)(x + (long long)j * S + c0 + 2 * f) = v;
  }
}

// asynchronous global -> shared copies (sm_80+ cp.async): the target tile of the accumulating
// inverse is fetched while the transform runs
__device__ __forceinline__ void cp_async_8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T, int MINB>
__global__ void __launch_bounds__(kStockThreads, MINB) k_dst_inverse_s(const T* __restrict__ y, void* out, int mode,
                                                                 double omega, long long S, ColGeom cg,
                                                                 DstPlan<T> plan, int F, const int* done) {
  using T2 = typename Vec2<T>::type;
  if (stop_requested(done)) return;
  const int N = plan.N, logN = plan.logN;
  const int nthr = N >= 8 ? N >> 3 : 1;
  const int Lp = padded_len(N);
  const int logF = __ffs(F) - 1;  // F is a power of two: shifts instead of divisions
  const T2* __restrict__ pre = (const T2*)plan.pre;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* sm = (T2*)smem_raw;
  const long long c0 = (long long)blockIdx.x * 2 * F;
  // mode 2 (FP32 accumulate): prefetch the target tile [N][F] behind the transform tile
  T2* tgt = sm + (size_t)F * Lp;
  if (mode == 2 && sizeof(T2) == 8) {
    if (F >= 2) {  // two neighbouring column pairs per 16-byte copy (addresses 16-byte aligned: F even)
      for (int idx = 2 * threadIdx.x; idx < N * F; idx += 2 * blockDim.x) {
        const int f = idx & (F - 1), t = idx >> logF;
        cp_async_16(tgt + idx, (const T*)out + (long long)t * S + c0 + 2 * f);
      }
    } else {
      for (int idx = threadIdx.x; idx < N * F; idx += blockDim.x) {
        const int f = idx & (F - 1), t = idx >> logF;
        cp_async_8(tgt + idx, (const T*)out + (long long)t * S + c0 + 2 * f);
      }
    }
  }
  // load: z_j = (-1)^j y_{j+1};  v_{j/2} = z_j (j even), v_{N-1-(j-1)/2} = z_j (j odd)
  for (int idx0 = threadIdx.x; idx0 < N * F; idx0 += 4 * blockDim.x) {
    T2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = idx0 + q * blockDim.x;
      if (idx < N * F) v[q] = *(const T2*)(y + (long long)(idx >> logF) * S + c0 + 2 * (idx & (F - 1)));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = idx0 + q * blockDim.x;
      if (idx < N * F) {
        const int f = idx & (F - 1), j = idx >> logF;
        int s;
        if (j & 1) {
          s = N - 1 - (j >> 1);
          v[q].x = -v[q].x;
          v[q].y = -v[q].y;
        } else {
          s = j >> 1;
        }
        sm[(size_t)f * Lp + pd(s)] = v[q];
      }
    }
  }
  __syncthreads();
  {
    const int f = threadIdx.x / nthr, tid = threadIdx.x - f * nthr;
    block_fft<T2>(sm + (size_t)f * Lp, logN, (const T2*)plan.twS, tid, nthr);
  }
  const bool pref = mode == 2 && sizeof(T2) == 8;
  if (pref) {
    cp_async_commit_wait_all();
    __syncthreads();
  }
  // post: V_a[m] = (C_m + conj C_{N-m})/2, V_b[m] = (C_m - conj C_{N-m})/(2i);
  //       X[m] = Re(e^{-i pi m/(2N)} V[m]);  u_{N-m} = X[m]  (time slot N-1-m)
  const int halfp = (N >> 1) + 1;
  for (int idx = threadIdx.x; idx < F * halfp; idx += blockDim.x) {
    const int f = idx & (F - 1), m = idx >> logF;
    const bool ga = ghost_col(cg, c0 + 2 * f), gb = ghost_col(cg, c0 + 2 * f + 1);
    const int q = m == 0 ? 0 : N - m;
    const T2* col = sm + (size_t)f * Lp;
    const T2 Cm = col[pd(m)], Cq = col[pd(q)];
    const T2 em = pre[m];
    const T var = (T)0.5 * (Cm.x + Cq.x), vai = (T)0.5 * (Cm.y - Cq.y);
    const T vbr = (T)0.5 * (Cm.y + Cq.y), vbi = (T)0.5 * (Cq.x - Cm.x);
    const T Xa = ga ? (T)0 : var * em.x + vai * em.y;
    const T Xb = gb ? (T)0 : vbr * em.x + vbi * em.y;
    const long long o1 = (long long)(N - 1 - m) * S + c0 + 2 * f;
    if (mode == 1) {
      double2* u = (double2*)((double*)out + o1);
      double2 cur = *u;
      cur.x += omega * (double)Xa;
      cur.y += omega * (double)Xb;
      *u = cur;
    } else if (mode == 2) {
      T2* o = (T2*)((T*)out + o1);
      const T2 cur = pref ? tgt[(N - 1 - m) * F + f] : *o;
      *o = mk<T2>(cur.x + (T)omega * Xa, cur.y + (T)omega * Xb);
    } else {
      *(T2*)((T*)out + o1) = mk<T2>(Xa, Xb);
    }
    if (m != 0 && q != m) {
      // X[q] with the roles of m and q exchanged -> time slot N-1-q = m-1
      const T2 eq = pre[q];
      const T var2 = (T)0.5 * (Cq.x + Cm.x), vai2 = (T)0.5 * (Cq.y - Cm.y);
      const T vbr2 = (T)0.5 * (Cq.y + Cm.y), vbi2 = (T)0.5 * (Cm.x - Cq.x);
      const T Xa2 = ga ? (T)0 : var2 * eq.x + vai2 * eq.y;
      const T Xb2 = gb ? (T)0 : vbr2 * eq.x + vbi2 * eq.y;
      const long long o2 = (long long)(m - 1) * S + c0 + 2 * f;
      if (mode == 1) {
        double2* u = (double2*)((double*)out + o2);
        double2 cur = *u;
        cur.x += omega * (double)Xa2;
        cur.y += omega * (double)Xb2;
        *u = cur;
      } else if (mode == 2) {
        T2* o = (T2*)((T*)out + o2);
        const T2 cur = pref ? tgt[(m - 1) * F + f] : *o;
        *o = mk<T2>(cur.x + (T)omega * Xa2, cur.y + (T)omega * Xb2);
      } else {
        *(T2*)((T*)out + o2) = mk<T2>(Xa2, Xb2);
      }
    }
  }
}

template <typename T>
bool stockham_ok(const DstPlan<T>& plan) {
  return plan.M == 0 && plan.twS != nullptr && plan.N >= 2 && plan.N <= kStockMaxN;
}

// complex columns per CTA for the Stockham kernels: a power of two within the thread, shared-
// memory and slice limits (C from the plan or the autotuner is an upper bound)
template <typename T>
int stockham_cols(const DstPlan<T>& plan, long long S) {
  const int nthr = plan.N >= 8 ? plan.N >> 3 : 1;
  const long long per = (long long)padded_len(plan.N) * 2 * sizeof(T);
  long long F = plan.C > 0 ? plan.C : kStockThreads / nthr;
  F = std::min<long long>(F, std::max(1, kStockThreads / nthr));
  F = std::min<long long>(F, std::max<long long>(1, (200 * 1024) / per));
  long long pw = 1;
  while (pw * 2 <= F) pw *= 2;
  F = pw;
  while (F > 1 && (S % (2 * F)) != 0) F >>= 1;
  return (int)F;
}

template <typename T>
int dst_cols(int L, long long S) {
  // complex columns (stride L) per CTA: a power of two, <= 16, using at most ~100 KB of shared memory
  const long long bytes = (long long)L * 2 * sizeof(T);
  long long C = (100 * 1024) / bytes;
  if (C < 1) C = 1;
  if (C > 16) C = 16;
  long long pw = 1;
  while (pw * 2 <= C) pw *= 2;
  C = pw;
  while (C > 1 && (S % (2 * C)) != 0) C >>= 1;
  if (2 * C > S) C = S / 2 > 0 ? S / 2 : 1;
  return (int)C;
}

}  // namespace

template <typename T>
int plan_stride(const DstPlan<T>& plan) {
  return plan.M > 0 ? plan.M + 1 : plan.N + 1;
}

template <typename T>
void launch_dst_forward(T* x, long long S, int dim, int n, int logP, DstPlan<T> plan, const int* done,
                        cudaStream_t st) {
  using T2 = typename Vec2<T>::type;
  const int L = plan_stride(plan);
  const int C = plan.C > 0 ? plan.C : dst_cols<T>(L, S);
  const size_t smem = (size_t)C * L * sizeof(T2);
  const int blocks = (int)(S / (2 * C));
  const ColGeom cg{dim, n, logP};
  double interior = plan.N;
  for (int d = 0; d < dim; ++d) interior *= n;
  LaunchScope ls("dst_forward", st, 2.0 * sizeof(T) * interior);
  if (stockham_ok(plan)) {
    const int F = stockham_cols(plan, S);
    const int nthr = plan.N >= 8 ? plan.N >> 3 : 1;
    const size_t sm = (size_t)F * padded_len(plan.N) * sizeof(T2);
    auto go = [&](auto kern) {
      set_smem_limit((const void*)kern, 200 * 1024);
      kern<<<(unsigned)(S / (2 * F)), F * nthr, sm, st>>>(x, S, cg, plan, F, done);
    };
    if constexpr (sizeof(T) == 8) {
      go(k_dst_forward_s<T, 2>);
    } else {
      if (plan.N >= 1024)
        go(k_dst_forward_s<T, 3>);
      else
        go(k_dst_forward_s<T, 4>);
    }
  } else if (plan.M > 0) {
    set_smem_limit((const void*)k_dst_forward<T, true>, 200 * 1024);
    k_dst_forward<T, true><<<blocks, kThreads, smem, st>>>(x, S, cg, plan, C, done);
  } else {
    set_smem_limit((const void*)k_dst_forward<T, false>, 200 * 1024);
    k_dst_forward<T, false><<<blocks, kThreads, smem, st>>>(x, S, cg, plan, C, done);
  }
}

template <typename T>
void launch_dst_inverse(const T* y, void* out, int mode, double omega, long long S, int dim, int n,
                        int logP, DstPlan<T> plan, const int* done, cudaStream_t st) {
  using T2 = typename Vec2<T>::type;
  const int L = plan_stride(plan);
  const int C = plan.C > 0 ? plan.C : dst_cols<T>(L, S);
  const size_t smem = (size_t)C * L * sizeof(T2);
  const int blocks = (int)(S / (2 * C));
  const ColGeom cg{dim, n, logP};
  double interior = plan.N;
  for (int d = 0; d < dim; ++d) interior *= n;
  LaunchScope ls("dst_inverse", st,
                 (sizeof(T) + (mode == 1 ? 16.0 : mode == 2 ? 2.0 * sizeof(T) : (double)sizeof(T))) * interior);
  if (stockham_ok(plan)) {
    const int F = stockham_cols(plan, S);
    const int nthr = plan.N >= 8 ? plan.N >> 3 : 1;
    const size_t sm = (size_t)F * padded_len(plan.N) * sizeof(T2) +
                      (mode == 2 && sizeof(T2) == 8 ? (size_t)F * plan.N * sizeof(T2) : 0);
    auto go = [&](auto kern) {
      set_smem_limit((const void*)kern, 200 * 1024);
      kern<<<(unsigned)(S / (2 * F)), F * nthr, sm, st>>>(y, out, mode, omega, S, cg, plan, F, done);
    };
    if constexpr (sizeof(T) == 8) {
      go(k_dst_inverse_s<T, 2>);
    } else {
      if (plan.N >= 1024)
        go(k_dst_inverse_s<T, 3>);
      else
        go(k_dst_inverse_s<T, 4>);
    }
  } else if (plan.M > 0) {
    set_smem_limit((const void*)k_dst_inverse<T, true>, 200 * 1024);
    k_dst_inverse<T, true><<<blocks, kThreads, smem, st>>>(y, out, mode, omega, S, cg, plan, C, done);
  } else {
    set_smem_limit((const void*)k_dst_inverse<T, false>, 200 * 1024);
    k_dst_inverse<T, false><<<blocks, kThreads, smem, st>>>(y, out, mode, omega, S, cg, plan, C, done);
  }
}

// Forward transform of `ncols` packed columns held at pitch S (S a multiple of 32, columns
// ncols..S-1 are padding whose results are discarded).  It records no CUDA events (only the
// launch count), so it allocates nothing on any path.  N must be a power of two.
void launch_dst_forward_plain(double* x, long long S, int ncols, DstPlan<double> plan, cudaStream_t st) {
  const int L = plan.N + 1;
  const int C = dst_cols<double>(L, S);
  const size_t smem = (size_t)C * L * sizeof(double2);
  set_smem_limit((const void*)k_dst_forward<double, false>, 200 * 1024);
  int logP = 0;
  while ((1LL << logP) <= S) ++logP;  // pitch above every column index: only column ncols is "ghost"
  const ColGeom cg{1, ncols, logP};
  note_launch();
  k_dst_forward<double, false><<<(int)(S / (2 * C)), kThreads, smem, st>>>(x, S, cg, plan, C, nullptr);
}

template void launch_dst_forward<float>(float*, long long, int, int, int, DstPlan<float>, const int*, cudaStream_t);
template void launch_dst_forward<double>(double*, long long, int, int, int, DstPlan<double>, const int*, cudaStream_t);
template void launch_dst_inverse<float>(const float*, void*, int, double, long long, int, int, int, DstPlan<float>, const int*, cudaStream_t);
template void launch_dst_inverse<double>(const double*, void*, int, double, long long, int, int, int, DstPlan<double>, const int*, cudaStream_t);

}  // namespace pt
