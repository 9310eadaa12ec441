// Shared-memory FFT building blocks of the transform kernels (temporal DST, spatial DST-I).
#pragma once

#include "stencil_common.cuh"

namespace pt {
namespace {

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

__device__ __forceinline__ int bitrev(int v, int logN) {
  return logN == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - logN));
}

// radix-2 decimation-in-frequency stages over C columns of length `len` (column stride L):
// natural order in, bit-reversed order out.  tw[k] = e^{2 pi i k / len}; sgn = +1 or -1.
template <typename T, typename T2>
__device__ __forceinline__ void dif_fft(T2* buf, int C, int L, int len, int loglen,
                                        const T2* __restrict__ tw, T sgn) {
  const int half = len >> 1;
  for (int s = 0; s < loglen; ++s) {
    const int h = half >> s;  // span
    const int tstep = 1 << s; // twiddle index stride: len / (2h)
    for (int idx = threadIdx.x; idx < C * half; idx += blockDim.x) {
      const int c = idx / half;
      const int b = idx - c * half;
      const int j = b & (h - 1);
      const int i = ((b >> (loglen - 1 - s)) << (loglen - s)) + j;  // (b / h) * 2h + j
      T2* col = buf + (size_t)c * L;
      const T2 a = col[i];
      const T2 bb = col[i + h];
      const T2 w = tw[j * tstep];
      const T dr = a.x - bb.x, di = a.y - bb.y;
      const T wr = w.x, wi = sgn * w.y;
      col[i].x = a.x + bb.x;
      col[i].y = a.y + bb.y;
      col[i + h].x = dr * wr - di * wi;
      col[i + h].y = dr * wi + di * wr;
    }
    __syncthreads();
  }
}

// radix-2 decimation-in-time stages: bit-reversed order in, natural order out.
template <typename T, typename T2>
__device__ __forceinline__ void dit_fft(T2* buf, int C, int L, int len, int loglen,
                                        const T2* __restrict__ tw, T sgn) {
  const int half = len >> 1;
  for (int s = 0; s < loglen; ++s) {
    const int h = 1 << s;
    for (int idx = threadIdx.x; idx < C * half; idx += blockDim.x) {
      const int c = idx / half;
      const int b = idx - c * half;
      const int j = b & (h - 1);
      const int i = ((b >> s) << (s + 1)) + j;
      T2* col = buf + (size_t)c * L;
      const T2 w = tw[j << (loglen - 1 - s)];
      const T wr = w.x, wi = sgn * w.y;
      const T2 a = col[i];
      const T2 b0 = col[i + h];
      const T br = b0.x * wr - b0.y * wi, bi = b0.x * wi + b0.y * wr;
      col[i].x = a.x + br;
      col[i].y = a.y + bi;
      col[i + h].x = a.x - br;
      col[i + h].y = a.y - bi;
    }
    __syncthreads();
  }
}

// ---- radix-8 Stockham building blocks (natural order in and out) ----

// padded shared-memory index: one spare element per 8 keeps radix-8 strided writes conflict-free
__device__ __forceinline__ int pd(int e) { return e + (e >> 3); }
__host__ __device__ constexpr int padded_len(int M) { return M + (M >> 3) + 1; }

template <typename T2>
__device__ __forceinline__ T2 mk(decltype(T2::x) x, decltype(T2::x) y) {
  T2 r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 w) {
  return mk<T2>(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
template <typename T2>
__device__ __forceinline__ T2 mul_mi(T2 a) { return mk<T2>(a.y, -a.x); }  // a * (-i)

// forward DFTs of length 2, 4, 8 in registers, natural order in and out (omega_R = e^{-2 pi i/R})
template <typename T2>
__device__ __forceinline__ void dft2(T2* u) {
  const T2 a = u[0];
  u[0] = cadd(a, u[1]);
  u[1] = csub(a, u[1]);
}
template <typename T2>
__device__ __forceinline__ void dft4(T2& u0, T2& u1, T2& u2, T2& u3) {
  const T2 s02 = cadd(u0, u2), d02 = csub(u0, u2), s13 = cadd(u1, u3), d13 = mul_mi(csub(u1, u3));
  u0 = cadd(s02, s13);
  u2 = csub(s02, s13);
  u1 = cadd(d02, d13);
  u3 = csub(d02, d13);
}
template <typename T2>
__device__ __forceinline__ void dft8(T2* u) {
  using T = decltype(T2::x);
  const T r = (T)0.70710678118654752440;  // 1/sqrt(2)
  T2 e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  T2 o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  o1 = mk<T2>((o1.x + o1.y) * r, (o1.y - o1.x) * r);   // * e^{-i pi/4}
  o2 = mul_mi(o2);                                       // * e^{-i pi/2}
  o3 = mk<T2>((o3.y - o3.x) * r, -(o3.x + o3.y) * r);  // * e^{-3 i pi/4}
  u[0] = cadd(e0, o0);
  u[4] = csub(e0, o0);
  u[1] = cadd(e1, o1);
  u[5] = csub(e1, o1);
  u[2] = cadd(e2, o2);
  u[6] = csub(e2, o2);
  u[3] = cadd(e3, o3);
  u[7] = csub(e3, o3);
}
template <int LR, typename T2>
__device__ __forceinline__ void dftR(T2* u) {
  if (LR == 1) dft2(u);
  if (LR == 2) dft4(u[0], u[1], u[2], u[3]);
  if (LR == 3) dft8(u);
}

// One Stockham (autosort) radix-2^LR pass of a length-M = 2^logM FFT, after passes of total
// radix p = 2^s: butterfly i reads in[i + m M/R], twiddles input m by omega_{pR}^{m k}
// (k = i mod p), and writes out[(i - k) R + k + m p].  tw[e] = e^{-2 pi i e / M}.
template <int LR, typename T2>
__device__ __forceinline__ void stockham_pass(const T2* __restrict__ in, T2* __restrict__ out, int logM, int s,
                                              const T2* __restrict__ tw, int lane) {
  constexpr int R = 1 << LR;
  const int nb = 1 << (logM - LR);
  const int p = 1 << s;
  const int tsh = logM - s - LR;
  for (int i = lane; i < nb; i += 32) {
    const int k = i & (p - 1);
    T2 u[R];
#pragma unroll
    for (int m = 0; m < R; ++m) u[m] = in[pd(i + m * nb)];
    if (s > 0) {
#pragma unroll
      for (int m = 1; m < R; ++m) u[m] = cmul(u[m], __ldg(&tw[(m * k) << tsh]));
    }
    dftR<LR>(u);
    const int j = ((i - k) << LR) + k;
#pragma unroll
    for (int m = 0; m < R; ++m) out[pd(j + m * p)] = u[m];
  }
}

// FFT of the warp's sequence in `a` (padded, natural order); `b` is scratch.  Returns the buffer
// holding the spectrum (natural order).
template <typename T2>
__device__ __forceinline__ T2* warp_fft(T2* a, T2* b, int logM, const T2* __restrict__ tw, int lane) {
  int s = 0;
  while (s < logM) {
    const int rem = logM - s;
    if (rem >= 5 || rem == 3) {
      stockham_pass<3>(a, b, logM, s, tw, lane);
      s += 3;
    } else if (rem == 4 || rem == 2) {
      stockham_pass<2>(a, b, logM, s, tw, lane);
      s += 2;
    } else {
      stockham_pass<1>(a, b, logM, s, tw, lane);
      s += 1;
    }
    __syncwarp();
    T2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Compile-time length (LOGM > 0): the same passes with every trip count, stride and shift a
// constant, fully unrolled.
template <int LR, int LOGM, int S, typename T2>
__device__ __forceinline__ void stockham_pass_c(const T2* __restrict__ in, T2* __restrict__ out,
                                                const T2* __restrict__ tw, int lane) {
  constexpr int R = 1 << LR;
  constexpr int NB = 1 << (LOGM - LR);
  constexpr int P = 1 << S;
  constexpr int TSH = LOGM - S - LR;
#pragma unroll
  for (int i0 = 0; i0 < NB; i0 += 32) {
    const int i = i0 + lane;
    if (NB >= 32 || i < NB) {
      const int k = i & (P - 1);
      T2 u[R];
#pragma unroll
      for (int m = 0; m < R; ++m) u[m] = in[pd(i + m * NB)];
      if (S > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) u[m] = cmul(u[m], __ldg(&tw[(m * k) << TSH]));
      }
      dftR<LR>(u);
      const int j = ((i - k) << LR) + k;
#pragma unroll
      for (int m = 0; m < R; ++m) out[pd(j + m * P)] = u[m];
    }
  }
}

template <int LOGM, int S, typename T2>
__device__ __forceinline__ T2* warp_fft_c(T2* a, T2* b, const T2* __restrict__ tw, int lane) {
  if constexpr (S >= LOGM) {
    return a;
  } else {
    constexpr int REM = LOGM - S;
    constexpr int LR = (REM >= 5 || REM == 3) ? 3 : (REM == 4 || REM == 2) ? 2 : 1;
    stockham_pass_c<LR, LOGM, S>(a, b, tw, lane);
    __syncwarp();
    return warp_fft_c<LOGM, S + LR>(b, a, tw, lane);
  }
}

// Block-cooperative Stockham pass: the FFTs of a CTA each own `nthr` threads (tid = thread index
// within its FFT) and every thread holds 8 values (N >= 8); read all, barrier, write all, barrier,
// so the pass is done in place.  Every thread of the CTA must call it.
template <int LR, typename T2>
__device__ __forceinline__ void block_pass(T2* buf, int logN, int s, const T2* __restrict__ tw, int tid,
                                           int nthr) {
  constexpr int R = 1 << LR;
  constexpr int Q = 8 / R;
  const int nb = 1 << (logN - LR);
  const int p = 1 << s;
  const int tsh = logN - s - LR;
  T2 u[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = tid + q * nthr;
    if (i < nb) {
#pragma unroll
      for (int m = 0; m < R; ++m) u[q][m] = buf[pd(i + m * nb)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = tid + q * nthr;
    if (i < nb) {
      const int k = i & (p - 1);
      if (s > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) u[q][m] = cmul(u[q][m], __ldg(&tw[(m * k) << tsh]));
      }
      dftR<LR>(u[q]);
      const int j = ((i - k) << LR) + k;
#pragma unroll
      for (int m = 0; m < R; ++m) buf[pd(j + m * p)] = u[q][m];
    }
  }
  __syncthreads();
}

// forward FFT (e^{-}) of every CTA-owned sequence in place, natural order in and out
template <typename T2>
__device__ __forceinline__ void block_fft(T2* buf, int logN, const T2* __restrict__ tw, int tid, int nthr) {
  int s = 0;
  while (s < logN) {
    const int rem = logN - s;
    if (rem >= 5 || rem == 3) {
      block_pass<3>(buf, logN, s, tw, tid, nthr);
      s += 3;
    } else if (rem == 4 || rem == 2) {
      block_pass<2>(buf, logN, s, tw, tid, nthr);
      s += 2;
    } else {
      block_pass<1>(buf, logN, s, tw, tid, nthr);
      s += 1;
    }
  }
}

}  // namespace
}  // namespace pt
