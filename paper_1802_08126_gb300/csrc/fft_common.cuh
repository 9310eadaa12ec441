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

}  // namespace
}  // namespace pt
