// Device helpers shared by the stencil, multigrid and transform kernels.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "pt_internal.cuh"

namespace pt {

constexpr int kThreads = 256;

inline int grid_for(long long work, int threads = kThreads, int max_blocks = 152 * 32) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

__device__ __forceinline__ bool stop_requested(const int* done) {
  return done != nullptr && *((volatile const int*)done) != 0;
}

// Decode a padded index into slot t and coordinates; returns true for interior points.
template <int DIM>
__device__ __forceinline__ bool decode(long long i, int logP, int n, long long& t, int& x, int& y,
                                       int& z) {
  const int P = 1 << logP;
  t = i >> (DIM * logP);
  long long rem = i & ((1LL << (DIM * logP)) - 1);
  x = (int)(rem & (P - 1));
  y = DIM >= 2 ? (int)((rem >> logP) & (P - 1)) : 0;
  z = DIM >= 3 ? (int)(rem >> (2 * logP)) : 0;
  return x < n && y < n && z < n;
}

// Face coefficients around interior point (x, y, z): am[d] on the lower, ap[d] on the upper
// face along axis d.  Tables: node_d[i] = g_d(pi m_d (i+1) h), face_d[j] = g_d(pi m_d (j+1/2) h).
template <int DIM, typename T>
__device__ __forceinline__ void face_coefs(const T* __restrict__ tab, int P, int x, int y, int z,
                                           T cth, T a0, T* am, T* ap) {
  const T* nx = tab;
  const T* fx = tab + P;
  if (DIM == 1) {
    am[0] = fma(cth, fx[x], a0);
    ap[0] = fma(cth, fx[x + 1], a0);
  } else if (DIM == 2) {
    const T* ny = tab + 2 * P;
    const T* fy = tab + 3 * P;
    const T gy = cth * ny[y];
    am[0] = fma(gy, fx[x], a0);
    ap[0] = fma(gy, fx[x + 1], a0);
    const T gx = cth * nx[x];
    am[1] = fma(gx, fy[y], a0);
    ap[1] = fma(gx, fy[y + 1], a0);
  } else {
    const T* ny = tab + 2 * P;
    const T* fy = tab + 3 * P;
    const T* nz = tab + 4 * P;
    const T* fz = tab + 5 * P;
    const T cx = cth * nx[x], cy = ny[y], cz = nz[z];
    const T gyz = cth * cy * cz;
    am[0] = fma(gyz, fx[x], a0);
    ap[0] = fma(gyz, fx[x + 1], a0);
    const T gxz = cx * cz;
    am[1] = fma(gxz, fy[y], a0);
    ap[1] = fma(gxz, fy[y + 1], a0);
    const T gxy = cx * cy;
    am[2] = fma(gxy, fz[z], a0);
    ap[2] = fma(gxy, fz[z + 1], a0);
  }
}

// sum_d [am_d (v_c - v_{i - s_d}) + ap_d (v_c - v_{i + s_d})]  (without the 1/h^2 factor)
template <int DIM, typename T, typename V>
__device__ __forceinline__ T stencil_sum(const V* __restrict__ v, long long i, T vc, const T* am,
                                         const T* ap, int P) {
  T s = am[0] * (vc - (T)v[i - 1]) + ap[0] * (vc - (T)v[i + 1]);
  if (DIM >= 2) s += am[1] * (vc - (T)v[i - P]) + ap[1] * (vc - (T)v[i + P]);
  if (DIM >= 3) {
    const long long P2 = (long long)P * P;
    s += am[2] * (vc - (T)v[i - P2]) + ap[2] * (vc - (T)v[i + P2]);
  }
  return s;
}

// (M v)_i for the P1 finite-element mass matrix over h^d (the M of eq. 2.1 when it is not the
// identity): 1-D [1/6, 2/3, 1/6]; 2-D, every grid square cut along its lower-left to upper-right
// diagonal: 1/2 at the point and 1/12 at the four axis neighbours and at the upper-right and
// lower-left diagonal ones.  Out-of-grid neighbours are the padded layout's zero ghosts (the
// lower-left one of the first point of a slice is a guard or the previous slice's ghost column).
template <int DIM, typename T, typename V>
__device__ __forceinline__ T mass_p1(const V* __restrict__ v, long long i, T vc, int P) {
  if (DIM == 1) return (T)(2.0 / 3.0) * vc + (T)(1.0 / 6.0) * ((T)v[i - 1] + (T)v[i + 1]);
  if (DIM == 2) {
    const T s = ((T)v[i - 1] + (T)v[i + 1]) + ((T)v[i - P] + (T)v[i + P]) +
                ((T)v[i - P - 1] + (T)v[i + P + 1]);
    return (T)0.5 * vc + (T)(1.0 / 12.0) * s;
  }
  return vc;  // (no P1 form in 3-D)
}

// diagonal entry of that mass matrix
template <int DIM, typename T>
__device__ __forceinline__ T mass_diag(int mass) {
  return mass == 0 ? (T)1 : (DIM == 1 ? (T)(2.0 / 3.0) : (DIM == 2 ? (T)0.5 : (T)1));
}

// (M v)_i with M the identity (mass == 0) or the P1 mass
template <int DIM, typename T, typename V>
__device__ __forceinline__ T mass_apply(int mass, const V* __restrict__ v, long long i, T vc, int P) {
  return mass == 0 ? vc : mass_p1<DIM, T, V>(v, i, vc, P);
}

template <int DIM, typename T>
__device__ __forceinline__ T face_sum(const T* am, const T* ap) {
  T s = am[0] + ap[0];
  if (DIM >= 2) s += am[1] + ap[1];
  if (DIM >= 3) s += am[2] + ap[2];
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; result valid in thread 0.  blockDim.x must be a multiple of 32, <= 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

template <typename T>
__device__ __forceinline__ void store_out(void* out, long long i, int mode, int out_fp64, T v) {
  if (out_fp64) {
    double* o = (double*)out;
    if (mode == 1)
      o[i] += (double)v;
    else
      o[i] = (double)v;
  } else {
    T* o = (T*)out;
    if (mode == 1)
      o[i] += v;
    else
      o[i] = v;
  }
}

}  // namespace pt
