// Exact spatial solves for the Schur preconditioner when the reference operator has a constant
// coefficient (Abar = a0 L_h, L_h the finite-difference Laplacian).  The sine transform of type I
// along each axis, (S v)_k = sum_{j=1}^{n} v_j sin(pi j k / M), M = n + 1, diagonalises L_h with
// eigenvalues (4/h^2) sum_d sin^2(pi k_d h / 2) and satisfies S S = (M/2) I.  Hence the block
// solve of §4, eq. 4.4,
//     Hhat_k^-1 = (2 tau / N) H_k^-1 Abar H_k^-1,  H_k = mu_k I + tau Abar,
// is, in the doubly transformed basis, the point-wise factor
//     (2 tau / N) (2/M)^d a0 l / (mu_k + tau a0 l)^2,   l = the eigenvalue of L_h,
// between two spatial transforms (this is the exact H of eq. 4.4, gamma = Gamma = 1 in eq. 4.7).
//
// One DST-I of length n costs one real DFT of length M instead of the 2M of the odd extension:
// with x_0 = x_M = 0 and s_j = sin(pi j / M), the sequence
//     y_j = s_j (x_j + x_{M-j}) + (x_j - x_{M-j}) / 2,   j = 0 .. M-1,
// has the real DFT Y_k = R_k + i I_k (e^{-2 pi i j k / M} convention) with
//     S_{2k} = -I_k,   S_{2k+1} = S_{2k-1} + R_k,   S_1 = R_0 / 2
// (the symmetric part of y pairs with the cosines, the antisymmetric part with the sines; the
// odd outputs are a prefix sum over k).  Two real lines share one complex FFT of length M, and
// each pair of lines is handled by one warp: radix-8 / 4 / 2 Stockham passes through a padded
// shared-memory ping-pong pair, the prefix sum as a chunked warp scan.
#include "fft_common.cuh"

namespace pt {
namespace {

constexpr int kWarpsMax = 8;

// z_j = (y^a_j + i y^b_j) / 2 from x_j = read(j - 1) (position j-1 holds x_j, x_0 = x_M = 0);
// sn[j] = sin(pi j / M) / 2 for j <= M/2.
template <int LOGMC, typename T, typename T2, typename Read>
__device__ __forceinline__ void dsti_pre(T2* z, int M_rt, const T* __restrict__ sn, int lane, Read read) {
  const int M = LOGMC > 0 ? (1 << LOGMC) : M_rt;
  const int H = M >> 1;
#pragma unroll
  for (int j = lane; j <= H; j += 32) {
    if (j == 0) {
      z[0] = mk<T2>((T)0, (T)0);
      continue;
    }
    const T2 xj = read(j - 1), xm = read(M - j - 1);
    const T s = sn[j];
    const T Aa = xj.x + xm.x, Ab = xj.y + xm.y;
    const T Da = (T)0.25 * (xj.x - xm.x), Db = (T)0.25 * (xj.y - xm.y);
    z[pd(j)] = mk<T2>(fma(s, Aa, Da), fma(s, Ab, Db));
    if (j != H) z[pd(M - j)] = mk<T2>(fma(s, Aa, -Da), fma(s, Ab, -Db));
  }
}

// From the spectrum Z of the packed pair: write(pos, (S^a, S^b)) for every position 0 .. M-1
// (S_q at position q-1, the ghost position M-1 gets 0).
template <int LOGMC, typename T, typename T2, typename Write>
__device__ __forceinline__ void dsti_post(const T2* Z, int M_rt, int lane, Write write) {
  const int M = LOGMC > 0 ? (1 << LOGMC) : M_rt;
  const int H = M >> 1;
  const int K = H >= 32 ? H >> 5 : 1;  // k's per lane, contiguous
  const int k0 = lane * K;
  const bool act = k0 < H;
  // contributions to the odd outputs: c_0 = R_0 / 2, c_k = R_k (the 1/2 of the pair split is in z)
  auto contrib = [&](int k) -> T2 {
    const T2 zk = Z[pd(k)];
    if (k == 0) return zk;
    const T2 zm = Z[pd(M - k)];
    return mk<T2>(zk.x + zm.x, zk.y + zm.y);
  };
  T ta = (T)0, tb = (T)0;
  if (act) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const T2 c = contrib(k0 + q);
      ta += c.x;
      tb += c.y;
    }
  }
  // warp inclusive scan of the chunk totals
  T ia = ta, ib = tb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T va = __shfl_up_sync(0xffffffffu, ia, o);
    const T vb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += va;
      ib += vb;
    }
  }
  if (!act) return;
  T pa = ia - ta, pb = ib - tb;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int k = k0 + q;
    const T2 c = contrib(k);
    pa += c.x;
    pb += c.y;
    write(2 * k, mk<T2>(pa, pb));  // S_{2k+1}
    if (k == 0) {
      write(M - 1, mk<T2>((T)0, (T)0));
    } else {
      const T2 zk = Z[pd(k)], zm = Z[pd(M - k)];
      write(2 * k - 1, mk<T2>(zm.y - zk.y, zk.x - zm.x));  // S_{2k} = -I_k
    }
  }
}

template <int LOGMC, typename T2>
__device__ __forceinline__ T2* fft_any(T2* a, T2* b, int logM, const T2* __restrict__ tw, int lane) {
  if constexpr (LOGMC > 0)
    return warp_fft_c<LOGMC, 0>(a, b, tw, lane);
  else
    return warp_fft<T2>(a, b, logM, tw, lane);
}

template <typename T>
struct DstiTabs {
  const typename Vec2<T>::type* tw;  // [M]   e^{-2 pi i e / M}
  const T* sn;                       // [M/2 + 1] sin(pi j / M) / 2
  const T* g;                        // padded like the data: the block-solve factor, 0 at ghosts
  // or, with g == nullptr, the same factor formed per point as c l / (m_k + l)^2 from l = the sum
  // of the axes' eigenvalues lam[.] (a0 L_h in the sine basis), m_k = mu_k / tau and c = c0 / tau^2
  const T* lam;                      // [M], lam[M - 1] = 0
  const T* m;                        // [N]
  T c;
};

// Rows (x, contiguous): every line pair of every slice, in place.  Lines 2q and 2q+1.
template <typename T, int LOGMC>
__global__ void __launch_bounds__(kWarpsMax * 32) k_dsti_rows(T* __restrict__ x, int logM_rt, int dim,
                                                              long long npairs, DstiTabs<T> tb) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int logM = LOGMC > 0 ? LOGMC : logM_rt;
  const int M = 1 << logM;
  const int W = padded_len(M);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  T2* A = (T2*)smem_raw + (size_t)warp * (2 * W + 1);
  T2* B = A + W;
  for (long long pr = (long long)blockIdx.x * wpb + warp; pr < npairs; pr += (long long)gridDim.x * wpb) {
    const long long la = 2 * pr;
    T* xa = x + la * M;
    T* xb = xa + M;
    dsti_pre<LOGMC, T, T2>(A, M, tb.sn, lane, [&](int pos) { return mk<T2>(xa[pos], xb[pos]); });
    __syncwarp();
    T2* Z = fft_any<LOGMC>(A, B, logM, tb.tw, lane);
    T2* O = Z == A ? B : A;
    dsti_post<LOGMC, T, T2>(Z, M, lane, [&](int pos, T2 v) { O[pd(pos)] = v; });
    __syncwarp();
    // ghost lines: y == n (2-D and 3-D) or z == n (3-D)
    auto ghost = [&](long long l) {
      const long long y = l & (M - 1);
      return y == M - 1 || (dim == 3 && ((l >> logM) & (M - 1)) == M - 1);
    };
    const bool ga = ghost(la), gb = ghost(la + 1);
#pragma unroll
    for (int pos = lane; pos < M; pos += 32) {
      const T2 v = O[pd(pos)];
      xa[pos] = ga ? (T)0 : v.x;
      xb[pos] = gb ? (T)0 : v.y;
    }
    __syncwarp();
  }
}

// Columns along a strided axis (1: y, stride M; 2: z, stride M^2), in place.  A block takes 2C
// consecutive columns (x .. x + 2C - 1) of one plane of one slice; warp w transforms columns
// 2w, 2w+1.  With `scale`, the column pair gets S diag(g) S, g the exact block-solve factor.
// Per-warp buffer stride (complex elements) of the column kernel: two transforms of length W and
// a pad.  FP32: the pad makes the stride 4 banks mod 32, so that the tile copies (a warp moves
// two positions of 16 consecutive columns) hit 32 distinct banks; FP64: one element.
template <typename T>
__host__ __device__ __forceinline__ int cols_stride(int W) {
  if (sizeof(T) == 8) return 2 * W + 1;
  const int q = ((2 - 2 * W) % 16 + 16) % 16;
  return 2 * W + (q == 0 ? 16 : q);
}

template <typename T, int LOGMC>
__global__ void __launch_bounds__(kWarpsMax * 32, (sizeof(T) == 4 && LOGMC > 0 && LOGMC <= 8) ? 5 : 1) k_dsti_cols(T* __restrict__ x, int logM_rt, int dim, int axis,
                                                              long long S, int scale, DstiTabs<T> tb) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int logM = LOGMC > 0 ? LOGMC : logM_rt;
  const int M = 1 << logM;
  const int W = padded_len(M);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int C = blockDim.x >> 5;
  const int tiles_x = M / (2 * C);
  const int tx = blockIdx.x % tiles_x;
  const int o = blockIdx.x / tiles_x;  // other in-plane coordinate (3-D), 0 in 2-D
  const int slice = blockIdx.y;
  const long long stride = axis == 1 ? (long long)M : (long long)M * M;
  const int x0 = tx * 2 * C;
  // column base: y axis -> o = z, z axis -> o = y
  const long long base = (long long)slice * S + (axis == 1 ? (long long)o * M * M : (long long)o * M) + x0;
  T2* bufs = (T2*)smem_raw;
  const int BS = cols_stride<T>(W);
  auto bufA = [&](int w) { return bufs + (size_t)w * BS; };
  // load the tile (columns fastest, coalesced); position M-1 is never read by the transform
  for (int idx = threadIdx.x; idx < 2 * C * (M - 1); idx += blockDim.x) {
    const int pos = idx / (2 * C), c = idx - pos * 2 * C;
    ((T*)(bufA(c >> 1) + pd(pos)))[c & 1] = x[base + pos * stride + c];
  }
  __syncthreads();
  T2* A = bufA(warp);
  T2* B = A + W;
  const int xa = x0 + 2 * warp;
  const bool ghost_o = dim == 3 && o == M - 1;
  dsti_pre<LOGMC, T, T2>(B, M, tb.sn, lane, [&](int pos) { return A[pd(pos)]; });
  __syncwarp();
  T2* Z = fft_any<LOGMC>(B, A, logM, tb.tw, lane);
  T2* O = Z == A ? B : A;
  if (scale) {
    if (tb.g) {
      // g from the precomputed table (same padded layout as the data, zero on ghosts)
      const T* gcol = tb.g + base + 2 * warp;
      dsti_post<LOGMC, T, T2>(Z, M, lane, [&](int pos, T2 v) {
        const T2 g = *(const T2*)(gcol + pos * stride);
        O[pd(pos)] = mk<T2>(v.x * g.x, v.y * g.y);
      });
    } else {
      // g formed here (FP32): the ghost column, plane and position are zeroed at the store
      const T lo = dim == 3 ? tb.lam[o] : (T)0;
      const T m = tb.m[slice], c = tb.c;
      const T la = tb.lam[xa] + lo, lb = tb.lam[xa + 1] + lo;
      dsti_post<LOGMC, T, T2>(Z, M, lane, [&](int pos, T2 v) {
        const T lp = tb.lam[pos];
        const T l_a = la + lp, l_b = lb + lp;
        const T d_a = m + l_a, d_b = m + l_b;
        O[pd(pos)] = mk<T2>(v.x * __fdividef(c * l_a, d_a * d_a), v.y * __fdividef(c * l_b, d_b * d_b));
      });
    }
    __syncwarp();
    T2* P2 = O == A ? B : A;  // second transform of the scaled spectrum
    dsti_pre<LOGMC, T, T2>(P2, M, tb.sn, lane, [&](int pos) { return O[pd(pos)]; });
    __syncwarp();
    T2* Z2 = fft_any<LOGMC>(P2, O, logM, tb.tw, lane);
    T2* O2 = Z2 == A ? B : A;
    dsti_post<LOGMC, T, T2>(Z2, M, lane, [&](int pos, T2 v) { O2[pd(pos)] = v; });
    O = O2;
  } else {
    dsti_post<LOGMC, T, T2>(Z, M, lane, [&](int pos, T2 v) { O[pd(pos)] = v; });
  }
  // every warp's result sits in the same one of its two buffers
  const int off = (int)(O - A);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * C * M; idx += blockDim.x) {
    const int pos = idx / (2 * C), c = idx - pos * 2 * C;
    const int xc = x0 + c;
    const bool gh = xc == M - 1 || ghost_o || pos == M - 1;
    const T v = ((const T*)(bufA(c >> 1) + off + pd(pos)))[c & 1];
    x[base + pos * stride + c] = gh ? (T)0 : v;
  }
}

// Whole planes in shared memory (M <= 128): the plane of one slot (2-D) or of one (slot, z) (3-D)
// is loaded once, transformed along x (rows) and y (columns) by the per-warp transforms above,
// and stored once.  MODE 0 (2-D): the whole exact block solve S_x S_y diag(g) S_y S_x; MODE 1
// (3-D): S_y S_x before the z-axis pass; MODE 2 (3-D): S_x S_y after it; MODE 3 (3-D): the z-axis
// pass S_z diag(g) S_z on the x-z plane of one (slot, y) (rows z at stride M^2, columns x).  The
// row pitch M + 2 keeps the column-pair reads of a warp (32 rows, one pair each) free of bank
// conflicts.
template <int M>
__host__ __device__ constexpr int plane_pitch() {
  return M + 2;
}

// warps per CTA of the plane kernel: 16 for the largest planes (two CTAs per SM fit in shared
// memory either way, so the wider CTA doubles the warps per SM), 8 otherwise
template <int LOGM>
__host__ __device__ constexpr int plane_warps() {
  return LOGM >= 7 ? 16 : kWarpsMax;
}

template <typename T, int LOGM, int MODE>
__global__ void __launch_bounds__(plane_warps<LOGM>() * 32, (LOGM >= 7 && sizeof(T) == 4) ? 2 : 1) k_dsti_plane(T* __restrict__ x, long long S, int planes,
                                                                         DstiTabs<T> tb) {
  using T2 = typename Vec2<T>::type;
  constexpr int M = 1 << LOGM, W = padded_len(M), PITCH = plane_pitch<M>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pl = (T*)smem_raw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T2* A = (T2*)(pl + M * PITCH) + (size_t)warp * (2 * W + 1);
  T2* B = A + W;
  constexpr bool SCALE = MODE == 0 || MODE == 3;
  constexpr long long RS = MODE == 3 ? (long long)M * M : M;  // global stride of the plane's rows
  // z: the plane's coordinate on the third axis (z for modes 1 and 2, y for mode 3)
  const int slice = (int)(blockIdx.x / planes), z = (int)(blockIdx.x - (long long)slice * planes);
  const long long base = (long long)slice * S + (long long)z * (MODE == 3 ? M : M * M);
  T* xp = x + base;
  if (MODE != 0 && z == M - 1) {  // the ghost plane stays zero
    for (int i = threadIdx.x; i < M * M; i += blockDim.x) xp[(i >> LOGM) * RS + (i & (M - 1))] = (T)0;
    return;
  }
  for (int i = threadIdx.x; i < M * M; i += blockDim.x)
    pl[(i >> LOGM) * PITCH + (i & (M - 1))] = xp[(i >> LOGM) * RS + (i & (M - 1))];
  __syncthreads();
  // x: line pairs (2q, 2q + 1), in place (the row's values are in the warp's buffer before the
  // spectrum is written back)
  auto rows = [&]() {
    for (int q = warp; q < M / 2; q += nw) {
      T* ra = pl + 2 * q * PITCH;
      T* rb = ra + PITCH;
      dsti_pre<LOGM, T, T2>(A, M, tb.sn, lane, [&](int pos) { return mk<T2>(ra[pos], rb[pos]); });
      __syncwarp();
      T2* Z = fft_any<LOGM>(A, B, LOGM, tb.tw, lane);
      T2* O = Z == A ? B : A;
      // (through the padded buffer: the lanes' output chunks written straight into the row would
      // collide in the shared-memory banks)
      dsti_post<LOGM, T, T2>(Z, M, lane, [&](int pos, T2 v) { O[pd(pos)] = v; });
      __syncwarp();
#pragma unroll
      for (int pos = lane; pos < M; pos += 32) {
        const T2 v = O[pd(pos)];
        ra[pos] = v.x;
        rb[pos] = v.y;
      }
      __syncwarp();
    }
  };
  // y: column pairs (2q, 2q + 1); MODE 0 also scales by the block-solve factor and transforms back
  auto cols = [&]() {
    for (int q = warp; q < M / 2; q += nw) {
      const int xa = 2 * q;
      T2* col = (T2*)(pl + xa);
      auto at = [&](int pos) -> T2& { return *(T2*)((T*)col + pos * PITCH); };
      dsti_pre<LOGM, T, T2>(A, M, tb.sn, lane, [&](int pos) { return at(pos); });
      __syncwarp();
      T2* Z = fft_any<LOGM>(A, B, LOGM, tb.tw, lane);
      if (SCALE) {
        T2* O = Z == A ? B : A;  // the scaled spectrum
        if (tb.g) {
          const T* gcol = tb.g + base + xa;
          dsti_post<LOGM, T, T2>(Z, M, lane, [&](int pos, T2 v) {
            const T2 g = *(const T2*)(gcol + pos * RS);
            O[pd(pos)] = mk<T2>(v.x * g.x, v.y * g.y);
          });
        } else {
          const T m = tb.m[slice], c = tb.c;
          const T lo = MODE == 3 ? tb.lam[z] : (T)0;
          const T la = tb.lam[xa] + lo, lb = tb.lam[xa + 1] + lo;
          dsti_post<LOGM, T, T2>(Z, M, lane, [&](int pos, T2 v) {
            const T lp = tb.lam[pos];
            const T l_a = la + lp, l_b = lb + lp;
            const T d_a = m + l_a, d_b = m + l_b;
            O[pd(pos)] = mk<T2>(v.x * __fdividef(c * l_a, d_a * d_a), v.y * __fdividef(c * l_b, d_b * d_b));
          });
        }
        __syncwarp();
        T2* P2 = O == A ? B : A;
        dsti_pre<LOGM, T, T2>(P2, M, tb.sn, lane, [&](int pos) { return O[pd(pos)]; });
        __syncwarp();
        Z = fft_any<LOGM>(P2, O, LOGM, tb.tw, lane);
      }
      T2* O = Z == A ? B : A;
      dsti_post<LOGM, T, T2>(Z, M, lane, [&](int pos, T2 v) { O[pd(pos)] = v; });
      __syncwarp();
#pragma unroll
      for (int pos = lane; pos < M; pos += 32) at(pos) = O[pd(pos)];
      __syncwarp();
    }
  };
  if (MODE == 3) {
    cols();
  } else if (MODE == 2) {
    cols();
    __syncthreads();
    rows();
  } else {
    rows();
    __syncthreads();
    cols();
    if (MODE == 0) {
      __syncthreads();
      rows();
    }
  }
  __syncthreads();
  // store, the ghost row and column exactly zero
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
    const int yy = i >> LOGM, xx = i & (M - 1);
    xp[yy * RS + xx] = (yy == M - 1 || xx == M - 1) ? (T)0 : pl[yy * PITCH + xx];
  }
}

// g = c0 l / (mu_k + tau l)^2 at every padded point (0 at ghosts), l = sum of the axes' lam
template <typename T>
__global__ void k_dsti_scale_table(T* __restrict__ g, const double* __restrict__ lam, const double* __restrict__ mu,
                                   double tau, double c0, int dim, int logM, long long total) {
  const int M = 1 << logM;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long t = i >> (dim * logM);
    const long long rem = i & ((1LL << (dim * logM)) - 1);
    const int x = (int)(rem & (M - 1));
    const int y = (int)((rem >> logM) & (M - 1));
    const int z = dim == 3 ? (int)(rem >> (2 * logM)) : 0;
    double v = 0.0;
    if (x < M - 1 && y < M - 1 && z < M - 1) {
      const double l = lam[x] + lam[y] + (dim == 3 ? lam[z] : 0.0);
      const double d = mu[t] + tau * l;
      v = c0 * l / (d * d);
    }
    g[i] = (T)v;
  }
}

template <typename T>
int warps_for(int M) {
  const size_t per = (size_t)(2 * padded_len(M) + 1) * 2 * sizeof(T);
  int w = (int)((200u * 1024u) / per);
  if (w > kWarpsMax) w = kWarpsMax;
  return w < 1 ? 1 : w;
}

template <typename T>
DstiTabs<T> tabs(const void* tw, const void* sn, const void* g, const DstiFactor* f = nullptr) {
  DstiTabs<T> t;
  t.tw = (const typename Vec2<T>::type*)tw;
  t.sn = (const T*)sn;
  t.g = (const T*)g;
  t.lam = f ? (const T*)f->lam : nullptr;
  t.m = f ? (const T*)f->m : nullptr;
  t.c = f ? (T)f->c : (T)0;
  return t;
}

}  // namespace

template <typename T>
void launch_dsti_scale_table(T* g, const double* lam, const double* mu, double tau, double c0, int dim, int logP,
                             long long S, int B, cudaStream_t st) {
  const long long total = S * B;
  LaunchScope ls("dsti_table", st, sizeof(T) * (double)total);
  k_dsti_scale_table<T><<<grid_for(total), kThreads, 0, st>>>(g, lam, mu, tau, c0, dim, logP, total);
}
template void launch_dsti_scale_table<float>(float*, const double*, const double*, double, double, int, int,
                                             long long, int, cudaStream_t);
template void launch_dsti_scale_table<double>(double*, const double*, const double*, double, double, int, int,
                                              long long, int, cudaStream_t);

template <typename T>
void launch_dsti_rows(T* x, int dim, int n, int logP, long long S, int B, const void* tw, const void* sn,
                      cudaStream_t st) {
  using T2 = typename Vec2<T>::type;
  const int M = n + 1;
  const int wpb = warps_for<T>(M);
  const size_t smem = (size_t)wpb * (2 * padded_len(M) + 1) * sizeof(T2);
  const long long npairs = (long long)B * (S / M) / 2;
  long long blocks = (npairs + wpb - 1) / wpb;
  if (blocks > (1LL << 30)) blocks = 1LL << 30;
  double d = B;
  for (int k = 0; k < dim; ++k) d *= n;
  LaunchScope ls("dsti_rows", st, 2.0 * sizeof(T) * d);
  auto go = [&](auto kern) {
    set_smem_limit((const void*)kern, 210 * 1024);
    kern<<<(unsigned)blocks, wpb * 32, smem, st>>>(x, logP, dim, npairs, tabs<T>(tw, sn, nullptr));
  };
  // (the run-time-length kernel: unrolling the row transform raises its register count past
  // what its occupancy can afford, measured slower in both precisions)
  go(k_dsti_rows<T, 0>);
}

template <typename T>
bool dsti_plane_ok(int dim, int n) {
  return n + 1 <= kPlaneMaxM && n + 1 >= 32 && (dim == 3 || sizeof(T) == 4);
}

template <typename T>
void launch_dsti_plane(T* x, int dim, int n, int logP, long long S, int B, int mode, const void* tw, const void* sn,
                       const void* gtab, cudaStream_t st, const DstiFactor* factor) {
  using T2 = typename Vec2<T>::type;
  const int M = n + 1;
  const int planes = dim == 3 ? M : 1;
  const int wpb = logP >= 7 ? plane_warps<7>() : plane_warps<6>();
  const size_t smem = (size_t)M * (M + 2) * sizeof(T) + (size_t)wpb * (2 * padded_len(M) + 1) * sizeof(T2);
  double d = B;
  for (int k = 0; k < dim; ++k) d *= n;
  LaunchScope ls(mode == 0 ? "dsti_plane_solve" : (mode == 3 ? "dsti_plane_z" : "dsti_plane"), st,
                 2.0 * sizeof(T) * d);
  const dim3 grid((unsigned)((long long)B * planes));
  auto go = [&](auto kern) {
    set_smem_limit((const void*)kern, 210 * 1024);
    kern<<<grid, wpb * 32, smem, st>>>(x, S, planes, tabs<T>(tw, sn, gtab, factor));
  };
  // (mode 0 is the FP32 2-D form only: the FP64 2-D block solve takes its y-part by eliminations)
#define PT_PLANE(LM)                                                   \
  if (mode == 1)                                                       \
    go(k_dsti_plane<T, LM, 1>);                                        \
  else if (mode == 2)                                                  \
    go(k_dsti_plane<T, LM, 2>);                                        \
  else if (mode == 3)                                                  \
    go(k_dsti_plane<T, LM, 3>);                                        \
  else if constexpr (sizeof(T) == 4)                                   \
    go(k_dsti_plane<T, LM, 0>);
  if (logP == 5) {
    PT_PLANE(5)
  } else if (logP == 6) {
    PT_PLANE(6)
  } else {
    PT_PLANE(7)
  }
#undef PT_PLANE
}

template <typename T>
void launch_dsti_cols(T* x, int dim, int n, int logP, long long S, int B, int axis, const void* tw,
                      const void* sn, const void* gtab, bool scale, cudaStream_t st, const DstiFactor* factor) {
  using T2 = typename Vec2<T>::type;
  const int M = n + 1;
  int C = warps_for<T>(M);
  while (2 * C > M && C > 1) C >>= 1;
  while (C > 1 && (size_t)C * cols_stride<T>(padded_len(M)) * sizeof(T2) > 200 * 1024) C >>= 1;
  const size_t smem = (size_t)C * cols_stride<T>(padded_len(M)) * sizeof(T2);
  const long long planes = dim == 3 ? M : 1;
  const dim3 grid((unsigned)((M / (2 * C)) * planes), (unsigned)B);
  double d = B;
  for (int k = 0; k < dim; ++k) d *= n;
  LaunchScope ls(scale ? "dsti_cols_scale" : "dsti_cols", st, 2.0 * sizeof(T) * d);
  auto go = [&](auto kern) {
    set_smem_limit((const void*)kern, 210 * 1024);
    kern<<<grid, C * 32, smem, st>>>(x, logP, dim, axis, S, scale ? 1 : 0, tabs<T>(tw, sn, gtab, factor));
  };
  // FP32: compile-time lengths (instruction-bound, the unrolled form measured 11 % faster);
  // FP64: bound by the FP64 pipe either way, the run-time-length kernel (fewer registers)
  if (sizeof(T) == 4) {
    switch (logP) {
      case 5: go(k_dsti_cols<T, 5>); break;
      case 6: go(k_dsti_cols<T, 6>); break;
      case 7: go(k_dsti_cols<T, 7>); break;
      case 8: go(k_dsti_cols<T, 8>); break;
      case 9: go(k_dsti_cols<T, 9>); break;
      default: go(k_dsti_cols<T, 0>); break;
    }
  } else {
    go(k_dsti_cols<T, 0>);
  }
}

template void launch_dsti_rows<float>(float*, int, int, int, long long, int, const void*, const void*,
                                      cudaStream_t);
template void launch_dsti_rows<double>(double*, int, int, int, long long, int, const void*, const void*,
                                       cudaStream_t);
template bool dsti_plane_ok<float>(int, int);
template bool dsti_plane_ok<double>(int, int);
template void launch_dsti_plane<float>(float*, int, int, int, long long, int, int, const void*, const void*,
                                       const void*, cudaStream_t, const DstiFactor*);
template void launch_dsti_plane<double>(double*, int, int, int, long long, int, int, const void*, const void*,
                                        const void*, cudaStream_t, const DstiFactor*);
template void launch_dsti_cols<float>(float*, int, int, int, long long, int, int, const void*, const void*,
                                      const void*, bool, cudaStream_t, const DstiFactor*);
template void launch_dsti_cols<double>(double*, int, int, int, long long, int, int, const void*, const void*,
                                       const void*, bool, cudaStream_t, const DstiFactor*);

}  // namespace pt

// ---- FP64 2-D: the y-part of the exact block solve by tridiagonal eliminations ----
// After the x-transform, H_k restricted to one x-frequency is the symmetric Toeplitz tridiagonal
// T = tridiag(a, d, a), d = mu_k + tau (lam_x + 2 a0/h^2), a = -tau a0/h^2, and Abar is
// Z = c (lam_x + 2 a0/h^2) I - c (a0/h^2) (shift up + shift down).  So
//     y-part of Hhat_k^-1 = T^-1 Z T^-1
// by LU elimination (pivots w_i = 1/d'_i, d'_0 = d, d'_i = d - a^2 w_{i-1}, precomputed), and,
// because T is persymmetric, the second solve runs the same elimination from the bottom with the
// pivots in reverse order.  Three sweeps per column (down, up, down), one thread per column:
//   down: yh_i = (r_i - a yh_{i-1}) w_i
//   up:   x_i = yh_i - a w_i x_{i+1};   z_{i+1} = cd x_{i+1} - co (x_i + x_{i+2});
//         yh'_{i+1} = (z_{i+1} - a yh'_{i+2}) w_{n-2-i}
//   down: v_j = yh'_j - a w_{n-1-j} v_{j-1}
// 11 operations per point against 36 for two y-transforms and the factor.  Used in FP64 (the
// elimination's error grows with cond(T), which FP32 cannot afford).
namespace pt {
namespace {

template <typename T>
__global__ void k_hsolve_trid_table(T* __restrict__ w, const double* __restrict__ lam,
                                    const double* __restrict__ mu, double tau, double a0h2, int n, int logP,
                                    long long S, int N) {
  const int P = 1 << logP;
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (col >= (long long)N * P) return;
  const int k = (int)(col >> logP), x = (int)(col & (P - 1));
  if (x >= n) return;
  const double d = mu[k] + tau * (lam[x] + 2.0 * a0h2), a = -tau * a0h2;
  T* wc = w + (long long)k * S + x;
  double wi = 1.0 / d;  // pivots in FP64, stored in T
  wc[0] = (T)wi;
  for (int i = 1; i < n; ++i) {
    wi = 1.0 / (d - a * a * wi);
    wc[(long long)i * P] = (T)wi;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_hsolve_trid(T* __restrict__ X, const T* __restrict__ w,
                                                      const double* __restrict__ lam, double tau_d, double a0h2_d,
                                                      double scale_d, int n, int logP, long long S) {
  const int P = 1 << logP;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (x >= n) return;
  const T a = (T)(-tau_d * a0h2_d);
  const T cd = (T)(scale_d * (lam[x] + 2.0 * a0h2_d)), co = (T)(scale_d * a0h2_d);
  T* c = X + (long long)k * S + x;
  const T* wc = w + (long long)k * S + x;
  auto at = [&](int i) { return (long long)i * P; };
  // down: forward elimination with T
  T yh = (T)0;
#pragma unroll 4
  for (int i = 0; i < n; ++i) {
    yh = (c[at(i)] - a * yh) * wc[at(i)];
    c[at(i)] = yh;
  }
  // up: back substitution -> x_i; z one row behind; forward elimination of the reversed system
  T x2 = (T)0, x1 = (T)0, yr = (T)0;  // x_{i+2}, x_{i+1}, yh' of the row above
#pragma unroll 4
  for (int i = n - 1; i >= 0; --i) {
    const T xi = c[at(i)] - a * wc[at(i)] * x1;
    if (i + 1 <= n - 1) {
      const T z = cd * x1 - co * (xi + x2);  // row i+1
      yr = (z - a * yr) * wc[at(n - 2 - i)];
      c[at(i + 1)] = yr;
    }
    x2 = x1;
    x1 = xi;
  }
  {
    const T z = cd * x1 - co * x2;  // row 0 (x_{-1} = 0)
    yr = (z - a * yr) * wc[at(n - 1)];
    c[at(0)] = yr;
  }
  // down: back substitution of the reversed system
  T v = (T)0;
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    v = c[at(j)] - a * wc[at(n - 1 - j)] * v;
    c[at(j)] = v;
  }
}

}  // namespace

template <typename T>
void launch_hsolve_trid_table(T* w, const double* lam, const double* mu, double tau, double a0h2, int n, int logP,
                              long long S, int N, cudaStream_t st) {
  const long long cols = (long long)N << logP;
  LaunchScope ls("hsolve_table", st, sizeof(T) * (double)N * n * n);
  k_hsolve_trid_table<T><<<(unsigned)((cols + 127) / 128), 128, 0, st>>>(w, lam, mu, tau, a0h2, n, logP, S, N);
}

template <typename T>
void launch_hsolve_trid(T* X, const T* w, const double* lam, double tau, double a0h2, double scale, int n,
                        int logP, long long S, int N, cudaStream_t st) {
  const int P = 1 << logP;
  LaunchScope ls("hsolve_y", st, 7.0 * sizeof(T) * (double)N * n * n);
  const dim3 grid((unsigned)((P + 127) / 128), (unsigned)N);
  k_hsolve_trid<T><<<grid, 128, 0, st>>>(X, w, lam, tau, a0h2, scale, n, logP, S);
}
template void launch_hsolve_trid_table<float>(float*, const double*, const double*, double, double, int, int,
                                              long long, int, cudaStream_t);
template void launch_hsolve_trid_table<double>(double*, const double*, const double*, double, double, int, int,
                                               long long, int, cudaStream_t);
template void launch_hsolve_trid<float>(float*, const float*, const double*, double, double, double, int, int,
                                        long long, int, cudaStream_t);
template void launch_hsolve_trid<double>(double*, const double*, const double*, double, double, double, int, int,
                                         long long, int, cudaStream_t);

}  // namespace pt
