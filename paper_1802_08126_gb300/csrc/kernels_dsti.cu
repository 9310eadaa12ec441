// Exact spatial solves for the Schur preconditioner when the reference operator has a constant
// coefficient (Abar = a0 L_h, L_h the finite-difference Laplacian).  The sine transform of type I
// along each axis, (S v)_k = sum_{j=1}^{n} v_j sin(pi j k / (n+1)), diagonalises L_h with
// eigenvalues (4/h^2) sum_d sin^2(pi k_d h / 2) and satisfies S S = ((n+1)/2) I.  Hence the block
// solve of §4, eq. 4.4,
//     Hhat_k^-1 = (2 tau / N) H_k^-1 Abar H_k^-1,  H_k = mu_k I + tau Abar,
// is, in the doubly transformed basis, the point-wise factor
//     (2 tau / N) (2/(n+1))^d a0 l / (mu_k + tau a0 l)^2,   l = the eigenvalue of L_h,
// between two spatial transforms (this is the exact H of eq. 4.4, gamma = Gamma = 1 in eq. 4.7).
//
// Each 1-D transform is computed through one complex FFT of length 2(n+1) of the odd extension
// [0, v_1 .. v_n, 0, -v_n .. -v_1], whose spectrum is -2i (S v); two real lines share one complex
// transform (real and imaginary parts).  Rows (x) are contiguous; columns (y, z) are strided by
// the pitch and are handled as tiles of consecutive columns, like the temporal transform.
#include "fft_common.cuh"

namespace pt {
namespace {

struct DstIArgs {
  int n, M, logM2;   // interior points, M = n + 1, log2(2M)
  int dim;
  long long S;       // slice stride
  long long stride;  // element distance between consecutive points along the transformed axis
  int nlines_slice;  // lines of one slice along this axis (including ghost lines)
};

// odd extension of line pair (a, b) into column c of the FFT buffer (length 2M, stride L)
template <typename T, typename T2>
__device__ __forceinline__ void put_odd(T2* col, int M, int j, T va, T vb) {
  T2 v, w;
  v.x = va;
  v.y = vb;
  w.x = -va;
  w.y = -vb;
  col[j + 1] = v;          // v_{j+1} at position j+1
  col[2 * M - 1 - j] = w;  // -v_{j+1} at position 2M - (j+1)
}

// rows along x, in place: v <- S v for every (slice, y, z) line
template <typename T>
__global__ void k_dsti_rows(T* x, DstIArgs a, const typename Vec2<T>::type* __restrict__ tw, int C,
                            long long nlines) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* buf = (T2*)smem_raw;
  const int L = 2 * a.M + 1;
  const long long line0 = (long long)blockIdx.x * 2 * C;
  const int P = a.M;
  for (int idx = threadIdx.x; idx < C * a.n; idx += blockDim.x) {
    const int c = idx / a.n, j = idx - c * a.n;
    const long long la = line0 + 2 * c, lb = la + 1;
    const T va = la < nlines ? x[la * P + j] : (T)0;
    const T vb = lb < nlines ? x[lb * P + j] : (T)0;
    put_odd<T, T2>(buf + (size_t)c * L, a.M, j, va, vb);
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    T2 z;
    z.x = (T)0;
    z.y = (T)0;
    buf[(size_t)c * L] = z;
    buf[(size_t)c * L + a.M] = z;
  }
  __syncthreads();
  dif_fft<T, T2>(buf, C, L, 2 * a.M, a.logM2, tw, (T)-1);
  // (S v_a)_k = -Im C_k / 2, (S v_b)_k = Re C_k / 2; the ghost entry (and ghost lines) stay zero
  for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
    const int c = idx / P, k = idx - c * P;
    const long long la = line0 + 2 * c, lb = la + 1;
    T ya = (T)0, yb = (T)0;
    if (k < a.n) {
      const T2 v = buf[(size_t)c * L + bitrev(k + 1, a.logM2)];
      ya = (T)-0.5 * v.y;
      yb = (T)0.5 * v.x;
    }
    const int ga = (int)(la % a.nlines_slice), gb = (int)(lb % a.nlines_slice);
    // line index within a slice: y (2-D) or z*P + y (3-D); ghost when y == n or z == n
    auto ghost = [&](int li) { return (li % P) == a.n || (a.dim == 3 && (li / P) == a.n); };
    if (la < nlines) x[la * P + k] = ghost(ga) ? (T)0 : ya;
    if (lb < nlines) x[lb * P + k] = ghost(gb) ? (T)0 : yb;
  }
}

// Columns along a strided axis: v <- S v; with `scale`, v <- S diag(g) S v where g is the exact
// block solve factor of the header comment (computed from the frequencies of all axes).
struct ScaleArgs {
  int enabled;
  const double* lam;   // [n] (4 a0 / h^2) sin^2(pi k h / 2), k = 1..n (x, y and z share it)
  const double* mu;    // [N] mu_k of the temporal basis
  double tau;          // reference step
  double c0;           // (2 tau / N) (2 / M)^d
};

template <typename T>
__global__ void k_dsti_cols(T* x, DstIArgs a, ScaleArgs sc, const typename Vec2<T>::type* __restrict__ tw,
                            int C) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 2 * a.M + 1;
  T2* buf = (T2*)smem_raw;
  T2* buf2 = buf + (size_t)C * L;  // second buffer for the transform back (scale mode)
  const int P = a.M;
  const int slice = blockIdx.y;
  // the 2C columns of this block: consecutive indices within the plane orthogonal to the axis
  const long long col0 = (long long)blockIdx.x * 2 * C;
  // column q -> base offset within the slice: for the y axis (stride P) q = z*P + x, for the z
  // axis (stride P^2) q = y*P + x
  auto col_base = [&](long long q) -> long long {
    if (a.stride == P) return (q / P) * (long long)P * P + (q % P);  // y axis: plane z, column x
    return q;                                                          // z axis: q = y*P + x
  };
  const long long sbase = (long long)slice * a.S;
  for (int idx = threadIdx.x; idx < C * a.n; idx += blockDim.x) {
    const int j = idx / C, c = idx - j * C;  // c fastest: consecutive columns, coalesced
    const long long qa = col0 + 2 * c;
    const T va = x[sbase + col_base(qa) + (long long)j * a.stride];
    const T vb = x[sbase + col_base(qa + 1) + (long long)j * a.stride];
    put_odd<T, T2>(buf + (size_t)c * L, a.M, j, va, vb);
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    T2 z;
    z.x = (T)0;
    z.y = (T)0;
    buf[(size_t)c * L] = z;
    buf[(size_t)c * L + a.M] = z;
    if (sc.enabled) {
      buf2[(size_t)c * L] = z;
      buf2[(size_t)c * L + a.M] = z;
    }
  }
  __syncthreads();
  dif_fft<T, T2>(buf, C, L, 2 * a.M, a.logM2, tw, (T)-1);
  T2* out = buf;
  if (sc.enabled) {
    // spectrum -> scaled odd extension in buf2 -> transform again
    const double mu = sc.mu[slice];
    for (int idx = threadIdx.x; idx < C * a.n; idx += blockDim.x) {
      const int c = idx / a.n, k = idx - c * a.n;
      const T2 v = buf[(size_t)c * L + bitrev(k + 1, a.logM2)];
      const long long qa = col0 + 2 * c;
      T g[2];
      for (int s = 0; s < 2; ++s) {
        const long long q = qa + s;
        const int cx = (int)(q % P);
        const int cy = (int)(q / P);  // y index (z-axis pass) or z index (y-axis pass, 3-D)
        double l = (cx < a.n ? sc.lam[cx] : 0.0) + sc.lam[k];
        if (a.dim == 3) l += cy < a.n ? sc.lam[cy] : 0.0;
        const bool ghost = cx >= a.n || (a.dim == 3 && cy >= a.n);
        const double d = mu + sc.tau * l;
        g[s] = ghost ? (T)0 : (T)(sc.c0 * l / (d * d));
      }
      put_odd<T, T2>(buf2 + (size_t)c * L, a.M, k, (T)-0.5 * v.y * g[0], (T)0.5 * v.x * g[1]);
    }
    __syncthreads();
    dif_fft<T, T2>(buf2, C, L, 2 * a.M, a.logM2, tw, (T)-1);
    out = buf2;
  }
  for (int idx = threadIdx.x; idx < C * P; idx += blockDim.x) {
    const int k = idx / C, c = idx - k * C;
    const long long qa = col0 + 2 * c;
    T ya = (T)0, yb = (T)0;
    if (k < a.n) {
      const T2 v = out[(size_t)c * L + bitrev(k + 1, a.logM2)];
      ya = (T)-0.5 * v.y;
      yb = (T)0.5 * v.x;
    }
    auto gh = [&](long long q) {
      const int cx = (int)(q % P), cy = (int)(q / P);
      return cx >= a.n || (a.dim == 3 && cy >= a.n);
    };
    x[sbase + col_base(qa) + (long long)k * a.stride] = gh(qa) ? (T)0 : ya;
    x[sbase + col_base(qa + 1) + (long long)k * a.stride] = gh(qa + 1) ? (T)0 : yb;
  }
}

template <typename T>
int lines_per_block(int M, int max_bytes) {
  const long long bytes = (long long)(2 * M + 1) * 2 * sizeof(T);
  long long C = max_bytes / bytes;
  if (C < 1) C = 1;
  if (C > 16) C = 16;
  long long pw = 1;
  while (pw * 2 <= C) pw *= 2;
  return (int)pw;
}

}  // namespace

template <typename T>
void launch_dsti_rows(T* x, int dim, int n, int logP, long long S, int B, const T* tw, cudaStream_t st) {
  using T2 = typename Vec2<T>::type;
  DstIArgs a;
  a.n = n;
  a.M = n + 1;
  a.logM2 = logP + 1;
  a.dim = dim;
  a.S = S;
  a.stride = 1;
  a.nlines_slice = (int)(S / a.M);
  const long long nlines = (long long)B * a.nlines_slice;
  const int C = lines_per_block<T>(a.M, 64 * 1024);
  const size_t smem = (size_t)C * (2 * a.M + 1) * sizeof(T2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dsti_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const long long blocks = (nlines + 2 * C - 1) / (2 * C);
  double d = B;
  for (int k = 0; k < dim; ++k) d *= n;
  LaunchScope ls("dsti_rows", st, 2.0 * sizeof(T) * d);
  k_dsti_rows<T><<<(unsigned)blocks, kThreads, smem, st>>>(x, a, (const T2*)tw, C, nlines);
}

template <typename T>
void launch_dsti_cols(T* x, int dim, int n, int logP, long long S, int B, int axis, const T* tw,
                      const double* lam, const double* mu, double tau, double c0, bool scale, cudaStream_t st) {
  using T2 = typename Vec2<T>::type;
  DstIArgs a;
  a.n = n;
  a.M = n + 1;
  a.logM2 = logP + 1;
  a.dim = dim;
  a.S = S;
  a.stride = axis == 1 ? (long long)a.M : (long long)a.M * a.M;
  a.nlines_slice = (int)(S / a.M);
  ScaleArgs sc;
  sc.enabled = scale ? 1 : 0;
  sc.lam = lam;
  sc.mu = mu;
  sc.tau = tau;
  sc.c0 = c0;
  const long long cols = S / a.M;  // columns of one slice orthogonal to this axis (incl. ghosts)
  int C = lines_per_block<T>(a.M, scale ? 48 * 1024 : 64 * 1024);
  while (2LL * C > cols && C > 1) C >>= 1;
  const size_t smem = (size_t)C * (2 * a.M + 1) * sizeof(T2) * (scale ? 2 : 1);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dsti_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const dim3 grid((unsigned)((cols + 2 * C - 1) / (2 * C)), (unsigned)B);
  double d = B;
  for (int k = 0; k < dim; ++k) d *= n;
  LaunchScope ls(scale ? "dsti_cols_scale" : "dsti_cols", st, 2.0 * sizeof(T) * d);
  k_dsti_cols<T><<<grid, kThreads, smem, st>>>(x, a, sc, (const T2*)tw, C);
}

template void launch_dsti_rows<float>(float*, int, int, int, long long, int, const float*, cudaStream_t);
template void launch_dsti_rows<double>(double*, int, int, int, long long, int, const double*, cudaStream_t);
template void launch_dsti_cols<float>(float*, int, int, int, long long, int, int, const float*, const double*,
                                      const double*, double, double, bool, cudaStream_t);
template void launch_dsti_cols<double>(double*, int, int, int, long long, int, int, const double*, const double*,
                                       const double*, double, double, bool, cudaStream_t);

}  // namespace pt
