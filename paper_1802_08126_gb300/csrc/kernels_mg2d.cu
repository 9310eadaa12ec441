// Fused 2-D multigrid level kernels (same V(1,1) as kernels_mg.cu, fewer passes over HBM).
//
// With a zero initial guess the pre-smoothed iterate is x1 = w D^-1 b, a point-wise function of
// the right-hand side, so it is never stored: the "down" kernel forms x1, the residual
// r = b - L x1 and its full-weighting restriction in shared memory and writes only the coarse
// right-hand side; the "up" kernel re-forms x1 from b, adds the prolonged coarse correction,
// applies the post-smoothing step x3 = x2 + w D^-1 (b - L x2), and writes (or accumulates) x3.
// Per level the fine grid is read twice and written once.
//
// Face coefficients are formed in shared memory from the 1-D tables (VAR) or are the constant
// a0 (the reference operator Abar has a time-mean coefficient, constant for every workload
// whose coefficient oscillates in time).  The Jacobi factor w D^-1 is a per-slice constant
// (constant coefficient), read from a per-level cache (FP64 variable coefficient, where the
// division would dominate the FP64 instruction budget), or computed (FP32).
#include <type_traits>

#include "stencil_common.cuh"

namespace pt {
namespace {

constexpr int kDownTX = 16, kDownTY = 8;  // coarse points per down tile
constexpr int kUpTX = 32, kUpTY = 16;     // fine points per up tile
constexpr int kStripMinP = 64;            // fine levels at least this wide use the warp-strip kernels

template <typename T>
struct Mg2Args {
  int nf, logPf;      // fine level
  long long Sf;
  int nc, logPc;      // coarse level
  long long Sc;
  const T* tab;       // fine-level tables: node_x, face_x, node_y, face_y (Pf each)
  T a0s;              // s * a0 / h^2
  T s_h2;             // s / h^2
  const T* sig;       // [B]
  const T* cth;       // [B]
  const T* dinv;      // [B] w / D per slice (DM == 0)
  const T* jinv;      // cached pairs (w / D, D) per point, fine padded layout (DM == 1)
  T omega;
};

// face coefficients of region (rows RH, cols RW, origin fy0, fx0), scaled by s/h^2:
//   fxs[ry][rx] = lower x-face of point (fy0+ry, fx0+rx), rx in [0, RW]
//   fys[ry][rx] = lower y-face of point (fy0+ry, fx0+rx), ry in [0, RH]
template <typename T>
__device__ __forceinline__ void load_faces(T* fxs, T* fys, int RW, int RH, int fx0, int fy0,
                                           const Mg2Args<T>& a, T cths) {
  const int Pf = 1 << a.logPf;
  const T* nx = a.tab;
  const T* fx = a.tab + Pf;
  const T* ny = a.tab + 2 * Pf;
  const T* fy = a.tab + 3 * Pf;
  for (int k = threadIdx.x; k < RH * (RW + 1); k += blockDim.x) {
    const int ry = k / (RW + 1), rx = k - ry * (RW + 1);
    const int x = fx0 + rx, y = fy0 + ry;
    T v = (T)0;
    if (y >= 0 && y < a.nf && x >= 0 && x <= a.nf) v = a.a0s + cths * ny[y] * fx[x];
    fxs[k] = v;
  }
  for (int k = threadIdx.x; k < (RH + 1) * RW; k += blockDim.x) {
    const int ry = k / RW, rx = k - ry * RW;
    const int x = fx0 + rx, y = fy0 + ry;
    T v = (T)0;
    if (x >= 0 && x < a.nf && y >= 0 && y <= a.nf) v = a.a0s + cths * nx[x] * fy[y];
    fys[k] = v;
  }
}

// w D^-1 at region point (ry, rx) = fine (y, x), interior only
template <typename T, bool VAR, int DM>
__device__ __forceinline__ T jacobi_factor(const Mg2Args<T>& a, int b, long long gi, const T* fxs,
                                           const T* fys, int RW, int ry, int rx, T sig) {
  if (DM == 0) return a.dinv[b];
  if (DM == 1) return a.jinv[2 * gi];
  T dsum;
  if (VAR) {
    dsum = fxs[ry * (RW + 1) + rx] + fxs[ry * (RW + 1) + rx + 1] + fys[ry * RW + rx] + fys[(ry + 1) * RW + rx];
  } else {
    dsum = (T)4 * a.a0s;
  }
  return a.omega / (sig + dsum);
}

template <typename T, bool VAR, int DM>
__global__ void __launch_bounds__(256) k_mg2_down(const T* __restrict__ bf, T* __restrict__ bc,
                                                  Mg2Args<T> a, const int* done) {
  if (stop_requested(done)) return;
  constexpr int RW = 2 * kDownTX + 3, RH = 2 * kDownTY + 3;
  __shared__ T sb[RH * RW];
  __shared__ T sx[RH * RW];
  __shared__ T sr[(RH - 2) * (RW - 2)];
  __shared__ T sfx[VAR ? RH * (RW + 1) : 1];
  __shared__ T sfy[VAR ? (RH + 1) * RW : 1];
  const int b = blockIdx.z;
  const int X0 = blockIdx.x * kDownTX, Y0 = blockIdx.y * kDownTY;  // coarse tile origin
  const int fx0 = 2 * X0 - 1, fy0 = 2 * Y0 - 1;                   // fine region origin
  const int Pf = 1 << a.logPf;
  const long long base = (long long)b * a.Sf;
  const T sig = a.sig[b];
  const T cths = a.s_h2 * a.cth[b];
  if (VAR) load_faces<T>(sfx, sfy, RW, RH, fx0, fy0, a, cths);
  __syncthreads();
  // b and x1 = w D^-1 b on the region (zero outside the interior)
  for (int k = threadIdx.x; k < RH * RW; k += blockDim.x) {
    const int ry = k / RW, rx = k - ry * RW;
    const int x = fx0 + rx, y = fy0 + ry;
    T bv = (T)0, xv = (T)0;
    if (x >= 0 && x < a.nf && y >= 0 && y < a.nf) {
      const long long gi = base + (long long)y * Pf + x;
      bv = bf[gi];
      xv = bv * jacobi_factor<T, VAR, DM>(a, b, gi, sfx, sfy, RW, ry, rx, sig);
    }
    sb[k] = bv;
    sx[k] = xv;
  }
  __syncthreads();
  // r = b - L x1 on the inner region (fine points 2X0 .. 2X0 + 2 TX)
  for (int k = threadIdx.x; k < (RH - 2) * (RW - 2); k += blockDim.x) {
    const int iy = k / (RW - 2), ix = k - iy * (RW - 2);
    const int ry = iy + 1, rx = ix + 1;
    const int c = ry * RW + rx;
    const T xc = sx[c];
    T Lx;
    if (DM == 1) {
      // cached diagonal D = sig + sum of faces: L x = D x_c - sum_f a_f x_f (fewer FP64 operations)
      const int x = fx0 + rx, y = fy0 + ry;
      Lx = (T)0;
      if (x < a.nf && y < a.nf) {
        const T D = a.jinv[2 * (base + (long long)y * Pf + x) + 1];
        const T aw = sfx[ry * (RW + 1) + rx], ae = sfx[ry * (RW + 1) + rx + 1];
        const T as = sfy[ry * RW + rx], an = sfy[(ry + 1) * RW + rx];
        Lx = D * xc - (aw * sx[c - 1] + ae * sx[c + 1] + as * sx[c - RW] + an * sx[c + RW]);
      }
    } else if (VAR) {
      const T aw = sfx[ry * (RW + 1) + rx], ae = sfx[ry * (RW + 1) + rx + 1];
      const T as = sfy[ry * RW + rx], an = sfy[(ry + 1) * RW + rx];
      Lx = sig * xc + aw * (xc - sx[c - 1]) + ae * (xc - sx[c + 1]) + as * (xc - sx[c - RW]) +
           an * (xc - sx[c + RW]);
    } else {
      Lx = (sig + (T)4 * a.a0s) * xc - a.a0s * ((sx[c - 1] + sx[c + 1]) + (sx[c - RW] + sx[c + RW]));
    }
    sr[k] = sb[c] - Lx;
  }
  __syncthreads();
  // full weighting onto the coarse tile
  const int Pc = 1 << a.logPc;
  for (int k = threadIdx.x; k < kDownTX * kDownTY; k += blockDim.x) {
    const int cy = k / kDownTX, cx = k - cy * kDownTX;
    const int X = X0 + cx, Y = Y0 + cy;
    if (X >= a.nc || Y >= a.nc) continue;
    const int RW2 = RW - 2;
    const int c = (2 * cy + 1) * RW2 + (2 * cx + 1);
    const T r0 = (T)0.25 * (sr[c - RW2 - 1] + sr[c - RW2 + 1]) + (T)0.5 * sr[c - RW2];
    const T r1 = (T)0.25 * (sr[c - 1] + sr[c + 1]) + (T)0.5 * sr[c];
    const T r2 = (T)0.25 * (sr[c + RW2 - 1] + sr[c + RW2 + 1]) + (T)0.5 * sr[c + RW2];
    bc[(long long)b * a.Sc + (long long)Y * Pc + X] = (T)0.25 * (r0 + r2) + (T)0.5 * r1;
  }
}

template <typename T, bool VAR, int DM>
__global__ void __launch_bounds__(256) k_mg2_up(const T* __restrict__ bf, const T* __restrict__ ec,
                                                void* out, int mode, int out_fp64, Mg2Args<T> a,
                                                const int* done) {
  if (stop_requested(done)) return;
  constexpr int RW = kUpTX + 2, RH = kUpTY + 2;
  constexpr int CW = kUpTX / 2 + 2, CH = kUpTY / 2 + 2;
  __shared__ T sb[RH * RW];
  __shared__ T sx[RH * RW];
  __shared__ T se[CH * CW];
  __shared__ T sfx[VAR ? RH * (RW + 1) : 1];
  __shared__ T sfy[VAR ? (RH + 1) * RW : 1];
  const int b = blockIdx.z;
  const int X0 = blockIdx.x * kUpTX, Y0 = blockIdx.y * kUpTY;  // fine tile origin (even)
  const int fx0 = X0 - 1, fy0 = Y0 - 1;
  const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;                 // coarse region origin
  const int Pf = 1 << a.logPf, Pc = 1 << a.logPc;
  const long long base = (long long)b * a.Sf;
  const T sig = a.sig[b];
  const T cths = a.s_h2 * a.cth[b];
  if (VAR) load_faces<T>(sfx, sfy, RW, RH, fx0, fy0, a, cths);
  for (int k = threadIdx.x; k < CH * CW; k += blockDim.x) {
    const int cy = k / CW, cx = k - cy * CW;
    const int X = cx0 + cx, Y = cy0 + cy;
    se[k] = (X >= 0 && X < a.nc && Y >= 0 && Y < a.nc) ? ec[(long long)b * a.Sc + (long long)Y * Pc + X] : (T)0;
  }
  __syncthreads();
  // x2 = w D^-1 b + P e on the region
  for (int k = threadIdx.x; k < RH * RW; k += blockDim.x) {
    const int ry = k / RW, rx = k - ry * RW;
    const int x = fx0 + rx, y = fy0 + ry;
    T bv = (T)0, xv = (T)0;
    if (x >= 0 && x < a.nf && y >= 0 && y < a.nf) {
      const long long gi = base + (long long)y * Pf + x;
      bv = bf[gi];
      xv = bv * jacobi_factor<T, VAR, DM>(a, b, gi, sfx, sfy, RW, ry, rx, sig);
      // d-linear interpolation: odd fine index = coarse point (x-1)/2, even = mean of x/2-1, x/2
      const int ex = (x >> 1) - cx0, ey = (y >> 1) - cy0;  // smem index of coarse x/2, y/2
      T row0, row1;
      if (x & 1) {
        row0 = se[(ey - ((y & 1) ? 0 : 1)) * CW + ex];
        row1 = se[ey * CW + ex];
      } else {
        row0 = (T)0.5 * (se[(ey - ((y & 1) ? 0 : 1)) * CW + ex - 1] + se[(ey - ((y & 1) ? 0 : 1)) * CW + ex]);
        row1 = (T)0.5 * (se[ey * CW + ex - 1] + se[ey * CW + ex]);
      }
      xv += (y & 1) ? row1 : (T)0.5 * (row0 + row1);
    }
    sb[k] = bv;
    sx[k] = xv;
  }
  __syncthreads();
  // x3 = x2 + w D^-1 (b - L x2) on the tile
  for (int k = threadIdx.x; k < kUpTX * kUpTY; k += blockDim.x) {
    const int iy = k / kUpTX, ix = k - iy * kUpTX;
    const int x = X0 + ix, y = Y0 + iy;
    if (x >= Pf || y >= Pf) continue;
    const long long gi = base + (long long)y * Pf + x;
    if (x >= a.nf || y >= a.nf) {
      if (mode == 0) store_out<T>(out, gi, 0, out_fp64, (T)0);
      continue;
    }
    const int ry = iy + 1, rx = ix + 1;
    const int c = ry * RW + rx;
    const T xc = sx[c];
    T Lx;
    if (VAR) {
      const T aw = sfx[ry * (RW + 1) + rx], ae = sfx[ry * (RW + 1) + rx + 1];
      const T as = sfy[ry * RW + rx], an = sfy[(ry + 1) * RW + rx];
      Lx = sig * xc + aw * (xc - sx[c - 1]) + ae * (xc - sx[c + 1]) + as * (xc - sx[c - RW]) +
           an * (xc - sx[c + RW]);
    } else {
      Lx = (sig + (T)4 * a.a0s) * xc - a.a0s * ((sx[c - 1] + sx[c + 1]) + (sx[c - RW] + sx[c + RW]));
    }
    const T jf = jacobi_factor<T, VAR, DM>(a, b, gi, sfx, sfy, RW, ry, rx, sig);
    store_out<T>(out, gi, mode, out_fp64, xc + jf * (sb[c] - Lx));
  }
}

// ---- warp-strip forms of the two level kernels (fine levels with P >= 64) ----
// A warp owns a band of consecutive fine columns, one per lane, and sweeps a strip of fine rows
// keeping the rows above and below in registers; x-neighbours come from warp shuffles.  The
// bands overlap by the halo so that no lane needs a value from outside its warp.

constexpr int kStripDownCols = 14;  // coarse columns per down warp (fine columns 2X0-1 .. 2X0+29)
constexpr int kStripDownRows = 16;  // coarse rows per down warp
constexpr int kStripUpCols = 30;    // fine output columns per up warp (lanes 1..30)
constexpr int kStripUpRows = 32;    // fine rows per up warp

// Face coefficients (scaled by s/h^2) of the lane's point (y, x).  FP64: formed once per face --
// the lane computes its lower x-face and upper y-face; the upper x-face is the lower x-face of
// the lane to the right (shuffle) and the lower y-face is the upper y-face of the row before.
template <typename T, bool VAR>
struct Faces {
  T xl, xr, yl, yu;
};
template <typename T, bool VAR>
struct FaceSweep {
  T gx;       // (s/h^2) c g_t g_x(x)
  T yu_last;  // upper y-face of the previous row (= lower y-face of the next)
  bool xok;   // 0 <= x <= n: the lane's lower x-face exists
  __device__ __forceinline__ void init(const Mg2Args<T>& a, const T* nx, const T* fy, T cths, int x, int y) {
    xok = x >= 0 && x <= a.nf;
    gx = (VAR && x >= 0 && x < a.nf) ? cths * nx[x] : (T)0;
    yu_last = (VAR && y >= 0 && y <= a.nf) ? fma(gx, fy[y], a.a0s) : a.a0s;
  }
  // faces of row y (every lane calls it, rows in increasing order).  Sharing saves FP64
  // instructions; in FP32 the shuffle costs more than the two multiply-adds it replaces.
  __device__ __forceinline__ Faces<T, VAR> row(const Mg2Args<T>& a, const T* fx, const T* ny, const T* fy, T cths,
                                               int x, int y) {
    Faces<T, VAR> f;
    if (VAR && sizeof(T) == 4) {
      f.xl = f.xr = f.yl = f.yu = (T)0;
      if (y >= 0 && y < a.nf && x >= 0 && x < a.nf) {
        const T gy = cths * ny[y];
        f.xl = fma(gy, fx[x], a.a0s);
        f.xr = fma(gy, fx[x + 1], a.a0s);
        f.yl = fma(gx, fy[y], a.a0s);
        f.yu = fma(gx, fy[y + 1], a.a0s);
      }
    } else if (VAR) {
      const bool yok = y >= 0 && y < a.nf;
      const T xl = (yok && xok) ? fma(cths * ny[y], fx[x], a.a0s) : (T)0;
      f.xl = xl;
      f.xr = __shfl_down_sync(0xffffffffu, xl, 1);
      if ((threadIdx.x & 31) == 31) f.xr = (yok && x + 1 <= a.nf) ? fma(cths * ny[y], fx[x + 1], a.a0s) : (T)0;
      f.yl = yu_last;
      f.yu = (y + 1 >= 0 && y + 1 <= a.nf) ? fma(gx, fy[y + 1], a.a0s) : a.a0s;
      yu_last = f.yu;
    } else {
      f.xl = f.xr = f.yl = f.yu = a.a0s;
    }
    return f;
  }
};

template <typename T, bool VAR, int DM>
__device__ __forceinline__ T jacobi_at(const Mg2Args<T>& a, int b, long long gi, const Faces<T, VAR>& f, T sig) {
  if (DM == 0) return a.dinv[b];
  if (DM == 1) return a.jinv[2 * gi];
  return a.omega / (sig + ((f.xl + f.xr) + (f.yl + f.yu)));
}

template <typename T, bool VAR, int DM>
__global__ void __launch_bounds__(256) k_mg2s_down(const T* __restrict__ bf, T* __restrict__ bc, Mg2Args<T> a,
                                                   int wpr, int strips, long long nwarps, const int* done) {
  if (stop_requested(done)) return;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wg >= nwarps) return;  // warp-uniform; no block-level barrier in this kernel
  const int lane = threadIdx.x & 31;
  const int wx = (int)(wg % wpr);
  const long long rest = wg / wpr;
  const int strip = (int)(rest % strips);
  const int b = (int)(rest / strips);
  const int X0 = kStripDownCols * wx, Y0 = kStripDownRows * strip;
  const int x = 2 * X0 - 1 + lane;  // fine column of this lane
  const int nf = a.nf, Pf = 1 << a.logPf, Pc = 1 << a.logPc;
  const bool xin = x >= 0 && x < nf;
  const long long base = (long long)b * a.Sf;
  const T sig = a.sig[b];
  const T cths = a.s_h2 * a.cth[b];
  const T* nx = a.tab;
  const T* fx = a.tab + Pf;
  const T* ny = a.tab + 2 * Pf;
  const T* fy = a.tab + 3 * Pf;
  const int yfirst = 2 * Y0 - 1, ylast = 2 * (Y0 + kStripDownRows);  // x1 rows needed: yfirst .. ylast + 1
  FaceSweep<T, VAR> fs;
  fs.init(a, nx, fy, cths, x, yfirst);
  // x1 = w D^-1 b and everything the residual at that row needs
  auto ld_b = [&](int y) -> T { return (xin && y >= 0 && y < nf) ? bf[base + (long long)y * Pf + x] : (T)0; };
  auto row = [&](int y, T bload, T& bv, T& x1, Faces<T, VAR>& f) {
    f = fs.row(a, fx, ny, fy, cths, x, y);
    bv = (T)0;
    x1 = (T)0;
    if (xin && y >= 0 && y < nf) {
      const long long gi = base + (long long)y * Pf + x;
      bv = bload;
      x1 = bv * jacobi_at<T, VAR, DM>(a, b, gi, f, sig);
    }
  };
  T bm, xm, bc_, xc, bn, xn;
  Faces<T, VAR> fm, fc, fn;
  row(yfirst, ld_b(yfirst), bm, xm, fm);
  row(yfirst + 1, ld_b(yfirst + 1), bc_, xc, fc);
  T b_next = ld_b(yfirst + 2);  // b of the row after next, loaded one iteration ahead
  T h1 = (T)0, h2 = (T)0;  // horizontal restrictions of the two previous rows
  const bool out_lane = (lane & 1) == 0 && lane >= 2 && lane <= 28;
  const int X = X0 + (lane >> 1) - 1;  // coarse column of an output lane (x = 2X + 1)
  for (int y = yfirst + 1; y <= ylast; ++y) {
    const T b_after = ld_b(y + 2);
    row(y + 1, b_next, bn, xn, fn);
    b_next = b_after;
    // residual of x1 at row y
    const T xW = __shfl_up_sync(0xffffffffu, xc, 1);
    const T xE = __shfl_down_sync(0xffffffffu, xc, 1);
    T r = (T)0;
    if (xin && y >= 0 && y < nf) {
      T Lx;
      if (VAR)
        Lx = sig * xc + fc.xl * (xc - xW) + fc.xr * (xc - xE) + fc.yl * (xc - xm) + fc.yu * (xc - xn);
      else
        Lx = (sig + (T)4 * a.a0s) * xc - a.a0s * ((xW + xE) + (xm + xn));
      r = bc_ - Lx;
    }
    const T rW = __shfl_up_sync(0xffffffffu, r, 1);
    const T rE = __shfl_down_sync(0xffffffffu, r, 1);
    const T h = (T)0.25 * (rW + rE) + (T)0.5 * r;
    // coarse row Y = (y - 2)/2 - ... : rows 2Y, 2Y+1, 2Y+2 are complete when y = 2Y + 2
    if (y >= 2 * Y0 + 2 && ((y - 2 * Y0) & 1) == 0) {
      const int Y = (y >> 1) - 1;
      if (out_lane && X < a.nc && Y < a.nc)
        bc[(long long)b * a.Sc + (long long)Y * Pc + X] = (T)0.25 * (h2 + h) + (T)0.5 * h1;
    }
    h2 = h1;
    h1 = h;
    bm = bc_;
    xm = xc;
    fm = fc;
    bc_ = bn;
    xc = xn;
    fc = fn;
  }
  (void)bm;
  (void)fm;
}

template <typename T, bool VAR, int DM>
__global__ void __launch_bounds__(256) k_mg2s_up(const T* __restrict__ bf, const T* __restrict__ ec, void* out,
                                                 int mode, int out_fp64, Mg2Args<T> a, int wpr, int strips,
                                                 long long nwarps, const int* done) {
  using T2c = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  if (stop_requested(done)) return;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wg >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int wx = (int)(wg % wpr);
  const long long rest = wg / wpr;
  const int strip = (int)(rest % strips);
  const int b = (int)(rest / strips);
  const int x = kStripUpCols * wx - 1 + lane;  // fine column; lanes 1..30 write
  const int y0 = kStripUpRows * strip;
  const int nf = a.nf, nc = a.nc, Pf = 1 << a.logPf, Pc = 1 << a.logPc;
  const bool xin = x >= 0 && x < nf;
  const long long base = (long long)b * a.Sf;
  const long long cbase = (long long)b * a.Sc;
  const T sig = a.sig[b];
  const T cths = a.s_h2 * a.cth[b];
  const T* nx = a.tab;
  const T* fx = a.tab + Pf;
  const T* ny = a.tab + 2 * Pf;
  const T* fy = a.tab + 3 * Pf;
  // x-interpolated coarse row Yc at this lane's column (0 outside the coarse interior)
  const int cxa = (x & 1) ? (x - 1) >> 1 : (x >> 1) - 1;  // first coarse column used
  auto crow = [&](int Yc) -> T {
    if (Yc < 0 || Yc >= nc || !xin) return (T)0;
    const T* er = ec + cbase + (long long)Yc * Pc;
    if (x & 1) return er[cxa];
    const T e0 = cxa >= 0 ? er[cxa] : (T)0;
    const T e1 = cxa + 1 < nc ? er[cxa + 1] : (T)0;
    return (T)0.5 * (e0 + e1);
  };
  // x2 = w D^-1 b + P e at row y, with b, faces and the Jacobi factor for the smoothing step
  T ex_lo = (T)0;  // crow(k - 1) for the current even row 2k (cached from the odd row before)
  int k_lo = -1000;
  FaceSweep<T, VAR> fs;
  fs.init(a, nx, fy, cths, x, y0 - 1);
  // global operands are loaded ahead of use (the kernel is latency-bound otherwise): b two rows
  // ahead, the accumulation target one row ahead
  auto ld_b = [&](int y) -> T { return (xin && y >= 0 && y < nf) ? bf[base + (long long)y * Pf + x] : (T)0; };
  const bool wlane = lane >= 1 && lane <= 30 && x < Pf;
  auto ld_o = [&](int y) -> double {
    if (mode != 1 || !wlane || !xin || y >= nf) return 0.0;
    const long long gi = base + (long long)y * Pf + x;
    return out_fp64 ? ((const double*)out)[gi] : (double)((const T*)out)[gi];
  };
  auto row = [&](int y, T bload, T& bv, T& x2, T& jf, T& dg, Faces<T, VAR>& f) {
    f = fs.row(a, fx, ny, fy, cths, x, y);
    bv = (T)0;
    x2 = (T)0;
    jf = (T)0;
    dg = (T)0;
    // prolongation of the coarse correction (rows: odd y -> (y-1)/2, even y -> y/2 - 1 and y/2)
    T pe;
    if (y & 1) {
      const int k = (y - 1) >> 1;
      ex_lo = (k_lo == k) ? ex_lo : crow(k);
      k_lo = k;
      pe = ex_lo;
    } else {
      const int k = y >> 1;
      const T lo = (k_lo == k - 1) ? ex_lo : crow(k - 1);
      const T hi = crow(k);
      pe = (T)0.5 * (lo + hi);
      ex_lo = hi;
      k_lo = k;
    }
    if (xin && y >= 0 && y < nf) {
      const long long gi = base + (long long)y * Pf + x;
      bv = bload;
      if (DM == 1) {
        const T2c jd = *(const T2c*)(a.jinv + 2 * gi);  // (w / D, D)
        jf = jd.x;
        dg = jd.y;
      } else {
        jf = jacobi_at<T, VAR, DM>(a, b, gi, f, sig);
      }
      x2 = fma(bv, jf, pe);
    }
  };
  T bm, xm, jm, bcv, xc, jc, bn, xn, jn, dm_, dc_, dn_;
  Faces<T, VAR> fm, fc, fn;
  row(y0 - 1, ld_b(y0 - 1), bm, xm, jm, dm_, fm);
  row(y0, ld_b(y0), bcv, xc, jc, dc_, fc);
  T b_next = ld_b(y0 + 1);
  double o_next = ld_o(y0);
  for (int y = y0; y < y0 + kStripUpRows && y < Pf; ++y) {
    const T b_after = ld_b(y + 2);
    const double o_cur = o_next;
    o_next = ld_o(y + 1);
    row(y + 1, b_next, bn, xn, jn, dn_, fn);
    b_next = b_after;
    const T xW = __shfl_up_sync(0xffffffffu, xc, 1);
    const T xE = __shfl_down_sync(0xffffffffu, xc, 1);
    if (wlane) {
      const long long gi = base + (long long)y * Pf + x;
      if (xin && y < nf) {
        T Lx;
        if (DM == 1)
          Lx = dc_ * xc - (fc.xl * xW + fc.xr * xE + fc.yl * xm + fc.yu * xn);
        else if (VAR)
          Lx = sig * xc + fc.xl * (xc - xW) + fc.xr * (xc - xE) + fc.yl * (xc - xm) + fc.yu * (xc - xn);
        else
          Lx = (sig + (T)4 * a.a0s) * xc - a.a0s * ((xW + xE) + (xm + xn));
        const T v = xc + jc * (bcv - Lx);
        if (mode == 1) {
          if (out_fp64)
            ((double*)out)[gi] = o_cur + (double)v;
          else
            ((T*)out)[gi] = (T)o_cur + v;
        } else {
          store_out<T>(out, gi, 0, out_fp64, v);
        }
      } else if (mode == 0) {
        store_out<T>(out, gi, 0, out_fp64, (T)0);
      }
    }
    bm = bcv;
    xm = xc;
    jm = jc;
    dm_ = dc_;
    fm = fc;
    bcv = bn;
    xc = xn;
    jc = jn;
    dc_ = dn_;
    fc = fn;
  }
  (void)bm;
  (void)jm;
  (void)dm_;
  (void)fm;
}

// ---- FP32 forms of the two strip kernels (the V-cycles of the mixed-precision path) ----
// Same sweep, geometry and arithmetic order as k_mg2s_down / k_mg2s_up with a variable
// coefficient and the Jacobi factor formed per point, with the per-row work cut down: the lane's
// x-tables and interpolation weights are loaded once, indices are 32-bit offsets within the
// slice, the output mode is a template parameter, and the Jacobi factor w / D uses the fast
// reciprocal (the same factor in the down and the up kernel of a level, so the V-cycle stays
// symmetric).

// per-lane constants of a fine column x: x-face table values, the y-face factor and the
// coarse columns and weights of the linear interpolation along x
struct LaneCols {
  float fxl, fxr, gxn;  // g_x at the lower / upper x-face, (s/h^2) c g_t(t) g_x(x) for the y-faces
  int c0, c1;           // coarse columns of the interpolation (clamped in range)
  float w0, w1;         // their weights (0 outside the coarse interior)
};

__device__ __forceinline__ LaneCols lane_cols(const Mg2Args<float>& a, int x, float cths) {
  const int Pf = 1 << a.logPf;
  LaneCols c;
  const bool xin = x >= 0 && x < a.nf;
  c.fxl = xin ? a.tab[Pf + x] : 0.f;
  c.fxr = xin ? a.tab[Pf + x + 1] : 0.f;
  c.gxn = xin ? cths * a.tab[x] : 0.f;
  int c0, c1;
  float w0, w1;
  if (x & 1) {  // fine 2X + 1 sits on coarse X
    c0 = (x - 1) >> 1;
    c1 = c0;
    w0 = 1.f;
    w1 = 0.f;
  } else {      // fine 2X sits between coarse X - 1 and X
    c0 = (x >> 1) - 1;
    c1 = x >> 1;
    w0 = 0.5f;
    w1 = 0.5f;
  }
  if (!xin) w0 = w1 = 0.f;
  if (c0 < 0 || c0 >= a.nc) {
    w0 = 0.f;
    c0 = 0;
  }
  if (c1 < 0 || c1 >= a.nc) {
    w1 = 0.f;
    c1 = 0;
  }
  c.c0 = c0;
  c.c1 = c1;
  c.w0 = w0;
  c.w1 = w1;
  return c;
}

template <int MODE>
__global__ void __launch_bounds__(256, 5) k_mg2s_up_f32(const float* __restrict__ bf, const float* __restrict__ ec,
                                                     float* __restrict__ out, Mg2Args<float> a, int wpr, int strips,
                                                     long long nwarps, const int* done) {
  if (stop_requested(done)) return;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wg >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int wx = (int)(wg % wpr);
  const long long rest = wg / wpr;
  const int strip = (int)(rest % strips);
  const int b = (int)(rest / strips);
  const int x = kStripUpCols * wx - 1 + lane;  // fine column; lanes 1..30 write
  const int y0 = kStripUpRows * strip;
  const int nf = a.nf, nc = a.nc, Pf = 1 << a.logPf, Pc = 1 << a.logPc;
  const bool xin = x >= 0 && x < nf;
  const float* __restrict__ bs = bf + (long long)b * a.Sf;
  float* __restrict__ os = out + (long long)b * a.Sf;
  const float* __restrict__ es = ec + (long long)b * a.Sc;
  const float sig = a.sig[b];
  const float cths = a.s_h2 * a.cth[b];
  const float a0s = a.a0s, omega = a.omega;
  const float* ny = a.tab + 2 * Pf;
  const float* fy = a.tab + 3 * Pf;
  const LaneCols lc = lane_cols(a, x, cths);
  // x-interpolated coarse row Yc at this lane's column
  auto crow = [&](int Yc) -> float {
    if (Yc < 0 || Yc >= nc) return 0.f;
    const float* er = es + Yc * Pc;
    return fmaf(lc.w0, er[lc.c0], lc.w1 * er[lc.c1]);
  };
  auto ld_b = [&](int y) -> float { return (xin && y >= 0 && y < nf) ? bs[y * Pf + x] : 0.f; };
  const bool wlane = lane >= 1 && lane <= 30 && x < Pf;
  auto ld_o = [&](int y) -> float { return (MODE == 1 && wlane && xin && y < nf) ? os[y * Pf + x] : 0.f; };
  float fy_carry = (y0 - 1 >= 0 && y0 - 1 <= nf) ? fy[y0 - 1] : 0.f;  // y-face table below the first row
  // Rows go in pairs (y0 is even): fine row 2k+1 sits on coarse row k, fine row 2k+2 between k and
  // k+1, so the interpolation in y needs one new coarse row every two fine rows.  cprev = the
  // x-interpolated coarse row below the next odd fine row.
  float cprev = crow((y0 >> 1) - 1);
  // one fine row: faces, Jacobi factor, and x2 = w D^-1 b + P e (pe: the interpolated correction)
  auto row = [&](int y, float bv_in, float pe, float& bv, float& x2, float& jf, float& xl, float& xr, float& yl,
                 float& yu) {
    const bool yin = y >= 0 && y < nf;
    const float gy = yin ? cths * ny[y] : 0.f;
    const float fyu = (y + 1 >= 0 && y + 1 <= nf) ? fy[y + 1] : 0.f;
    xl = fmaf(gy, lc.fxl, a0s);
    xr = fmaf(gy, lc.fxr, a0s);
    yl = fmaf(lc.gxn, fy_carry, a0s);
    yu = fmaf(lc.gxn, fyu, a0s);
    fy_carry = fyu;
    const bool in = xin && yin;
    bv = in ? bv_in : 0.f;
    jf = __fdividef(omega, sig + ((xl + xr) + (yl + yu)));
    x2 = in ? fmaf(bv, jf, pe) : 0.f;
  };
  auto pe_odd = [&]() { return cprev; };
  auto pe_even = [&](int y) {
    const float cnext = crow(y >> 1);
    const float pe = 0.5f * (cprev + cnext);
    cprev = cnext;
    return pe;
  };
  float bm, xm, jm, xlm, xrm, ylm, yum;
  float bc, xc, jc, xlc, xrc, ylc, yuc;
  float bn, xn, jn, xln, xrn, yln, yun;
  row(y0 - 1, ld_b(y0 - 1), pe_odd(), bm, xm, jm, xlm, xrm, ylm, yum);
  row(y0, ld_b(y0), pe_even(y0), bc, xc, jc, xlc, xrc, ylc, yuc);
  float b_next = ld_b(y0 + 1);
  float o_next = ld_o(y0);
  // output of row y from the rows y-1 (m), y (c), y+1 (n); then the window moves down one row
  auto emit = [&](int y, float o_cur) {
    const float xW = __shfl_up_sync(0xffffffffu, xc, 1);
    const float xE = __shfl_down_sync(0xffffffffu, xc, 1);
    if (wlane) {
      const int gi = y * Pf + x;
      if (xin && y < nf) {
        const float Lx = sig * xc + xlc * (xc - xW) + xrc * (xc - xE) + ylc * (xc - xm) + yuc * (xc - xn);
        const float v = xc + jc * (bc - Lx);
        os[gi] = MODE == 1 ? o_cur + v : v;
      } else if (MODE == 0) {
        os[gi] = 0.f;
      }
    }
    xm = xc;
    bc = bn;
    xc = xn;
    jc = jn;
    xlc = xln;
    xrc = xrn;
    ylc = yln;
    yuc = yun;
  };
  const int yend = min(y0 + kStripUpRows, Pf);
  for (int y = y0; y < yend; y += 2) {
    {  // row y (even): its lower neighbour row y+1 is odd
      const float b_after = ld_b(y + 2);
      const float o_cur = o_next;
      o_next = ld_o(y + 1);
      row(y + 1, b_next, pe_odd(), bn, xn, jn, xln, xrn, yln, yun);
      b_next = b_after;
      emit(y, o_cur);
    }
    if (y + 1 < yend) {  // row y+1 (odd): its lower neighbour row y+2 is even
      const float b_after = ld_b(y + 3);
      const float o_cur = o_next;
      o_next = ld_o(y + 2);
      row(y + 2, b_next, pe_even(y + 2), bn, xn, jn, xln, xrn, yln, yun);
      b_next = b_after;
      emit(y + 1, o_cur);
    }
  }
  (void)bm;
  (void)jm;
  (void)xlm;
  (void)xrm;
  (void)ylm;
  (void)yum;
}

__global__ void __launch_bounds__(256) k_mg2s_down_f32(const float* __restrict__ bf, float* __restrict__ bcg,
                                                       Mg2Args<float> a, int wpr, int strips, long long nwarps,
                                                       const int* done) {
  if (stop_requested(done)) return;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wg >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int wx = (int)(wg % wpr);
  const long long rest = wg / wpr;
  const int strip = (int)(rest % strips);
  const int b = (int)(rest / strips);
  const int X0 = kStripDownCols * wx, Y0 = kStripDownRows * strip;
  const int x = 2 * X0 - 1 + lane;  // fine column of this lane
  const int nf = a.nf, Pf = 1 << a.logPf, Pc = 1 << a.logPc;
  const bool xin = x >= 0 && x < nf;
  const float* __restrict__ bs = bf + (long long)b * a.Sf;
  float* __restrict__ cs = bcg + (long long)b * a.Sc;
  const float sig = a.sig[b];
  const float cths = a.s_h2 * a.cth[b];
  const float a0s = a.a0s, omega = a.omega;
  const float* ny = a.tab + 2 * Pf;
  const float* fy = a.tab + 3 * Pf;
  const LaneCols lc = lane_cols(a, x, cths);
  const int yfirst = 2 * Y0 - 1, ylast = 2 * (Y0 + kStripDownRows);
  float fy_carry = (yfirst >= 0 && yfirst <= nf) ? fy[yfirst] : 0.f;
  auto ld_b = [&](int y) -> float { return (xin && y >= 0 && y < nf) ? bs[y * Pf + x] : 0.f; };
  // x1 = w D^-1 b and the faces of row y
  auto row = [&](int y, float bv_in, float& bv, float& x1, float& xl, float& xr, float& yl, float& yu) {
    const bool yin = y >= 0 && y < nf;
    const float gy = yin ? cths * ny[y] : 0.f;
    const float fyu = (y + 1 >= 0 && y + 1 <= nf) ? fy[y + 1] : 0.f;
    xl = fmaf(gy, lc.fxl, a0s);
    xr = fmaf(gy, lc.fxr, a0s);
    yl = fmaf(lc.gxn, fy_carry, a0s);
    yu = fmaf(lc.gxn, fyu, a0s);
    fy_carry = fyu;
    const bool in = xin && yin;
    bv = in ? bv_in : 0.f;
    x1 = in ? bv * __fdividef(omega, sig + ((xl + xr) + (yl + yu))) : 0.f;
  };
  float bm, xm, xlm, xrm, ylm, yum;
  float bc, xc, xlc, xrc, ylc, yuc;
  float bn, xn, xln, xrn, yln, yun;
  row(yfirst, ld_b(yfirst), bm, xm, xlm, xrm, ylm, yum);
  row(yfirst + 1, ld_b(yfirst + 1), bc, xc, xlc, xrc, ylc, yuc);
  float b_next = ld_b(yfirst + 2);
  float h1 = 0.f, h2 = 0.f;  // horizontal restrictions of the two previous rows
  const bool out_lane = (lane & 1) == 0 && lane >= 2 && lane <= 28;
  const int X = X0 + (lane >> 1) - 1;  // coarse column of an output lane (x = 2X + 1)
  for (int y = yfirst + 1; y <= ylast; ++y) {
    const float b_after = ld_b(y + 2);
    row(y + 1, b_next, bn, xn, xln, xrn, yln, yun);
    b_next = b_after;
    const float xW = __shfl_up_sync(0xffffffffu, xc, 1);
    const float xE = __shfl_down_sync(0xffffffffu, xc, 1);
    float r = 0.f;
    if (xin && y >= 0 && y < nf) {
      const float Lx = sig * xc + xlc * (xc - xW) + xrc * (xc - xE) + ylc * (xc - xm) + yuc * (xc - xn);
      r = bc - Lx;
    }
    const float rW = __shfl_up_sync(0xffffffffu, r, 1);
    const float rE = __shfl_down_sync(0xffffffffu, r, 1);
    const float h = 0.25f * (rW + rE) + 0.5f * r;
    if (y >= 2 * Y0 + 2 && ((y - 2 * Y0) & 1) == 0) {
      const int Y = (y >> 1) - 1;
      if (out_lane && X < a.nc && Y < a.nc) cs[Y * Pc + X] = 0.25f * (h2 + h) + 0.5f * h1;
    }
    h2 = h1;
    h1 = h;
    xm = xc;
    bc = bn;
    xc = xn;
    xlc = xln;
    xrc = xrn;
    ylc = yln;
    yuc = yun;
  }
  (void)bm;
  (void)xlm;
  (void)xrm;
  (void)ylm;
  (void)yum;
}

// (w D^-1, D) for every interior point of one level (FP64 variable-coefficient cache)
template <typename T>
__global__ void k_make_jinv(T* __restrict__ jinv, StencilGeom<T> g, OpBatch<T> op, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    T v = (T)0, d = (T)0;
    if (decode<2>(i, g.logP, g.n, t, x, y, z)) {
      T am[3], ap[3];
      face_coefs<2, T>(g.tab, g.P, x, y, z, op.cth[t], g.a0, am, ap);
      d = op.sig[t] + op.s * g.h2inv * face_sum<2, T>(am, ap);
      v = op.omega / d;
    }
    jinv[2 * i] = v;
    jinv[2 * i + 1] = d;
  }
}

}  // namespace

template <typename T>
void vcycle2d(const MGPlan<T>& plan, OpBatch<T> op, const T* b0, void* out, int mode, int out_fp64,
              bool var, const T* const* dinv_slice, const T* const* jinv, const int* done,
              cudaStream_t st) {
  const int B = plan.B;
  auto args = [&](int l) {
    Mg2Args<T> a;
    const Level& F = plan.lev[l];
    const Level& C = plan.lev[l + 1];
    a.nf = F.n;
    a.logPf = F.logP;
    a.Sf = F.S;
    a.nc = C.n;
    a.logPc = C.logP;
    a.Sc = C.S;
    a.tab = plan.tab + F.tab;
    const double h2inv = 1.0 / (F.h * F.h);
    a.a0s = (T)((double)op.s * (double)plan.a0 * h2inv);
    a.s_h2 = (T)((double)op.s * h2inv);
    a.sig = op.sig;
    a.cth = op.cth;
    a.dinv = dinv_slice ? dinv_slice[l] : nullptr;
    a.jinv = jinv ? jinv[l] : nullptr;
    a.omega = op.omega;
    return a;
  };
  const int dm = var ? (jinv ? 1 : 2) : 0;
  const T* bl = b0;
  for (int l = 0; l < plan.lc; ++l) {
    const Mg2Args<T> a = args(l);
    const dim3 grid((a.nc + kDownTX - 1) / kDownTX, (a.nc + kDownTY - 1) / kDownTY, B);
    const double df = (double)B * a.nf * a.nf, dc = (double)B * a.nc * a.nc;
    LaunchScope ls("mg2_down", st, sizeof(T) * (df + dc) + (dm == 1 ? sizeof(T) * df : 0.0));
    T* bc = (T*)plan.buf[l + 1].b;
    // (FP64: the tile kernel spends fewer FP64 instructions per point on this level)
    if (sizeof(T) == 4 && (1 << a.logPf) >= kStripMinP) {
      const int wpr = (a.nc + kStripDownCols - 1) / kStripDownCols;
      const int strips = (a.nc + kStripDownRows - 1) / kStripDownRows;
      const long long nw = (long long)wpr * strips * B;
      const unsigned blocks = (unsigned)((nw + 7) / 8);
      if constexpr (std::is_same<T, float>::value) {
        if (dm == 2) {
          k_mg2s_down_f32<<<blocks, 256, 0, st>>>(bl, bc, a, wpr, strips, nw, done);
          bl = bc;
          continue;
        }
      }
      if (dm == 0)
        k_mg2s_down<T, false, 0><<<blocks, 256, 0, st>>>(bl, bc, a, wpr, strips, nw, done);
      else if (dm == 1)
        k_mg2s_down<T, true, 1><<<blocks, 256, 0, st>>>(bl, bc, a, wpr, strips, nw, done);
      else
        k_mg2s_down<T, true, 2><<<blocks, 256, 0, st>>>(bl, bc, a, wpr, strips, nw, done);
    } else if (dm == 0)
      k_mg2_down<T, false, 0><<<grid, 256, 0, st>>>(bl, bc, a, done);
    else if (dm == 1)
      k_mg2_down<T, true, 1><<<grid, 256, 0, st>>>(bl, bc, a, done);
    else
      k_mg2_down<T, true, 2><<<grid, 256, 0, st>>>(bl, bc, a, done);
    bl = bc;
  }
  vcycle_coarse<T>(plan, op, bl, out, mode, out_fp64, done, st);
  for (int l = plan.lc - 1; l >= 0; --l) {
    const Mg2Args<T> a = args(l);
    const int Pf = 1 << a.logPf;
    const dim3 grid((Pf + kUpTX - 1) / kUpTX, (Pf + kUpTY - 1) / kUpTY, B);
    const T* bf = l == 0 ? b0 : (const T*)plan.buf[l].b;
    void* o = l == 0 ? out : plan.buf[l].x;
    const int om = l == 0 ? mode : 0;
    const int of = l == 0 ? out_fp64 : 0;
    const double df = (double)B * a.nf * a.nf, dc = (double)B * a.nc * a.nc;
    const double ob = of ? (om == 1 ? 16.0 : 8.0) : (om == 1 ? 2.0 * sizeof(T) : (double)sizeof(T));
    LaunchScope ls("mg2_up", st, sizeof(T) * (df + dc) + ob * df + (dm == 1 ? sizeof(T) * df : 0.0));
    const T* e = (const T*)plan.buf[l + 1].x;
    if (Pf >= kStripMinP) {
      const int wpr = (Pf + kStripUpCols - 1) / kStripUpCols;
      const int strips = (Pf + kStripUpRows - 1) / kStripUpRows;
      const long long nw = (long long)wpr * strips * B;
      const unsigned blocks = (unsigned)((nw + 7) / 8);
      if constexpr (std::is_same<T, float>::value) {
        if (dm == 2 && !of) {
          if (om == 1)
            k_mg2s_up_f32<1><<<blocks, 256, 0, st>>>(bf, e, (float*)o, a, wpr, strips, nw, done);
          else
            k_mg2s_up_f32<0><<<blocks, 256, 0, st>>>(bf, e, (float*)o, a, wpr, strips, nw, done);
          continue;
        }
      }
      if (dm == 0)
        k_mg2s_up<T, false, 0><<<blocks, 256, 0, st>>>(bf, e, o, om, of, a, wpr, strips, nw, done);
      else if (dm == 1)
        k_mg2s_up<T, true, 1><<<blocks, 256, 0, st>>>(bf, e, o, om, of, a, wpr, strips, nw, done);
      else
        k_mg2s_up<T, true, 2><<<blocks, 256, 0, st>>>(bf, e, o, om, of, a, wpr, strips, nw, done);
    } else if (dm == 0)
      k_mg2_up<T, false, 0><<<grid, 256, 0, st>>>(bf, e, o, om, of, a, done);
    else if (dm == 1)
      k_mg2_up<T, true, 1><<<grid, 256, 0, st>>>(bf, e, o, om, of, a, done);
    else
      k_mg2_up<T, true, 2><<<grid, 256, 0, st>>>(bf, e, o, om, of, a, done);
  }
}

template <typename T>
void launch_make_jinv(T* jinv, StencilGeom<T> g, OpBatch<T> op, int B, cudaStream_t st) {
  const long long total = g.S * B;
  LaunchScope ls("make_jinv", st, sizeof(T) * (double)total);
  k_make_jinv<T><<<grid_for(total), kThreads, 0, st>>>(jinv, g, op, total);
}

template void vcycle2d<float>(const MGPlan<float>&, OpBatch<float>, const float*, void*, int, int, bool,
                              const float* const*, const float* const*, const int*, cudaStream_t);
template void vcycle2d<double>(const MGPlan<double>&, OpBatch<double>, const double*, void*, int, int, bool,
                               const double* const*, const double* const*, const int*, cudaStream_t);
template void launch_make_jinv<float>(float*, StencilGeom<float>, OpBatch<float>, int, cudaStream_t);
template void launch_make_jinv<double>(double*, StencilGeom<double>, OpBatch<double>, int, cudaStream_t);

}  // namespace pt
