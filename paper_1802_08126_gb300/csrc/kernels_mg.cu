// Batched geometric multigrid for the spatial solves of the Uzawa preconditioners
// (A~_n^-1 of §3, eq. 3.2-3.3 and H~_k^-1 of §4, eq. 4.6-4.7).
//
// The paper only asks for "MG V-cycles with Jacobi smoothers" (§8.2).  Reading used here:
// symmetric V(1,1) with zero initial guess, weighted Jacobi before and after the coarse-grid
// correction, full-weighting restriction R = P^T / 2^d, d-linear prolongation P, level
// operators rediscretised from the same coefficient at the level's face midpoints, exact
// solve on the one-point grid.  Every launch covers all B slices of the batch (all time
// steps, or all DST frequencies) at once.  Levels whose slices have at most kCoarseMaxElems
// padded points are finished by one CTA per slice in shared memory.
//
// Also here: the exact batched tridiagonal solve used for 1-D problems.
#include <algorithm>
#include <cmath>

#include "bulk_pipe.cuh"
#include "stencil_common.cuh"

namespace pt {

namespace {

template <int DIM, typename T>
__device__ __forceinline__ T diag_at(StencilGeom<T> g, T sig, T s, T cth, int x, int y, int z,
                                     T* am, T* ap, int mass) {
  face_coefs<DIM, T>(g.tab, g.P, x, y, z, cth, g.a0, am, ap);
  return sig * mass_diag<DIM, T>(mass) + s * g.h2inv * face_sum<DIM, T>(am, ap);
}

// x = w D^-1 b   (pre-smoothing from a zero iterate)
template <int DIM, typename T>
__global__ void k_jacobi0(const T* __restrict__ b, T* __restrict__ x, StencilGeom<T> g,
                          OpBatch<T> op, long long total, const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int xx, y, z;
    T v = (T)0;
    if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
      T am[3], ap[3];
      const T D = diag_at<DIM, T>(g, op.sig[t], op.s, op.cth[t], xx, y, z, am, ap, op.mass);
      v = op.omega * b[i] / D;
    }
    x[i] = v;
  }
}

// r = b - L x
template <int DIM, typename T>
__global__ void k_residual(const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r,
                           StencilGeom<T> g, OpBatch<T> op, long long total, const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int xx, y, z;
    T v = (T)0;
    if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
      T am[3], ap[3];
      face_coefs<DIM, T>(g.tab, g.P, xx, y, z, op.cth[t], g.a0, am, ap);
      const T xc = x[i];
      v = b[i] - (op.sig[t] * mass_apply<DIM, T>(op.mass, x, i, xc, g.P) +
                  op.s * g.h2inv * stencil_sum<DIM, T>(x, i, xc, am, ap, g.P));
    }
    r[i] = v;
  }
}

// Post-smoothing in one pass: out (mode) x + w D^-1 (b - L x), the residual never stored.  out
// must not alias x.
template <int DIM, typename T>
__global__ void k_post_smooth(const T* __restrict__ b, const T* __restrict__ x, void* out, int mode,
                              int out_fp64, StencilGeom<T> g, OpBatch<T> op, long long total, const int* done) {
  if (stop_requested(done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int xx, y, z;
    if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
      T am[3], ap[3];
      const T D = diag_at<DIM, T>(g, op.sig[t], op.s, op.cth[t], xx, y, z, am, ap, op.mass);
      const T xc = x[i];
      const T Lx = op.sig[t] * mass_apply<DIM, T>(op.mass, x, i, xc, g.P) +
                   op.s * g.h2inv * stencil_sum<DIM, T>(x, i, xc, am, ap, g.P);
      store_out<T>(out, i, mode, out_fp64, xc + op.omega * (b[i] - Lx) / D);
    } else if (mode == 0) {
      store_out<T>(out, i, 0, out_fp64, (T)0);
    }
  }
}

// offset (within a slice) of the fine point 2I+1 that coincides with coarse point I
template <int DIM>
__device__ __forceinline__ long long fine_center(int x, int y, int z, int Pf) {
  if (DIM == 1) return 2 * x + 1;
  if (DIM == 2) return (long long)(2 * y + 1) * Pf + (2 * x + 1);
  return ((long long)(2 * z + 1) * Pf + (2 * y + 1)) * Pf + (2 * x + 1);
}

// full weighting: bc[I] = sum_{o in {-1,0,1}^d} prod_d w(o_d) r[2I+1+o],  w(0)=1/2, w(+-1)=1/4
template <int DIM, typename T>
__global__ void k_restrict(const T* __restrict__ r, T* __restrict__ bc, int nf_logP, long long Sf,
                           int nc, int nc_logP, long long total_c, const int* done) {
  if (stop_requested(done)) return;
  const int Pf = 1 << nf_logP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total_c;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int x, y, z;
    T v = (T)0;
    if (decode<DIM>(i, nc_logP, nc, t, x, y, z)) {
      const long long fc = t * Sf + fine_center<DIM>(x, y, z, Pf);
      if (DIM == 1) {
        v = (T)0.25 * r[fc - 1] + (T)0.5 * r[fc] + (T)0.25 * r[fc + 1];
      } else if (DIM == 2) {
        T rows[3];
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy) {
          const long long c = fc + (long long)oy * Pf;
          rows[oy + 1] = (T)0.25 * r[c - 1] + (T)0.5 * r[c] + (T)0.25 * r[c + 1];
        }
        v = (T)0.25 * rows[0] + (T)0.5 * rows[1] + (T)0.25 * rows[2];
      } else {
        const long long Pf2 = (long long)Pf * Pf;
        T planes[3];
#pragma unroll
        for (int oz = -1; oz <= 1; ++oz) {
          T rows[3];
#pragma unroll
          for (int oy = -1; oy <= 1; ++oy) {
            const long long c = fc + (long long)oz * Pf2 + (long long)oy * Pf;
            rows[oy + 1] = (T)0.25 * r[c - 1] + (T)0.5 * r[c] + (T)0.25 * r[c + 1];
          }
          planes[oz + 1] = (T)0.25 * rows[0] + (T)0.5 * rows[1] + (T)0.25 * rows[2];
        }
        v = (T)0.25 * planes[0] + (T)0.5 * planes[1] + (T)0.25 * planes[2];
      }
    }
    bc[i] = v;
  }
}

// d-linear interpolation weights along one axis for fine index f: coarse c0,c1 with w0,w1
__device__ __forceinline__ void interp_axis(int f, int& c0, int& c1, bool& two) {
  if (f & 1) {
    c0 = f >> 1;
    c1 = c0;
    two = false;
  } else {
    c0 = (f >> 1) - 1;
    c1 = f >> 1;
    two = true;
  }
}

template <int DIM, typename T>
__device__ __forceinline__ T prolong_at(const T* __restrict__ ec, long long slot_off, int Pc, int x,
                                        int y, int z) {
  int x0, x1, y0 = 0, y1 = 0, z0 = 0, z1 = 0;
  bool tx, ty = false, tz = false;
  interp_axis(x, x0, x1, tx);
  if (DIM >= 2) interp_axis(y, y0, y1, ty);
  if (DIM >= 3) interp_axis(z, z0, z1, tz);
  auto row = [&](int zz, int yy) -> T {
    const long long base = slot_off + ((long long)zz * Pc + yy) * Pc;
    return tx ? (T)0.5 * (ec[base + x0] + ec[base + x1]) : ec[base + x0];
  };
  auto plane = [&](int zz) -> T {
    if (DIM == 1) return row(0, 0);
    return ty ? (T)0.5 * (row(zz, y0) + row(zz, y1)) : row(zz, y0);
  };
  if (DIM <= 2) return plane(0);
  return tz ? (T)0.5 * (plane(z0) + plane(z1)) : plane(z0);
}

// x += P ec
template <int DIM, typename T>
__global__ void k_prolong_add(T* __restrict__ x, const T* __restrict__ ec, StencilGeom<T> g,
                              int Pc_logP, long long Sc, long long total, const int* done) {
  if (stop_requested(done)) return;
  const int Pc = 1 << Pc_logP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long t;
    int xx, y, z;
    if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) x[i] += prolong_at<DIM, T>(ec, t * Sc, Pc, xx, y, z);
  }
}

// ---- 3-D FP32 levels of 32 <= P <= 128: residual and post-smoothing streamed by rows ----
// A CTA owns a band of YB = 256 / P rows (all P columns) of one slice and walks a strip of R
// z-planes, one thread per (x, y); a producer warp bulk-copies, plane after plane, the band's x
// rows y0 - 1 .. y0 + YB (contiguous, with a 16-byte halo each side) and its b row into a ring of
// stages (stage j: x of plane z0 - 1 + j, b of plane z0 - 2 + j).  x- and y-neighbours come from
// the stage, z-neighbours from registers.  The arithmetic is that of k_residual / k_post_smooth
// (faces, diagonal and stencil formed in the same order, the exact division), so the V-cycle keeps
// the first Jacobi step's factor.  KIND 1: r = b - L x; 2: out (mode) x + w (b - L x) / D.
constexpr int kLvBand = 256, kLvStages = 8, kLvHalo = 4;

template <int LOGP>
struct LvStage {
  static constexpr int P = 1 << LOGP, YB = kLvBand / P, XR = (YB + 2) * P + 2 * kLvHalo;
  float x[XR];
  float b[kLvBand];
};

__device__ __forceinline__ void lv_timeout(int* fault) {
  if (fault) *(volatile int*)fault = 1;
}

template <int LOGP, int KIND>
__global__ void __launch_bounds__(kLvBand + 32, 4) k_level3_rows(const float* __restrict__ b,
                                                                 const float* __restrict__ x, void* out, int mode,
                                                                 int out_fp64, StencilGeom<float> g,
                                                                 OpBatch<float> op, int B, int logR, int* fault,
                                                                 const int* done) {
  using Stage = LvStage<LOGP>;
  constexpr int P = Stage::P, YB = Stage::YB, XR = Stage::XR;
  static_assert(sizeof(Stage) % 16 == 0, "bulk copies need 16-byte aligned stage buffers");
  if (stop_requested(done)) return;
  __shared__ __align__(128) Stage stage[kLvStages];
  __shared__ __align__(8) RowRing<kLvStages> ring;
  const int R = 1 << logR;
  constexpr int bands = P / YB;
  const int strips = P >> logR;
  const long long ntasks = (long long)B * bands * strips;
  const long long P2 = (long long)P * P;
  const int n = g.n;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) ring.init(kLvBand / 32);
  __syncthreads();
  if (tid >= kLvBand) {
    if (lane == 0) {
      bool ok = true;
      unsigned c = 0;
      for (long long task = blockIdx.x; task < ntasks && ok; task += gridDim.x) {
        const int y0 = (int)(task % bands) * YB;
        const long long rest = task / bands;
        const int z0 = (int)(rest % strips) << logR;
        const int t = (int)(rest / strips);
        const long long slot = (long long)t * g.S;
        for (int j = 0; j < R + 2; ++j, ++c) {
          if (!ring.acquire(c)) {
            ok = false;
            break;
          }
          const int z = z0 - 1 + j, zr = z - 1;
          const bool cp_x = z <= P - 1;
          const unsigned xbytes = (unsigned)(y0 + YB < P ? XR : XR - P) * 4u;
          const bool cp_b = j >= 2 && zr < n;
          const unsigned bytes = (cp_x ? xbytes : 0u) + (cp_b ? (unsigned)kLvBand * 4u : 0u);
          uint64_t* bar = ring.commit(c, bytes);
          Stage& s = stage[c % kLvStages];
          if (cp_x) bulk_g2s(s.x, x + slot + ((long long)z * P + y0 - 1) * P - kLvHalo, xbytes, bar);
          if (cp_b) bulk_g2s(s.b, b + slot + ((long long)zr * P + y0) * P, kLvBand * 4u, bar);
        }
      }
      if (!ok) ring.give_up();
      if (!ring.drain(c)) ok = false;
      if (!ok) lv_timeout(fault);
    }
    return;
  }
  const float* nx = g.tab;
  const float* fx = g.tab + P;
  const float* ny = g.tab + 2 * P;
  const float* fy = g.tab + 3 * P;
  const float* nz = g.tab + 4 * P;
  const float* fz = g.tab + 5 * P;
  const float a0 = g.a0, sh = op.s * g.h2inv;
  const int xx = tid & (P - 1), yl = tid >> LOGP;
  const int sc = kLvHalo + (yl + 1) * P + xx;
  bool ok = true;
  unsigned c = 0;
  for (long long task = blockIdx.x; task < ntasks && ok; task += gridDim.x) {
    const int y0 = (int)(task % bands) * YB;
    const long long rest = task / bands;
    const int z0 = (int)(rest % strips) << logR;
    const int t = (int)(rest / strips);
    const int y = y0 + yl;
    const bool xyin = xx < n && y < n;
    const float cth = op.cth[t], sig = op.sig[t];
    const float cx = cth * nx[xx], cy = ny[y];
    const float fxl = fx[xx], fxr = fx[xx + 1 < P ? xx + 1 : xx];
    const float fyl = fy[y], fyu = fy[y + 1 < P ? y + 1 : y];
    const long long o0 = (long long)t * g.S + (long long)y * P + xx;
    float x_m = 0.f, x_c = 0.f, xW = 0.f, xE = 0.f, xS = 0.f, xN = 0.f;
    for (int j = 0; j < R + 2; ++j, ++c) {
      if (!ring.wait(c)) {
        ok = false;
        break;
      }
      const Stage& s = stage[c % kLvStages];
      const float x_p = s.x[sc], x_pW = s.x[sc - 1], x_pE = s.x[sc + 1], x_pS = s.x[sc - P], x_pN = s.x[sc + P];
      const float bi = s.b[tid];
      ring.release(c);
      if (j >= 2) {
        const int z = z0 + j - 2;
        const bool in = xyin && z < n;
        const long long o = o0 + z * P2;
        if (in) {
          const float cz = nz[z];
          const float gyz = cth * cy * cz;
          const float am0 = fmaf(gyz, fxl, a0), ap0 = fmaf(gyz, fxr, a0);
          const float gxz = cx * cz;
          const float am1 = fmaf(gxz, fyl, a0), ap1 = fmaf(gxz, fyu, a0);
          const float gxy = cx * cy;
          const float am2 = fmaf(gxy, fz[z], a0), ap2 = fmaf(gxy, fz[z + 1], a0);
          float st = am0 * (x_c - xW) + ap0 * (x_c - xE);
          st += am1 * (x_c - xS) + ap1 * (x_c - xN);
          st += am2 * (x_c - x_m) + ap2 * (x_c - x_p);
          const float Lx = sig * x_c + sh * st;
          if (KIND == 1) {
            ((float*)out)[o] = bi - Lx;
          } else {
            float fs = am0 + ap0;
            fs += am1 + ap1;
            fs += am2 + ap2;
            const float D = sig + sh * fs;
            store_out<float>(out, o, mode, out_fp64, x_c + op.omega * (bi - Lx) / D);
          }
        } else if (KIND == 1) {
          ((float*)out)[o] = 0.f;
        } else if (mode == 0) {
          store_out<float>(out, o, 0, out_fp64, 0.f);
        }
      }
      x_m = x_c;
      x_c = x_p;
      xW = x_pW;
      xE = x_pE;
      xS = x_pS;
      xN = x_pN;
    }
  }
  if (!ok) {
    ring.give_up();
    if (lane == 0) lv_timeout(fault);
  }
}

}  // namespace

void prepare_level3_rows() {
  const void* kernels[] = {(const void*)k_level3_rows<5, 1>, (const void*)k_level3_rows<5, 2>,
                           (const void*)k_level3_rows<6, 1>, (const void*)k_level3_rows<6, 2>,
                           (const void*)k_level3_rows<7, 1>, (const void*)k_level3_rows<7, 2>};
  for (const void* k : kernels) resident_grid(k, kLvBand + 32, 0, 1 << 30);
}

namespace {

// the streamed form when it applies (FP32, 3-D, 32 <= P <= 128); false otherwise
template <typename T, int KIND>
bool launch_level3_rows(const T* b, const T* x, void* out, int mode, int out_fp64, StencilGeom<T> g, OpBatch<T> op,
                        int B, int* fault, const int* done, cudaStream_t st) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    if (g.dim != 3 || g.P < 32 || g.P > 128 || op.mass != 0) return false;
    auto go = [&](auto kern, int P) {
      const int grid = resident_grid((const void*)kern, kLvBand + 32, 0, 1 << 30);
      int logR = 5;
      while (logR > 3 && (long long)B * (P / (kLvBand / P)) * (P >> logR) < 4LL * grid) --logR;
      kern<<<grid, kLvBand + 32, 0, st>>>(b, x, out, mode, out_fp64, g, op, B, logR, fault, done);
    };
    if (g.P == 32)
      go(k_level3_rows<5, KIND>, 32);
    else if (g.P == 64)
      go(k_level3_rows<6, KIND>, 64);
    else
      go(k_level3_rows<7, KIND>, 128);
    return true;
  }
}

// ---- one-CTA-per-slice coarse V-cycle ------------------------------------------------------
struct CoarseLevel {
  int n, logP;
  int S;       // slice elements
  int guard;   // zero elements in front
  int off;     // offset (elements) of this level's b array in shared memory; x, r follow
  long long tab;
  float h2inv;
  double h2inv_d;
};

struct CoarsePlan {
  int nl;                       // number of levels handled (lc..L)
  CoarseLevel lv[kMaxLevels];
};

template <int DIM, typename T>
__global__ void k_coarse_vcycle(const T* __restrict__ bglob, long long Sg, void* out, int mode,
                                int out_fp64, const T* __restrict__ tab_all, T a0, OpBatch<T> op,
                                CoarsePlan cp, const int* done) {
  if (stop_requested(done)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = (T*)smem_raw;
  const int slice = blockIdx.x;
  const T sig = op.sig[slice], cth = op.cth[slice], s = op.s, w = op.omega;
  // zero everything (ghosts and guards must read as zero)
  const int total_sm = cp.lv[cp.nl - 1].off + 3 * (cp.lv[cp.nl - 1].guard + cp.lv[cp.nl - 1].S);
  for (int i = threadIdx.x; i < total_sm; i += blockDim.x) sm[i] = (T)0;
  __syncthreads();
  auto B = [&](int l) { return sm + cp.lv[l].off + cp.lv[l].guard; };
  auto X = [&](int l) { return sm + cp.lv[l].off + (cp.lv[l].guard + cp.lv[l].S) + cp.lv[l].guard; };
  auto R = [&](int l) { return sm + cp.lv[l].off + 2 * (cp.lv[l].guard + cp.lv[l].S) + cp.lv[l].guard; };
  // load this slice's rhs
  {
    const CoarseLevel& L0 = cp.lv[0];
    T* b = B(0);
    for (int i = threadIdx.x; i < L0.S; i += blockDim.x) b[i] = bglob[(long long)slice * Sg + i];
  }
  __syncthreads();
  auto geom = [&](int l) {
    StencilGeom<T> g;
    g.dim = DIM;
    g.n = cp.lv[l].n;
    g.logP = cp.lv[l].logP;
    g.P = 1 << g.logP;
    g.S = cp.lv[l].S;
    g.tab = tab_all + cp.lv[l].tab;
    g.a0 = a0;
    g.h2inv = sizeof(T) == 8 ? (T)cp.lv[l].h2inv_d : (T)cp.lv[l].h2inv;
    return g;
  };
  // downward sweep
  for (int l = 0; l + 1 < cp.nl; ++l) {
    const StencilGeom<T> g = geom(l);
    T* b = B(l);
    T* x = X(l);
    T* r = R(l);
    for (int i = threadIdx.x; i < g.S; i += blockDim.x) {
      long long t;
      int xx, y, z;
      if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
        T am[3], ap[3];
        const T D = diag_at<DIM, T>(g, sig, s, cth, xx, y, z, am, ap, op.mass);
        x[i] = w * b[i] / D;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.S; i += blockDim.x) {
      long long t;
      int xx, y, z;
      if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
        T am[3], ap[3];
        face_coefs<DIM, T>(g.tab, g.P, xx, y, z, cth, g.a0, am, ap);
        const T xc = x[i];
        r[i] = b[i] - (sig * mass_apply<DIM, T>(op.mass, x, i, xc, g.P) +
                       s * g.h2inv * stencil_sum<DIM, T>(x, i, xc, am, ap, g.P));
      }
    }
    __syncthreads();
    const CoarseLevel& C = cp.lv[l + 1];
    T* bc = B(l + 1);
    const int Pf = g.P;
    for (int i = threadIdx.x; i < C.S; i += blockDim.x) {
      long long t;
      int x0, y0, z0;
      if (decode<DIM>(i, C.logP, C.n, t, x0, y0, z0)) {
        const long long fc = fine_center<DIM>(x0, y0, z0, Pf);
        T v;
        if (DIM == 1) {
          v = (T)0.25 * r[fc - 1] + (T)0.5 * r[fc] + (T)0.25 * r[fc + 1];
        } else if (DIM == 2) {
          T rows[3];
          for (int oy = -1; oy <= 1; ++oy) {
            const long long c = fc + (long long)oy * Pf;
            rows[oy + 1] = (T)0.25 * r[c - 1] + (T)0.5 * r[c] + (T)0.25 * r[c + 1];
          }
          v = (T)0.25 * rows[0] + (T)0.5 * rows[1] + (T)0.25 * rows[2];
        } else {
          T planes[3];
          for (int oz = -1; oz <= 1; ++oz) {
            T rows[3];
            for (int oy = -1; oy <= 1; ++oy) {
              const long long c = fc + (long long)oz * Pf * Pf + (long long)oy * Pf;
              rows[oy + 1] = (T)0.25 * r[c - 1] + (T)0.5 * r[c] + (T)0.25 * r[c + 1];
            }
            planes[oz + 1] = (T)0.25 * rows[0] + (T)0.5 * rows[1] + (T)0.25 * rows[2];
          }
          v = (T)0.25 * planes[0] + (T)0.5 * planes[1] + (T)0.25 * planes[2];
        }
        bc[i] = v;
      }
    }
    __syncthreads();
  }
  // coarsest level: one point, exact
  {
    const int l = cp.nl - 1;
    const StencilGeom<T> g = geom(l);
    if (threadIdx.x == 0) {
      T am[3], ap[3];
      const T D = diag_at<DIM, T>(g, sig, s, cth, 0, 0, 0, am, ap, op.mass);
      X(l)[0] = B(l)[0] / D;
    }
    __syncthreads();
  }
  // upward sweep
  for (int l = cp.nl - 2; l >= 0; --l) {
    const StencilGeom<T> g = geom(l);
    T* b = B(l);
    T* x = X(l);
    T* r = R(l);
    const T* ec = X(l + 1);
    const int Pc = 1 << cp.lv[l + 1].logP;
    for (int i = threadIdx.x; i < g.S; i += blockDim.x) {
      long long t;
      int xx, y, z;
      if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) x[i] += prolong_at<DIM, T>(ec, 0, Pc, xx, y, z);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.S; i += blockDim.x) {
      long long t;
      int xx, y, z;
      if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
        T am[3], ap[3];
        face_coefs<DIM, T>(g.tab, g.P, xx, y, z, cth, g.a0, am, ap);
        const T xc = x[i];
        r[i] = b[i] - (sig * mass_apply<DIM, T>(op.mass, x, i, xc, g.P) +
                       s * g.h2inv * stencil_sum<DIM, T>(x, i, xc, am, ap, g.P));
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.S; i += blockDim.x) {
      long long t;
      int xx, y, z;
      if (decode<DIM>(i, g.logP, g.n, t, xx, y, z)) {
        T am[3], ap[3];
        const T D = diag_at<DIM, T>(g, sig, s, cth, xx, y, z, am, ap, op.mass);
        x[i] = x[i] + w * r[i] / D;
      }
    }
    __syncthreads();
  }
  // write the level-lc result of this slice
  {
    const CoarseLevel& L0 = cp.lv[0];
    const T* x = X(0);
    for (int i = threadIdx.x; i < L0.S; i += blockDim.x) {
      long long t;
      int xx, y, z;
      const bool inner = decode<DIM>(i, L0.logP, L0.n, t, xx, y, z);
      const long long gi = (long long)slice * Sg + i;
      if (inner)
        store_out<T>(out, gi, mode, out_fp64, x[i]);
      else if (mode == 0)
        store_out<T>(out, gi, 0, out_fp64, (T)0);
    }
  }
}

// ---- exact tridiagonal solve (1-D), one thread per slice -----------------------------------
template <typename T>
__global__ void k_tridiag(const T* __restrict__ r, void* out, int mode, int out_fp64,
                          StencilGeom<T> g, OpBatch<T> op, int B, T* __restrict__ work,
                          const int* done) {
  if (stop_requested(done)) return;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int n = g.n;
  const long long base = (long long)b * g.S;
  T* cp = work + (long long)b * 2 * g.P;
  T* dp = cp + g.P;
  const T sig = op.sig[b], cth = op.cth[b], sh = op.s * g.h2inv;
  const T so = op.mass ? sig * (T)(1.0 / 6.0) : (T)0;  // P1 mass: sig/6 off the diagonal
  T prev_c = (T)0, prev_d = (T)0;
  for (int i = 0; i < n; ++i) {
    T am[1], ap[1];
    face_coefs<1, T>(g.tab, g.P, i, 0, 0, cth, g.a0, am, ap);
    const T lo = i > 0 ? so - sh * am[0] : (T)0;
    const T up = i < n - 1 ? so - sh * ap[0] : (T)0;
    const T di = sig * mass_diag<1, T>(op.mass) + sh * (am[0] + ap[0]);
    const T denom = di - lo * prev_c;
    prev_c = up / denom;
    prev_d = (r[base + i] - lo * prev_d) / denom;
    cp[i] = prev_c;
    dp[i] = prev_d;
  }
  T xn = (T)0;
  for (int i = n - 1; i >= 0; --i) {
    xn = dp[i] - cp[i] * xn;
    store_out<T>(out, base + i, mode, out_fp64, xn);
  }
  if (mode == 0) store_out<T>(out, base + n, 0, out_fp64, (T)0);  // ghost
}

// The same solves by parallel cyclic reduction (n + 1 <= 1024): one CTA per slice, thread i owns
// equation i (a_i x_{i-1} + b_i x_i + c_i x_{i+1} = r_i).  Step s eliminates the couplings at
// distance s by combining equation i with i - s and i + s, so after ceil(log2 n) steps every
// equation stands alone.  The matrices are diagonally dominant (sigma >= 0, a > 0), for which
// the reduction is stable.
template <typename T>
__global__ void k_tridiag_pcr(const T* __restrict__ r, void* out, int mode, int out_fp64, StencilGeom<T> g,
                              OpBatch<T> op, const int* done) {
  if (stop_requested(done)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = g.P, n = g.n, L = blockDim.x;  // L = max(P, 32) rows; rows >= n are identities
  T* sa = (T*)smem_raw;
  T* sb = sa + L;
  T* sc = sb + L;
  T* sr = sc + L;
  const int b = blockIdx.x, i = threadIdx.x;
  const long long base = (long long)b * g.S;
  T ai = (T)0, bi = (T)1, ci = (T)0, ri = (T)0;
  if (i < n) {
    T am[1], ap[1];
    const T sh = op.s * g.h2inv;
    const T so = op.mass ? op.sig[b] * (T)(1.0 / 6.0) : (T)0;  // P1 mass: sig/6 off the diagonal
    face_coefs<1, T>(g.tab, P, i, 0, 0, op.cth[b], g.a0, am, ap);
    ai = i > 0 ? so - sh * am[0] : (T)0;
    ci = i < n - 1 ? so - sh * ap[0] : (T)0;
    bi = op.sig[b] * mass_diag<1, T>(op.mass) + sh * (am[0] + ap[0]);
    ri = r[base + i];
  }
  sa[i] = ai;
  sb[i] = bi;
  sc[i] = ci;
  sr[i] = ri;
  __syncthreads();
  for (int s = 1; s < n; s <<= 1) {
    const int im = i - s, ip = i + s;
    T alpha = (T)0, gamma = (T)0, na = (T)0, nc = (T)0, nb = bi, nr = ri;
    if (i < n && im >= 0) {
      alpha = -ai / sb[im];
      na = alpha * sa[im];
      nb = fma(alpha, sc[im], nb);
      nr = fma(alpha, sr[im], nr);
    }
    if (i < n && ip < n) {
      gamma = -ci / sb[ip];
      nc = gamma * sc[ip];
      nb = fma(gamma, sa[ip], nb);
      nr = fma(gamma, sr[ip], nr);
    }
    __syncthreads();
    ai = na;
    bi = nb;
    ci = nc;
    ri = nr;
    sa[i] = ai;
    sb[i] = bi;
    sc[i] = ci;
    sr[i] = ri;
    __syncthreads();
  }
  if (i < n)
    store_out<T>(out, base + i, mode, out_fp64, ri / bi);
  else if (i < P && mode == 0)
    store_out<T>(out, base + i, 0, out_fp64, (T)0);  // ghost
}

template <int DIM>
double level_dofs(int n, int B) {
  double d = B;
  for (int k = 0; k < DIM; ++k) d *= n;
  return d;
}

// levels lc..nlev-1 of all B slices: one CTA per slice in shared memory; the level-lc input is
// bl, the result goes to `out` (mode) when lc == 0, else to the level-lc correction buffer.
template <int DIM, typename T>
void coarse_launch(const MGPlan<T>& plan, OpBatch<T> op, const T* bl, void* out, int mode,
                   int out_fp64, const int* done, cudaStream_t st) {
  const int B = plan.B;
  CoarsePlan cp;
  cp.nl = plan.nlev - plan.lc;
  int off = 0;
  for (int k = 0; k < cp.nl; ++k) {
    const Level& L = plan.lev[plan.lc + k];
    CoarseLevel& c = cp.lv[k];
    c.n = L.n;
    c.logP = L.logP;
    c.S = (int)L.S;
    c.guard = 0;
    for (int d = 0, pk = 1; d < DIM; ++d, pk *= L.P) c.guard += pk;  // (-1,-1,-1) corner
    c.guard = (c.guard + 3) & ~3;
    c.off = off;
    c.tab = L.tab;
    c.h2inv_d = 1.0 / (L.h * L.h);
    c.h2inv = (float)c.h2inv_d;
    off += 3 * (c.guard + c.S);
  }
  const size_t smem = (size_t)off * sizeof(T);
  set_smem_limit((const void*)k_coarse_vcycle<DIM, T>, 200 * 1024);
  void* dst = plan.lc == 0 ? out : plan.buf[plan.lc].x;
  const int dmode = plan.lc == 0 ? mode : 0;
  const int dfp64 = plan.lc == 0 ? out_fp64 : 0;
  const int threads = plan.lev[plan.lc].S >= 256 ? 256 : 128;
  const double dl = level_dofs<DIM>(plan.lev[plan.lc].n, B);
  LaunchScope ls("mg_coarse", st, dl * (sizeof(T) + (dfp64 ? (dmode == 1 ? 16.0 : 8.0) : (double)sizeof(T))));
  k_coarse_vcycle<DIM, T><<<B, threads, smem, st>>>(bl, plan.lev[plan.lc].S, dst, dmode, dfp64,
                                                    plan.tab, plan.a0, op, cp, done);
}

template <int DIM, typename T>
void vcycle_dim(const MGPlan<T>& plan, OpBatch<T> op, const T* b0, void* out, int mode,
                int out_fp64, const int* done, cudaStream_t st) {
  const int B = plan.B;
  auto geom = [&](int l) {
    StencilGeom<T> g;
    g.dim = DIM;
    g.n = plan.lev[l].n;
    g.P = plan.lev[l].P;
    g.logP = plan.lev[l].logP;
    g.S = plan.lev[l].S;
    g.tab = plan.tab + plan.lev[l].tab;
    g.a0 = plan.a0;
    g.h2inv = (T)(1.0 / (plan.lev[l].h * plan.lev[l].h));
    return g;
  };
  const T* bl = b0;
  for (int l = 0; l < plan.lc; ++l) {
    const StencilGeom<T> g = geom(l);
    const long long total = g.S * B;
    T* x = (T*)plan.buf[l].x;
    T* r = (T*)plan.buf[l].r;
    const Level& C = plan.lev[l + 1];
    const double df = level_dofs<DIM>(g.n, B), dc = level_dofs<DIM>(C.n, B), s = sizeof(T);
    {
      LaunchScope ls("mg_jacobi0", st, 2 * s * df);
      k_jacobi0<DIM, T><<<grid_for(total), kThreads, 0, st>>>(bl, x, g, op, total, done);
    }
    {
      LaunchScope ls("mg_residual", st, 3 * s * df);
      if (!launch_level3_rows<T, 1>(bl, x, r, 0, 0, g, op, B, plan.fault, done, st))
        k_residual<DIM, T><<<grid_for(total), kThreads, 0, st>>>(bl, x, r, g, op, total, done);
    }
    const long long total_c = C.S * B;
    {
      LaunchScope ls("mg_restrict", st, s * (df + dc));
      k_restrict<DIM, T><<<grid_for(total_c), kThreads, 0, st>>>(r, (T*)plan.buf[l + 1].b, g.logP, g.S,
                                                                 C.n, C.logP, total_c, done);
    }
    bl = (const T*)plan.buf[l + 1].b;
  }
  coarse_launch<DIM, T>(plan, op, bl, out, mode, out_fp64, done, st);
  // upward sweep over the global levels: x = x1 + P e, then the post-smoothing in one pass into
  // the level's r buffer (levels > 0; it is the next finer level's coarse correction) or `out`
  for (int l = plan.lc - 1; l >= 0; --l) {
    const StencilGeom<T> g = geom(l);
    const long long total = g.S * B;
    const T* b = l == 0 ? b0 : (const T*)plan.buf[l].b;
    T* x = (T*)plan.buf[l].x;
    T* r = (T*)plan.buf[l].r;
    const Level& C = plan.lev[l + 1];
    const T* ec = (const T*)(l + 1 == plan.lc ? plan.buf[l + 1].x : plan.buf[l + 1].r);
    const double df = level_dofs<DIM>(g.n, B), dc = level_dofs<DIM>(C.n, B), s = sizeof(T);
    {
      LaunchScope ls("mg_prolong_add", st, s * (2 * df + dc));
      k_prolong_add<DIM, T><<<grid_for(total), kThreads, 0, st>>>(x, ec, g, C.logP, C.S, total, done);
    }
    if (l == 0) {
      const double ob = out_fp64 ? (mode == 1 ? 16.0 : 8.0) : (mode == 1 ? 2 * s : s);
      LaunchScope ls("mg_post_smooth", st, (2 * s + ob) * df);
      if (!launch_level3_rows<T, 2>(b, x, out, mode, out_fp64, g, op, B, plan.fault, done, st))
        k_post_smooth<DIM, T><<<grid_for(total), kThreads, 0, st>>>(b, x, out, mode, out_fp64, g, op, total,
                                                                    done);
    } else {
      LaunchScope ls("mg_post_smooth", st, 3 * s * df);
      if (!launch_level3_rows<T, 2>(b, x, r, 0, 0, g, op, B, plan.fault, done, st))
        k_post_smooth<DIM, T><<<grid_for(total), kThreads, 0, st>>>(b, x, r, 0, 0, g, op, total, done);
    }
  }
}

}  // namespace

template <typename T>
void vcycle(const MGPlan<T>& plan, OpBatch<T> op, const T* b0, void* out, int mode, int out_fp64,
            const int* done, cudaStream_t st) {
  switch (plan.dim) {
    case 1: vcycle_dim<1, T>(plan, op, b0, out, mode, out_fp64, done, st); break;
    case 2: vcycle_dim<2, T>(plan, op, b0, out, mode, out_fp64, done, st); break;
    default: vcycle_dim<3, T>(plan, op, b0, out, mode, out_fp64, done, st); break;
  }
}

template <typename T>
void launch_op_residual(const T* b, const T* x, T* r, StencilGeom<T> g, OpBatch<T> op, int B,
                        const int* done, cudaStream_t st) {
  const long long total = g.S * B;
  double d = B;
  for (int k = 0; k < g.dim; ++k) d *= g.n;
  LaunchScope ls("mg_residual", st, 3.0 * sizeof(T) * d);
  switch (g.dim) {
    case 1: k_residual<1, T><<<grid_for(total), kThreads, 0, st>>>(b, x, r, g, op, total, done); break;
    case 2: k_residual<2, T><<<grid_for(total), kThreads, 0, st>>>(b, x, r, g, op, total, done); break;
    default: k_residual<3, T><<<grid_for(total), kThreads, 0, st>>>(b, x, r, g, op, total, done); break;
  }
}

template <typename T>
void vcycle_coarse(const MGPlan<T>& plan, OpBatch<T> op, const T* bl, void* out, int mode, int out_fp64,
                   const int* done, cudaStream_t st) {
  switch (plan.dim) {
    case 1: coarse_launch<1, T>(plan, op, bl, out, mode, out_fp64, done, st); break;
    case 2: coarse_launch<2, T>(plan, op, bl, out, mode, out_fp64, done, st); break;
    default: coarse_launch<3, T>(plan, op, bl, out, mode, out_fp64, done, st); break;
  }
}

template <typename T>
void launch_tridiag(const T* r, void* out, int mode, int out_fp64, StencilGeom<T> g, OpBatch<T> op,
                    int B, T* work, const int* done, cudaStream_t st) {
  const double d = (double)B * g.n, ob = out_fp64 ? (mode == 1 ? 16.0 : 8.0) : (double)sizeof(T);
  LaunchScope ls("tridiag", st, d * (sizeof(T) + ob));
  if (g.P <= 1024)
    k_tridiag_pcr<T><<<B, g.P < 32 ? 32 : g.P, 4 * sizeof(T) * (g.P < 32 ? 32 : g.P), st>>>(r, out, mode, out_fp64,
                                                                                         g, op, done);
  else
    k_tridiag<T><<<(B + 63) / 64, 64, 0, st>>>(r, out, mode, out_fp64, g, op, B, work, done);
}

template void vcycle<float>(const MGPlan<float>&, OpBatch<float>, const float*, void*, int, int, const int*, cudaStream_t);
template void vcycle<double>(const MGPlan<double>&, OpBatch<double>, const double*, void*, int, int, const int*, cudaStream_t);
template void launch_op_residual<float>(const float*, const float*, float*, StencilGeom<float>, OpBatch<float>, int, const int*, cudaStream_t);
template void launch_op_residual<double>(const double*, const double*, double*, StencilGeom<double>, OpBatch<double>, int, const int*, cudaStream_t);
template void vcycle_coarse<float>(const MGPlan<float>&, OpBatch<float>, const float*, void*, int, int, const int*, cudaStream_t);
template void vcycle_coarse<double>(const MGPlan<double>&, OpBatch<double>, const double*, void*, int, int, const int*, cudaStream_t);
template void launch_tridiag<float>(const float*, void*, int, int, StencilGeom<float>, OpBatch<float>, int, float*, const int*, cudaStream_t);
template void launch_tridiag<double>(const double*, void*, int, int, StencilGeom<double>, OpBatch<double>, int, double*, const int*, cudaStream_t);

}  // namespace pt
