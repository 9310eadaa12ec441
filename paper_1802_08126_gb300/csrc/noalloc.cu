// Allocation-free variant of the forward temporal transform (pt_dst_forward_noalloc).
//
// Some callers of this library cannot let it allocate device memory: their device memory is
// owned by another allocator (for example a framework's caching allocator sized to the whole
// GPU), or they run latency-critical loops in which a cudaMalloc, which may synchronise the
// device, is not acceptable.  For them this entry point computes the same transform as
// pt_dst_forward without a pt_problem and without any allocation: the working copy of the
// input and the transform tables live in one file-scope device array of fixed size.  The array
// is reserved on a device when the library's device code is loaded there; under CUDA's default
// lazy module loading that happens at the first call on the device (its symbol lookup), which
// is why the first call must come before any stream capture.  The device keeps it until the
// process exits.  The address looked up at the first call stays valid for the life of the
// device's context: a cudaDeviceReset invalidates it (and every other device pointer the
// caller holds), so this entry point must not be used on a device after it has been reset.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "pt_internal.cuh"

namespace {

constexpr int kMaxN = 8192;                         // largest number of time slots
constexpr long long kMaxData = 1LL << 21;           // N * padded columns (16 MiB of doubles)
constexpr long long kTables = 3LL * kMaxN;          // twiddles (<= N/2 complex) + pre-twiddles (N complex)
constexpr long long kScratchElems = kTables + kMaxData;

// The scratch array.  In host code its name is only a host-side stand-in: the device address
// comes from cudaGetSymbolAddress, taken once per device below (with that device current).
static __device__ __align__(256) double g_noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices] = {};
std::mutex g_setup_mu;

__global__ void k_tables(double* __restrict__ tw, double* __restrict__ pre, int N) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double s, c;
    if (2 * i < N || (N == 1 && i == 0)) {
      sincospi(2.0 * i / N, &s, &c);  // e^{2 pi i k / N}
      tw[2 * i] = c;
      tw[2 * i + 1] = s;
    }
    sincospi(i / (2.0 * N), &s, &c);  // e^{i pi m / (2N)}
    pre[2 * i] = c;
    pre[2 * i + 1] = s;
  }
}

// copy [N][ncols] into pitch S, zero-filling columns ncols..S-1 (every data element written)
__global__ void k_pack_cols(const double* __restrict__ src, double* __restrict__ dst, int N,
                            long long ncols, long long S) {
  const long long total = (long long)N * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long t = i / S, c = i - t * S;
    dst[i] = c < ncols ? src[t * ncols + c] : 0.0;
  }
}

__global__ void k_unpack_cols(const double* __restrict__ src, double* __restrict__ dst, int N,
                              long long ncols, long long S) {
  const long long total = (long long)N * ncols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long t = i / ncols, c = i - t * ncols;
    dst[i] = src[t * S + c];
  }
}

int blocks_for(long long work) {
  long long b = (work + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

pt_status fail(pt_status s, const std::string& m) {
  pt::set_last_error(m.c_str());
  return s;
}

}  // namespace

extern "C" {

pt_status pt_dst_forward_noalloc(const double* r_dev, double* out_dev, int N_t, long long ncols,
                                 void* stream) {
  pt::set_last_error("");
  if (!r_dev || !out_dev) return fail(PT_EINVAL, "NULL argument");
  if (N_t < 1 || N_t > kMaxN || (N_t & (N_t - 1)) != 0)
    return fail(PT_EINVAL, "N_t must be a power of two in [1, 8192]");
  if (ncols < 1) return fail(PT_EINVAL, "ncols must be >= 1");
  const long long S = (ncols + 31) / 32 * 32;
  if ((long long)N_t * S > kMaxData)
    return fail(PT_EINVAL, "N_t * ceil32(ncols) = " + std::to_string((long long)N_t * S) +
                               " exceeds the fixed scratch of " + std::to_string(kMaxData) +
                               " doubles (16 MiB)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PT_EINVAL, "device index out of range");
  double* base = nullptr;
  {
    // first call on this device: resolve the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(PT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_dev[dev] = (double*)ptr;
    }
    base = g_scratch_dev[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* tw = base;                   // max(1, N/2) complex: <= kMaxN doubles
  double* pre = base + kMaxN;          // N complex: <= 2 kMaxN doubles
  double* data = base + kTables;       // N x S padded copy of the input, transformed in place
  int logN = 0;
  while ((1 << logN) < N_t) ++logN;
  k_tables<<<blocks_for(N_t), 256, 0, st>>>(tw, pre, N_t);
  k_pack_cols<<<blocks_for((long long)N_t * S), 256, 0, st>>>(r_dev, data, N_t, ncols, S);
  pt::note_launch(2);
  pt::DstPlan<double> plan;
  plan.N = N_t;
  plan.logN = logN;
  plan.tw = tw;
  plan.pre = pre;
  pt::launch_dst_forward_plain(data, S, (int)ncols, plan, st);
  k_unpack_cols<<<blocks_for((long long)N_t * ncols), 256, 0, st>>>(data, out_dev, N_t, ncols, S);
  pt::note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PT_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return PT_OK;
}

}  // extern "C"
