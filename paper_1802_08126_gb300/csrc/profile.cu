// Kernel launch accounting and optional per-kernel timing.
//
// Every launch of the library goes through a LaunchScope, which counts it.  When timing is
// switched on (pt_profile_enable), the scope also records a CUDA event pair on the launch
// stream around the kernel, tagged with the kernel's name and its algorithmic traffic (bytes
// each launch must read and write at least once) and FP64 operation count.  pt_profile_get
// synchronises the pending events and returns per-kernel totals.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "pt_internal.cuh"

namespace pt {
namespace {

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_enabled{0};

struct Pending {
  const char* name;
  cudaEvent_t e0, e1;
  double bytes, flops;
};

struct Totals {
  double ms = 0.0, bytes = 0.0, flops = 0.0;
  unsigned long long launches = 0;
};

std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
std::map<std::string, Totals> g_totals;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_locked() {
  for (Pending& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      Totals& t = g_totals[p.name];
      t.ms += ms;
      t.bytes += p.bytes;
      t.flops += p.flops;
      t.launches += 1;
    }
    g_free.push_back(p.e0);
    g_free.push_back(p.e1);
  }
  g_pending.clear();
}

}  // namespace

std::mutex g_attr_mu;
std::set<std::pair<int, const void*>> g_attr_done;

cudaError_t set_smem_limit(const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done.count({dev, func})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_attr_done.insert({dev, func});
  return e;
}

std::map<std::pair<int, const void*>, int> g_resident;

int resident_grid(const void* func, int threads, size_t smem, int cap) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cap;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto it = g_resident.find({dev, func});
  if (it == g_resident.end()) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      per_sm = 0;
      sms = 0;
    }
    it = g_resident.emplace(std::make_pair(dev, func), per_sm * sms).first;
  }
  const int g = it->second;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

thread_local int g_capturing = 0;
thread_local unsigned long long g_captured = 0;
thread_local int g_step_kind = kAnyStep;

void set_step_kind(int kind) { g_step_kind = kind; }

void note_launch(int count) { g_launches.fetch_add((unsigned long long)count, std::memory_order_relaxed); }

bool profiling_enabled() { return g_enabled.load(std::memory_order_relaxed) != 0; }

void capture_begin() {
  g_capturing = 1;
  g_captured = 0;
}

unsigned long long capture_end() {
  g_capturing = 0;
  return g_captured;
}

LaunchScope::LaunchScope(const char* name, cudaStream_t st, double bytes, double flops, int works_on)
    : name_(name), st_(st), bytes_(bytes), flops_(flops), e0_(nullptr) {
  if (works_on != kAnyStep && g_step_kind != kAnyStep && works_on != g_step_kind) bytes_ = flops_ = 0.0;
  if (g_capturing) {  // recorded into a graph: counted when the graph is launched
    ++g_captured;
    return;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_enabled.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_mu);
    e0_ = take_event();
    cudaEventRecord((cudaEvent_t)e0_, st_);
  }
}

LaunchScope::~LaunchScope() {
  if (e0_ == nullptr) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e1 = take_event();
  cudaEventRecord(e1, st_);
  g_pending.push_back(Pending{name_, (cudaEvent_t)e0_, e1, bytes_, flops_});
  if (g_pending.size() > 4096) drain_locked();
}

}  // namespace pt

extern "C" {

unsigned long long pt_kernel_launch_count(void) { return pt::g_launches.load(); }

void pt_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(pt::g_mu);
  pt::drain_locked();
  pt::g_enabled.store(on ? 1 : 0);
}

void pt_profile_reset(void) {
  std::lock_guard<std::mutex> lk(pt::g_mu);
  pt::drain_locked();
  pt::g_totals.clear();
}

int pt_profile_get(int index, char* name, int name_len, double* total_ms, double* bytes, double* flops,
                   unsigned long long* launches) {
  std::lock_guard<std::mutex> lk(pt::g_mu);
  pt::drain_locked();
  if (index < 0) return (int)pt::g_totals.size();
  int i = 0;
  for (auto& kv : pt::g_totals) {
    if (i++ != index) continue;
    if (name && name_len > 0) {
      const std::string& s = kv.first;
      const int n = (int)s.size() < name_len - 1 ? (int)s.size() : name_len - 1;
      s.copy(name, n);
      name[n] = '\0';
    }
    if (total_ms) *total_ms = kv.second.ms;
    if (bytes) *bytes = kv.second.bytes;
    if (flops) *flops = kv.second.flops;
    if (launches) *launches = kv.second.launches;
    return (int)pt::g_totals.size();
  }
  return -1;
}

}  // extern "C"
