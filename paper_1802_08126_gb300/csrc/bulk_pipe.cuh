// Row streaming through shared memory: 1-D bulk copies (cp.async.bulk, the TMA engine's untiled
// form) completing on mbarriers, with bounded waits.
//
// A producer warp copies whole rows of the input arrays into a ring of stages; consumer warps wait
// for a stage's "full" barrier (phase parity), read it, and arrive on its "empty" barrier, which
// the producer waits on before refilling the stage.  The copies need no registers while in flight,
// so a few stages per CTA keep enough bytes in flight to cover the DRAM latency without the
// register cost of a deep per-thread load queue.
//
// Every wait is bounded (about two seconds of GPU time, and an iteration cap): a wait that runs
// out returns false and the kernel reports PT_ETIMEOUT instead of spinning forever.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pt {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async (bulk-copy) proxy; follow with __syncthreads.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One arrival that also announces `bytes` of bulk-copy data completing on this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of one wait
constexpr int kWaitTries = 1 << 24;                      // and of its iterations

// Wait until the phase of `bar` with the given parity has completed.  Returns false when the
// bound runs out or *abort (when given) is set by another warp that gave up, true otherwise.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, const volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int k = 0; k < kWaitTries; ++k) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((abort != nullptr && *abort != 0) || global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to shared memory,
// completing on `bar`'s transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace pt

namespace pt {

// Ring of NS stages filled by one producer thread and drained by `consumers` warps.  The producer
// and every consumer walk the same sequence of fills, counting them in `c`: fill c goes to stage
// c % NS, and is that stage's fill number c / NS (the parity of the barrier phases).
template <int NS>
struct RowRing {
  uint64_t full[NS];
  uint64_t empty[NS];
  int abort;

  // one thread, then __syncthreads() before any use
  __device__ __forceinline__ void init(int consumer_warps) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], (unsigned)consumer_warps);
    }
    abort = 0;
    mbar_init_fence();
  }
  // producer: wait until fill c may overwrite its stage; false if the wait gave up
  __device__ __forceinline__ bool acquire(unsigned c) {
    const unsigned r = c / NS;
    return r == 0 || mbar_wait(&empty[c % NS], (r - 1) & 1, &abort);
  }
  // producer: the bulk copies of fill c bring `bytes` in total (issue them after this call)
  __device__ __forceinline__ uint64_t* commit(unsigned c, unsigned bytes) {
    uint64_t* b = &full[c % NS];
    mbar_arrive_expect_tx(b, bytes);
    return b;
  }
  // consumer warp (all lanes): wait for fill c; false for the whole warp if any lane gave up
  __device__ __forceinline__ bool wait(unsigned c) {
    return __all_sync(0xffffffffu, mbar_wait(&full[c % NS], (c / NS) & 1, &abort));
  }
  // consumer warp (all lanes, after their reads of fill c)
  __device__ __forceinline__ void release(unsigned c) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[c % NS]);
  }
  // any thread: make every other wait on this ring give up
  __device__ __forceinline__ void give_up() { *(volatile int*)&abort = 1; }
  // producer, after its last fill (c fills issued): every copy has landed before the CTA exits
  __device__ __forceinline__ bool drain(unsigned c) {
    bool ok = true;
    for (unsigned s = 0; s < (unsigned)NS && s < c; ++s) {
      const unsigned fills = (c - s + NS - 1) / NS;
      ok = mbar_wait(&full[s], (fills - 1) & 1, nullptr) && ok;
    }
    return ok;
  }
};

}  // namespace pt
