// Inline PTX for sm_100-family asynchronous copies: mbarrier and the bulk
// (non-tensor) global<->shared copy engine.  Every wait is bounded in time.
#pragma once

#include <cstdint>

namespace pgs {

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // default limit, 2 s: far above any legitimate wait
constexpr uint32_t kErrWaitTimeout = 1u;           // error word bit: a bounded wait expired
constexpr uint32_t kErrBadTile = 2u;               // error word bit: a merge tile did not fit its buffer

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their memory is visible, then let this grid's own
// dependents be scheduled.  Both are no-ops for a grid launched without it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// True once any kernel of the call has set the device error word.  Every
// kernel whose addresses depend on the data (merge-path searches, bulk copies,
// the exchange) returns at once when it is set: a failed tile leaves its
// output unsorted, and the invariants those addresses rest on (sorted lists,
// monotone cuts) no longer hold.  The rest of the call then does nothing
// beyond the statistics, which report the error.
__device__ __forceinline__ bool poisoned(const uint32_t* err) {
  return *reinterpret_cast<const volatile uint32_t*>(err) != 0u;
}

// The same test decided once for the whole CTA (thread 0 reads, a barrier
// shares it), for kernels that synchronise after an early exit.  Every
// thread of the CTA must call it.
__device__ __forceinline__ bool cta_poisoned(const uint32_t* err) {
  __shared__ int s_poisoned;
  if (threadIdx.x == 0) s_poisoned = poisoned(err) ? 1 : 0;
  __syncthreads();
  return s_poisoned != 0;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the async proxy (the copy engine).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive on the barrier and announce `bytes` of transactions to wait for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Wait for phase `phase` of the barrier to complete, for at most limit_ns of
// %globaltimer (0: kWaitLimitNs).  Returns false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint64_t limit_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const uint64_t limit = limit_ns ? limit_ns : kWaitLimitNs;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, phase)) {
    if (global_timer_ns() - t0 > limit) return false;
  }
  return true;
}

// Bulk copy global -> shared; completion is signalled as transaction bytes on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bulk copy shared -> global (the async proxy reads the shared memory; no
// load/store-unit traffic).  dst, src 16-byte aligned; bytes a multiple of 16.
// The writing threads must have run fence_proxy_async_smem() and a barrier
// before it is issued.
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until every committed bulk store of this thread has read its shared
// memory source (the shared memory may then be reused or released).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

}  // namespace pgs
