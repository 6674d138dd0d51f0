// Bulk asynchronous copies (the Blackwell tensor memory accelerator, TMA) from
// global to shared memory with mbarrier completion, as inline PTX:
//   cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes
// copies `bytes` (a multiple of 16; both addresses 16-byte aligned) and signals the
// transferred byte count on an mbarrier; a thread that arms the barrier with the
// expected byte count (arrive.expect_tx) and then waits on its phase parity sees the
// data once the phase completes.  Every wait here is bounded: it gives up after
// kWaitLimit polls and reports failure, so a kernel never spins forever.
#pragma once
#include <cstdint>

namespace octo {
namespace tma {

// A 640-byte copy lands within microseconds; 65536 polls (each may suspend the
// thread briefly) bound a wait to well under a second.
constexpr int kWaitLimit = 1 << 16;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One arrival per phase (the issuing thread's arrive.expect_tx).
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Invalidates a barrier whose phases have all completed, so that its shared memory
// can be initialised again (or used for anything else): re-initialising a valid
// mbarrier is undefined.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Makes initialised barriers visible to the asynchronous proxy (the copy engine).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier shared-memory accesses before later asynchronous-proxy
// writes to the same shared memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Arms the barrier's current phase for `bytes` of incoming data (this thread's arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Global -> shared bulk copy completing on `bar`.
__device__ __forceinline__ void copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits (at most kWaitLimit polls) for the phase with the given parity; true once
// it has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}

}  // namespace tma
}  // namespace octo
