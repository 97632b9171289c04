// mbar.cuh — shared-memory mbarriers with bounded waits, and bulk asynchronous copies
// (global -> shared) that complete on them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace csar {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the local mbarrier at `a`, for limit_ns at most; false if
// the limit ran out (no endless spin).
__device__ __forceinline__ bool mbar_wait_for(uint32_t a, uint32_t parity, uint64_t limit_ns) {
  if (mbar_test(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int k = 0; k < 64; ++k)
      if (mbar_test(a, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
// The exchange waits: one second at most, after which the kernel latches kErrTimeout
// and goes on.
__device__ __forceinline__ void mbar_wait(uint32_t a, uint32_t parity, Ctl* ctl) {
  if (!mbar_wait_for(a, parity, 1000000000ull) && ctl) atomicOr(&ctl->err, kErrTimeout);
}

// One thread: make an mbarrier initialised by this thread visible to the bulk-copy
// (async) proxy, then arm it for `bytes` and start the copy of `bytes` (a multiple of
// 16, both addresses 16-byte aligned) from global `src` to shared `dst`.
__device__ __forceinline__ void bulk_load_armed(uint32_t dst, const void* src, uint32_t bytes, uint32_t mb) {
  asm volatile("fence.mbarrier_init.release.cluster;\n\tfence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mb)
      : "memory");
}

}  // namespace csar
