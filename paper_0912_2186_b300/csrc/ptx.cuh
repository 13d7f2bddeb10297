// Inline-PTX helpers for bulk asynchronous global -> shared copies completed on mbarriers.
// Every wait is bounded: after `limit` polls the caller gets false and records the failure
// instead of spinning on.
#pragma once
#include <cstdint>

#include "wmg_common.cuh"

namespace wmg {

WMG_D uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Programmatic dependent launch (sm_90 and later): a kernel launched with programmatic stream
// serialisation may start while the previous kernel of the stream runs; griddep_wait blocks until
// that kernel has completed and its memory operations are visible (a no-op without the launch
// attribute), and griddep_launch_dependents lets the next such kernel start once every CTA of this
// one has issued it or exited.
WMG_D void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
WMG_D void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

WMG_D void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
WMG_D void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// arrive once and announce `bytes` of bulk-copy transactions on the barrier
WMG_D void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
WMG_D void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

WMG_D bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(phase)
      : "memory");
  return done != 0;
}

WMG_D bool mbar_wait_bounded(uint32_t bar, uint32_t phase, long long limit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

}  // namespace wmg
