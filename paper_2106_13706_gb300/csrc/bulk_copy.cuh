// bulk_copy.cuh -- global -> shared bulk asynchronous copies (the TMA engine's
// untiled form) completed on shared-memory mbarriers, with bounded waits.
#pragma once
#include <cstdint>

#include "ddks_internal.cuh"

namespace ddks {
namespace bulk {

constexpr unsigned long long kWaitNs = 1000000000ull;   // default bound on one wait (1 s)
// Bound on the waits for copies still in flight after a wait gave up: these
// copies were issued and land within microseconds, and no CTA may exit while
// one of its copies can still write its shared memory.
constexpr unsigned long long kDrainNs = 1000000000ull;

DDKS_DEV void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// makes the initialised barriers visible to the async proxy
DDKS_DEV void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// expect `bytes` more transaction bytes on the current phase of `bar`
DDKS_DEV void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned), counted on `bar`.  Generic-proxy accesses to the destination must
// be ordered before it with fence_async().
DDKS_DEV void load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

DDKS_DEV void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

DDKS_DEV unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of `bar` to complete; false once limit_ns of
// %globaltimer have passed since the first unsuccessful try.
DDKS_DEV bool wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace bulk
}  // namespace ddks
