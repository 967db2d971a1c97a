// msz_tma.cuh -- mbarrier and TMA (cp.async.bulk.tensor) primitives of the
// code pass's plane ring on sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "msz_device.cuh"

namespace msz {
namespace tma {

constexpr uint64_t kWaitNs = 2000000000ull;      // bound of one mbarrier wait (2 s of %globaltimer)
constexpr uint64_t kTestWaitNs = 250000000ull;   // ... under the test hook that withholds a copy

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase of the given parity; gives up after limit_ns, or as
// soon as *dead is set by another thread of the block.  Returns whether the
// phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity, volatile uint32_t *dead,
                                                  uint64_t limit_ns = kWaitNs) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 63u) == 63u) {
            if (*dead) return false;
            const uint64_t now = global_ns();
            if (!t0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// The same between generic-proxy writes to global memory (made visible to
// this thread, e.g. by a grid barrier) and its later TMA reads of them.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One 3D box of a tensor map (coordinates x, y, z; out-of-range elements are
// filled as the map says) into shared memory at dst, completing on bar.
__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

}  // namespace tma
}  // namespace msz
