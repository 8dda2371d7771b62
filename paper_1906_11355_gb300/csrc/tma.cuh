// tma.cuh -- tensor-memory-accelerator (TMA) tile copies and mbarriers in
// inline PTX (sm_90 and later; used on sm_103a).
//
// A tile copy moves one box of a 3- or 4-D float32 tensor between global and
// shared memory without per-thread loads: the load completes on an mbarrier
// (with the byte count announced by expect_tx), the store is tracked by bulk
// groups.  Coordinates are innermost first; the innermost one must be a
// multiple of 4 (16 bytes).  A box in shared memory is dense, innermost
// dimension fastest, 128-byte aligned.
#pragma once

#include <cstdint>
#include <cuda.h>

namespace mclahe {

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (then a block barrier)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// One bounded probe of phase `parity` of the barrier: true once it completed.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` with an iteration limit; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 64) __nanosleep(256);
    }
    return false;
}

// generic-proxy writes to shared memory before an async-proxy read of them
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int R>
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, const int (&c)[R],
                                         uint32_t bar) {
    static_assert(R == 3 || R == 4, "3- or 4-D boxes");
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    if constexpr (R == 3) {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(bar)
            : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(bar)
            : "memory");
    }
}

template <int R>
__device__ __forceinline__ void tma_store(const CUtensorMap *map, const int (&c)[R], uint32_t src) {
    static_assert(R == 3 || R == 4, "3- or 4-D boxes");
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    if constexpr (R == 3) {
        asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
                     ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(src)
                     : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
            ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(src)
            : "memory");
    }
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// at most N bulk groups may still be reading their shared-memory source
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// every bulk group complete (its global writes done)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace mclahe
