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

#include "mclahe.h"

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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
    static_assert(R >= 2 && R <= 4, "2- to 4-D boxes");
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    if constexpr (R == 2) {
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(bar)
            : "memory");
    } else if constexpr (R == 3) {
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

// ---------------------------------------------------------------------------
// TMA tile walk over the rows of a box (histogram pass).
//
// TmaRing: NS stages of STAGE bytes in shared memory and their mbarriers,
// initialised once per CTA (tma_ring_init, all threads) and kept across walks;
// seq counts the tiles consumed so far, so tile q uses stage q mod NS at
// parity (q / NS) mod 2.
// ---------------------------------------------------------------------------
template <int NS>
struct TmaRing {
    uint32_t bar0;     // NS mbarriers, 8 bytes apart
    uint32_t stage0;   // NS stages, 128-byte aligned
    uint32_t seq;
    uint32_t *status;  // workspace status word (a wait that gave up), nullable
};

template <int NS>
__device__ __forceinline__ TmaRing<NS> tma_ring_init(uint64_t *bars, uint32_t stage0, uint32_t *status) {
    TmaRing<NS> r;
    r.bar0 = uint32_t(__cvta_generic_to_shared(bars));
    r.stage0 = stage0;
    r.seq = 0;
    r.status = status;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) mbar_init(r.bar0 + 8u * i, 1);
        mbar_init_fence();
    }
    __syncthreads();
    return r;
}

constexpr uint32_t kTmaWaitSpins = 1u << 22;

// Rows [r0, r1) of a box (rows: all dims but the last, box-relative, C order)
// as tiles of By consecutive rows along dim D-2 (within one plane of the
// outer dims) and Bx elements along the last dim from the 16-byte boundary at
// or below the box start (head = box_lo[D-1] mod 4; head + box_len[D-1] <= Bx).
// Thread t takes quads t + i * blockDim (i < QT) of every tile, at tile
// position (tx, ty) = (4 q mod Bx, 4 q / Bx), with slot data
// slot_fn(i, tx - head); quad_fn(sd, i, v) runs for the quads whose row lies
// in [r0, r1) and in the box and which touch the box along the last dim.
// Thread 0 keeps NS tiles in flight.  All threads of the block call it.
template <int D, int NS, int QT, uint32_t STAGE, typename SD, typename SlotFn, typename QuadFn>
__device__ __forceinline__ void walk_tile_tma(const CUtensorMap *map, const int *box_lo,
                                              const int *box_len, int r0, int r1, int Bx, int By,
                                              TmaRing<NS> &ring, SlotFn slot_fn, QuadFn quad_fn) {
    static_assert(D >= 2 && D <= 4, "2- to 4-D boxes");
    if (r1 <= r0) return;
    const int L = box_len[D - 1];
    const int xa = box_lo[D - 1] & ~3, head = box_lo[D - 1] - xa;
    const int ly = box_len[D - 2];
    const int tile_q = (Bx * By) >> 2;
    SD sd[QT];
    int ty[QT];
    bool ok[QT];
#pragma unroll
    for (int i = 0; i < QT; ++i) {
        const int qi = int(threadIdx.x) + i * int(blockDim.x);
        const int e = 4 * qi;
        const int tx = e % Bx;
        ty[i] = e / Bx;
        const int e0 = tx - head;
        ok[i] = qi < tile_q && e0 < L && e0 + 4 > 0;
        sd[i] = slot_fn(i, e0);
    }
    // tiles: from (plane pa, row ya) on, By rows at a time, restarting at row
    // 0 of each plane, up to flattened row r1
    const int pa = r0 / ly, pb = (r1 - 1) / ly, ya = r0 - pa * ly;
    const int nt = pa == pb ? (r1 - r0 + By - 1) / By
                            : (ly - ya + By - 1) / By + (pb - pa - 1) * ((ly + By - 1) / By) +
                                  (r1 - pb * ly + By - 1) / By;
    auto advance = [&](int &p, int &y) {
        y += By;
        if (y >= ly) {
            ++p;
            y = 0;
        }
    };
    const uint32_t tile_bytes = uint32_t(Bx * By) * 4u;
    int ip = pa, iy = ya;   // next tile to load (thread 0)
    auto issue = [&](int k) {
        const uint32_t s = (ring.seq + uint32_t(k)) % NS;
        int c[D];
        c[0] = xa;
        c[1] = box_lo[D - 2] + iy;
        int rest = ip;
#pragma unroll
        for (int j = D - 3; j >= 0; --j) {
            const int q = rest / box_len[j];
            c[D - 1 - j] = box_lo[j] + (rest - q * box_len[j]);
            rest = q;
        }
        advance(ip, iy);
        mbar_expect_tx(ring.bar0 + 8u * s, tile_bytes);
        tma_load<D>(ring.stage0 + s * STAGE, map, c, ring.bar0 + 8u * s);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < NS && k < nt; ++k) issue(k);
    int cp = pa, cy = ya;   // tile being consumed
    for (int k = 0; k < nt; ++k) {
        const uint32_t q = ring.seq + uint32_t(k), s = q % NS;
        if (!mbar_wait_bounded(ring.bar0 + 8u * s, (q / NS) & 1u, kTmaWaitSpins) && ring.status)
            atomicCAS(ring.status, 0u, uint32_t(MCLAHE_ERR_TIMEOUT));
        const int fr = cp * ly + cy;           // flattened row of the tile's first row
        const int rows = min(By, ly - cy);     // tile rows inside the box
        const uint32_t base = ring.stage0 + s * STAGE;
#pragma unroll
        for (int i = 0; i < QT; ++i) {
            const int r = fr + ty[i];
            if (ok[i] && ty[i] < rows && r >= r0 && r < r1) {
                float4 v;
                asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                             : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                             : "r"(base + 16u * uint32_t(int(threadIdx.x) + i * int(blockDim.x))));
                quad_fn(sd[i], i, v);
            }
        }
        advance(cp, cy);
        __syncthreads();   // the stage is free again
        if (threadIdx.x == 0 && k + NS < nt) issue(k + NS);
    }
    ring.seq += uint32_t(nt);
}

}  // namespace mclahe
