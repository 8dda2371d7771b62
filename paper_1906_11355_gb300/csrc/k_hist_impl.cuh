// k_hist_impl.cuh -- kernels and launcher templates of the histogram pass of
// one volume (Algorithm 1; the work on one group of kernels along the last
// dimension is in hist_impl.cuh), instantiated per row walk (HW) in k_hist.cu
// (cp.async ring), k_hist_tma.cu (TMA tiles) and k_hist_lsu.cu (per-thread
// loads).  Two forms:
//   cluster: one thread-block cluster per group builds its histograms and
//            mapping tables;
//   flat:    every group is cut into equal shares of its rows, and the shares
//            of all groups are dealt out in order to a persistent grid (one
//            wave), so every CTA does the same work; counts meet in the
//            global histograms and the last CTA of a group builds its tables.
//            With the adaptive range a flat range pass of the same shape
//            first leaves every kernel's min/max.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "hist_impl.cuh"

namespace mclahe {

// Shared-memory address of the TMA stages: behind the histogram words (or
// the keys of the range pass), 128-byte aligned.
__device__ __forceinline__ uint32_t hist_tma_stage0(const uint32_t *sh, size_t words) {
    return (uint32_t(__cvta_generic_to_shared(sh)) + uint32_t(words * 4) + 127u) & ~127u;
}

// 4-D volumes also run 512-thread CTAs (their lane copies fill the shared
// memory, so twice the warps per SM share one copy set).
template <int D, bool ADAPTIVE, int HW, typename T = float>
__global__ void __launch_bounds__(D >= 4 ? 512 : 256, D >= 4 ? 1 : (HW == kHistTma ? 2 : 3))
    k_hist(Geom g, const __grid_constant__ CUtensorMap tmap, int tbx, int tby,
           const T *__restrict__ in, const uint32_t *__restrict__ keys,
           const float *__restrict__ d_clip, uint32_t *__restrict__ hist, float *__restrict__ lut,
           float *__restrict__ lo_out, float *__restrict__ scale_out, int G, int R,
           uint32_t *status, int64_t item0, uint32_t *__restrict__ kkeys) {
    extern __shared__ __align__(128) uint32_t sh[];
    __shared__ __align__(8) uint64_t s_tbar[kHistTmaStages];
    // items in reverse launch order: the first clusters take the volume's end,
    // which the preceding pass (range sweep, or the previous step's mapping)
    // touched last and may still hold in L2; the mapping pass that follows
    // starts at the volume's beginning, which this pass touches last
    const unsigned ncl = cg::this_cluster().num_blocks();
    const int64_t item = item0 + (gridDim.x / ncl - 1 - blockIdx.x / ncl);
    TmaRing<kHistTmaStages> tr{};
    if constexpr (HW == kHistTma)
        tr = tma_ring_init<kHistTmaStages>(s_tbar, hist_tma_stage0(sh, hist_smem_words(g.P, R, G)),
                                           status);
    const HistTma ht{&tmap, tbx, tby};
    // kkeys (nullable): per-kernel ranges left by k_range_kernels
    hist_group<D, ADAPTIVE, kHistCluster, HW, T>(g, in, keys, d_clip, hist, lut, lo_out, scale_out,
                                              item, G, R, sh, 0, 1, 1, nullptr, kkeys, &ht, &tr);
}

// Flat forms: CTA b takes shares [total * b / grid, total * (b + 1) / grid)
// of the work items' S shares each, item by item.
template <int D, bool ADAPTIVE, int MODE, int HW, typename T = float>
__global__ void __launch_bounds__(D >= 4 ? 512 : 256, D >= 4 ? 1 : (HW == kHistTma ? 2 : 3))
    k_hist_flat(Geom g, const __grid_constant__ CUtensorMap tmap, int tbx, int tby,
                const T *__restrict__ in, const uint32_t *__restrict__ keys,
                const float *__restrict__ d_clip, uint32_t *__restrict__ hist,
                float *__restrict__ lut, float *__restrict__ lo_out, float *__restrict__ scale_out,
                uint32_t *__restrict__ kkeys, uint32_t *__restrict__ tickets, int G, int R, int S,
                int64_t total, uint32_t *status) {
    extern __shared__ __align__(128) uint32_t sh[];
    __shared__ __align__(8) uint64_t s_tbar[kHistTmaStages];
    TmaRing<kHistTmaStages> tr{};
    if constexpr (HW == kHistTma)
        tr = tma_ring_init<kHistTmaStages>(
            s_tbar,
            hist_tma_stage0(sh, MODE == kHistMinMax ? 5 * size_t(G) : hist_smem_words(g.P, R, G)),
            status);
    const HistTma ht{&tmap, tbx, tby};
    const int64_t b0 = total * blockIdx.x / gridDim.x;
    const int64_t b1 = total * (blockIdx.x + 1) / gridDim.x;
    for (int64_t s = b0; s < b1;) {
        const int64_t item = s / S;
        const int c0 = int(s - item * S);
        const int64_t rest = b1 - item * S;
        const int c1 = rest < S ? int(rest) : S;
        hist_group<D, ADAPTIVE, MODE, HW, T>(g, in, keys, d_clip, hist, lut, lo_out, scale_out, item, G,
                                          R, sh, c0, c1, S, tickets, kkeys, &ht, &tr);
        s = item * S + c1;
        __syncthreads();   // shared memory is reused by the next item
    }
}

// The TMA box of the histogram pass (Bx, By) and its tensor map, or none.
struct HistTmaArgs {
    CUtensorMap map;
    int bx = 0, by = 0;
};

template <int D, bool ADAPTIVE, int HW, typename T>
static cudaError_t launch_hist_cluster(const mclahe_plan_s &p, const T *in, unsigned char *ws,
                                       const float *d_clip, cudaStream_t st, const HistTmaArgs &ta,
                                       int64_t item0 = 0, int64_t nitems = -1) {
    const Geom &g = p.g;
    const int C = p.t.hist_chunks;
    const size_t smem = hist_smem_bytes(g, p.t.hist_copies, p.t.hist_group, HW, p.t.hist_threads);
    auto kern = k_hist<D, ADAPTIVE, HW, T>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), size_t(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    // items [item0, item0 + nitems) (all by default)
    cfg.gridDim = dim3(unsigned((nitems < 0 ? hist_items(g, p.t.hist_group) : nitems) * C));
    cfg.blockDim = dim3(p.t.hist_threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g, ta.map, ta.bx, ta.by, in,
                              reinterpret_cast<const uint32_t *>(ws + p.ws.keys), d_clip,
                              reinterpret_cast<uint32_t *>(ws + p.ws.hist),
                              reinterpret_cast<float *>(ws + p.ws.lut),
                              reinterpret_cast<float *>(ws + p.ws.lo),
                              reinterpret_cast<float *>(ws + p.ws.scale), p.t.hist_group,
                              p.t.hist_copies, reinterpret_cast<uint32_t *>(ws + p.ws.status), item0,
                              ADAPTIVE && uses_range_pass(p) ? reinterpret_cast<uint32_t *>(ws + p.ws.keys) + 2
                                                             : nullptr);
}

// One launch of a flat form: a persistent grid of as many CTAs as fit on the
// device at once (at most one per share).
template <int D, bool ADAPTIVE, int MODE, int HW, typename T>
static cudaError_t launch_hist_flat(const mclahe_plan_s &p, const T *in, unsigned char *ws,
                                    const float *d_clip, cudaStream_t st, const HistTmaArgs &ta) {
    const Geom &g = p.g;
    const int G = p.t.hist_group, R = p.t.hist_copies, S = p.t.hist_shares;
    const size_t smem = MODE == kHistMinMax ? hist_range_smem_bytes(G, HW, p.t.hist_threads)
                                            : hist_smem_bytes(g, R, G, HW, p.t.hist_threads);
    auto kern = k_hist_flat<D, ADAPTIVE, MODE, HW, T>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), size_t(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cached_occupancy(reinterpret_cast<const void *>(kern), p.t.hist_threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const int sms = device_sms();
    if (per_sm < 1 || sms < 1) return cudaErrorInvalidConfiguration;
    const int64_t total = hist_items(g, G) * S;
    const int grid = int(std::min<int64_t>(total, int64_t(per_sm) * sms));
    p.flat_ctas = grid;
    uint32_t *kkeys = reinterpret_cast<uint32_t *>(ws + p.ws.keys) + 2;
    kern<<<grid, p.t.hist_threads, smem, st>>>(
        g, ta.map, ta.bx, ta.by, in, reinterpret_cast<const uint32_t *>(ws + p.ws.keys), d_clip,
        reinterpret_cast<uint32_t *>(ws + p.ws.hist), reinterpret_cast<float *>(ws + p.ws.lut),
        reinterpret_cast<float *>(ws + p.ws.lo), reinterpret_cast<float *>(ws + p.ws.scale), kkeys,
        reinterpret_cast<uint32_t *>(ws + p.ws.tickets), G, R, S, total,
        reinterpret_cast<uint32_t *>(ws + p.ws.status));
    return cudaGetLastError();
}

// Histogram pass (or, with RANGE, the flat form's adaptive range pass) of a
// D-dimensional volume with row walk HW.
template <int HW, typename T = float>
static cudaError_t launch_hist_walk(const mclahe_plan_s &p, const T *in, unsigned char *ws,
                                    const float *d_clip, cudaStream_t st, const HistTmaArgs &ta,
                                    bool range) {
    const bool adaptive = p.g.mode == MCLAHE_RANGE_ADAPTIVE;
    const bool flat = p.t.hist_shares > 0;
    auto go = [&](auto dtag) -> cudaError_t {
        constexpr int D = decltype(dtag)::value;
        if (range) return launch_hist_flat<D, true, kHistMinMax, HW, T>(p, in, ws, nullptr, st, ta);
        if (flat)
            return adaptive ? launch_hist_flat<D, true, kHistFlat, HW, T>(p, in, ws, d_clip, st, ta)
                            : launch_hist_flat<D, false, kHistFlat, HW, T>(p, in, ws, d_clip, st, ta);
        return adaptive ? launch_hist_cluster<D, true, HW, T>(p, in, ws, d_clip, st, ta)
                        : launch_hist_cluster<D, false, HW, T>(p, in, ws, d_clip, st, ta);
    };
    switch (p.g.D) {
        case 2: return go(std::integral_constant<int, 2>{});
        case 3: return go(std::integral_constant<int, 3>{});
        case 4: return go(std::integral_constant<int, 4>{});
        default:
            if constexpr (HW == kHistTma) return cudaErrorInvalidValue;   // 2- to 4-D boxes
            else return go(std::integral_constant<int, 1>{});
    }
}

}  // namespace mclahe
