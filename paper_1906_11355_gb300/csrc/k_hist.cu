// k_hist.cu -- the histogram pass of one volume: shapes, shared-memory sizes,
// the TMA box, and the launches with the cp.async row ring (the TMA-tile and
// per-thread-load launches are in k_hist_tma.cu and k_hist_lsu.cu; kernels in
// k_hist_impl.cuh).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "k_hist_impl.cuh"

namespace mclahe {

size_t hist_smem_bytes(const Geom &g, int copies, int group, int walk, int threads) {
    const size_t words = hist_smem_words(g.P, copies, group);
    if (walk == kHistRing) return hist_ring_offset_words(words) * sizeof(uint32_t) + hist_ring_bytes(threads);
    if (walk == kHistTma) return words * sizeof(uint32_t) + 128 + size_t(kHistTmaStages) * kHistTmaStage;
    return words * sizeof(uint32_t);
}

// The range pass of the flat form keeps only keys and ranges, plus the walk's buffers.
size_t hist_range_smem_bytes(int group, int walk, int threads) {
    const size_t words = 5 * size_t(group);
    if (walk == kHistTma) return words * sizeof(uint32_t) + 128 + size_t(kHistTmaStages) * kHistTmaStage;
    if (walk == kHistRing) return hist_ring_offset_words(words) * sizeof(uint32_t) + hist_ring_bytes(threads);
    return words * sizeof(uint32_t);
}

int64_t hist_items(const Geom &g, int group) {
    const int n = g.d[g.D - 1].n;
    return (g.K / n) * ((n + group - 1) / group);
}

// TMA tiles of the histogram pass: every box a work item of G kernels visits
// starts at most 3 elements after a 16-byte boundary and spans at most Bx
// elements from it along the last dim (Bx <= 256, a multiple of 4); By rows
// along dim D-2 fill at most kHistTileFloats.  2- to 4-D volumes whose rows
// start on 16-byte boundaries (last extent a multiple of 4).
bool hist_tma_box(const Geom &g, int G, int &bx, int &by) {
    if (g.D < 2 || g.d[g.D - 1].s % 4 != 0) return false;
    const Dim &dl = g.d[g.D - 1];
    int need = 4;
    for (int kl0 = 0; kl0 < dl.n; kl0 += G) {
        const int kl1 = std::min(kl0 + G, dl.n);
        if (kl1 - kl0 == 1) {
            const Pieces pc = footprint_pieces(dl, kl0);
            for (int i = 0; i < pc.n; ++i)
                need = std::max(need, (pc.a[i] & 3) + std::min(pc.e[i] - pc.a[i], kHistSeg));
        } else {
            int lo = dl.s, hi = 0;
            for (int k = kl0; k < kl1; ++k) {
                const Foot f = footprint(dl, k);
                lo = std::min(lo, f.lo);
                hi = std::max(hi, f.hi);
            }
            need = std::max(need, (lo & 3) + std::min(hi - lo, kHistSeg));
        }
    }
    bx = (need + 3) & ~3;
    if (bx > 256) return false;
    by = std::max(1, std::min({256, kHistTileFloats / bx, g.d[g.D - 2].b}));
    return true;
}

cudaError_t launch_hist_tma(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                            const float *d_clip, cudaStream_t st, bool range, int bx, int by);
cudaError_t launch_hist_lsu(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                            const float *d_clip, cudaStream_t st, bool range);
cudaError_t launch_hist_staged(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                               const float *d_clip, cudaStream_t st);

static cudaError_t launch_any(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                              const float *d_clip, cudaStream_t st, bool range) {
    int bx, by;
    if (p.t.hist_walk == 1 && hist_tma_box(p.g, p.t.hist_group, bx, by))
        return launch_hist_tma(p, in, ws, d_clip, st, range, bx, by);
    if (p.t.hist_walk == 2) return launch_hist_lsu(p, in, ws, d_clip, st, range);
    if (p.t.hist_walk == 3 && !range) return launch_hist_staged(p, in, ws, d_clip, st);
    HistTmaArgs none;
    std::memset(&none.map, 0, sizeof(none.map));
    return launch_hist_walk<kHistRing>(p, in, ws, d_clip, st, none, range);
}

cudaError_t launch_hist_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                              cudaStream_t st) {
    return launch_any(p, in, ws, nullptr, st, true);
}

cudaError_t launch_hist(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                        const float *d_clip, cudaStream_t st) {
    return launch_any(p, in, ws, d_clip, st, false);
}

// Items [item0, item0 + nitems) of the cluster form with the cp.async row ring
// (the plan's groups, clusters and copies; a flat plan runs as one-CTA clusters)
cudaError_t launch_hist_items(const mclahe_plan_s &plan, const float *in, unsigned char *ws,
                              const float *d_clip, cudaStream_t st, int64_t item0, int64_t nitems) {
    // slabs of rows: each footprint's range is swept inside the pass
    mclahe_plan_s p = plan;
    p.t.range_pass = 0;
    HistTmaArgs none;
    std::memset(&none.map, 0, sizeof(none.map));
    const bool a = p.g.mode == MCLAHE_RANGE_ADAPTIVE;
    switch (p.g.D) {
        case 1: return a ? launch_hist_cluster<1, true, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems)
                         : launch_hist_cluster<1, false, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems);
        case 2: return a ? launch_hist_cluster<2, true, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems)
                         : launch_hist_cluster<2, false, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems);
        case 3: return a ? launch_hist_cluster<3, true, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems)
                         : launch_hist_cluster<3, false, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems);
        case 4: return a ? launch_hist_cluster<4, true, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems)
                         : launch_hist_cluster<4, false, kHistRing, float>(p, in, ws, d_clip, st, none, item0, nitems);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
