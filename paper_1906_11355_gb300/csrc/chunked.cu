// chunked.cu -- mclahe_forward_chunked: Algorithm 1 on a volume held in host
// memory, streamed through a device staging buffer in slabs along dimension
// 0, for volumes that do not fit the device (the limitation the paper names
// in Sec. V: the whole dataset in memory).
//
// Slabs are cut on kernel boundaries along dimension 0:
//   1. global range (GHR without a given range): every slab of rows in turn,
//      min/max accumulated in the range keys;
//   2. histograms: a slab holds the whole footprints (Sec. III.B, mirror
//      images included) of a run of kernel rows [ka, kb) along dimension 0,
//      so their histograms and tables complete within it; the cluster-form
//      histogram kernels run on the items of those rows only;
//   3. mapping: a slab holds the voxels of a run of cell rows [ca, cb) (every
//      table is ready by then); the mapping kernels run on those cells only
//      and the output slab is copied back.
// The kernels address the slab through a base pointer shifted back by the
// slab's first row, so they run unchanged on global coordinates.  The input
// is read from the host two or three times, the output written once.
#include <algorithm>

#include "mclahe_internal.cuh"

namespace mclahe {

cudaError_t launch_range_buffer(const float *buf, int64_t n, uint32_t *keys, cudaStream_t st);
cudaError_t launch_hist_items(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                              const float *d_clip, cudaStream_t st, int64_t item0, int64_t nitems);
cudaError_t launch_map_cells(const mclahe_plan_s &p, const float *in, float *out,
                             const unsigned char *ws, cudaStream_t st, int64_t cell0, int64_t ncells);

namespace {

// a pointer to element -off of p (the kernels index only inside the slab)
template <typename T>
T *shifted(T *p, int64_t off) {
    return reinterpret_cast<T *>(reinterpret_cast<uintptr_t>(p) - uintptr_t(off) * sizeof(float));
}

struct Rows {
    int64_t lo, hi;   // original rows [lo, hi) along dimension 0
};
Rows kernel_rows(const Geom &g, int ka, int kb) {
    Rows r{g.d[0].s, 0};
    for (int k = ka; k < kb; ++k) {
        const Foot f = footprint(g.d[0], k);
        r.lo = std::min<int64_t>(r.lo, f.lo);
        r.hi = std::max<int64_t>(r.hi, f.hi);
    }
    return r;
}
// cell c along dimension 0 covers [c b + b/2 - p0, + b) clamped to [0, s)
Rows cell_rows(const Geom &g, int ca, int cb) {
    const Dim &d = g.d[0];
    auto clampd = [&](int64_t v) { return std::min<int64_t>(std::max<int64_t>(v, 0), d.s); };
    const int64_t a = clampd(int64_t(ca) * d.b + d.b / 2 - d.p0);
    const int64_t b = clampd(int64_t(cb - 1) * d.b + d.b / 2 - d.p0 + d.b);
    return Rows{a, b};
}

}  // namespace

}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_forward_chunked(mclahe_plan_t p, const float *h_in, float *h_out, void *d_ws,
                                                size_t ws_bytes, void *d_stage, size_t stage_bytes,
                                                const float *d_clip, mclahe_stream_t stream) {
    if (!p || !h_in || !h_out || h_in == h_out) return MCLAHE_ERR_INVALID_ARG;
    const Geom &g = p->g;
    if (g.D < 2) return MCLAHE_ERR_UNSUPPORTED;
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & (kWsAlign - 1)) || ws_bytes < p->ws.total)
        return MCLAHE_ERR_WORKSPACE;
    if (!d_stage || (reinterpret_cast<uintptr_t>(d_stage) & 255)) return MCLAHE_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    // two halves of the staging buffer (input and output slabs), in whole rows
    const int64_t row = g.N / g.d[0].s;   // elements per row along dimension 0
    // (a slab starts at its first element rounded down to a multiple of 4, so
    // that the kernels' 16-byte loads stay aligned: 3 elements of slack)
    const int64_t half_rows = (int64_t(stage_bytes / 2 / sizeof(float)) - 8) / row;
    // the widest slab of one kernel row or one cell row must fit
    int64_t need = 0;
    for (int k = 0; k < g.d[0].n; ++k) {
        const Rows r = kernel_rows(g, k, k + 1);
        need = std::max(need, r.hi - r.lo);
    }
    need = std::max<int64_t>(need, g.d[0].b);
    if (half_rows < need) return MCLAHE_ERR_WORKSPACE;
    float *sin = static_cast<float *>(d_stage);
    // the output half starts after the input half's slab (and its slack), 16-byte aligned
    float *sout = sin + ((half_rows * row + 3 + 3) & ~int64_t(3));
    // the histogram pass's shapes: the cluster form with the row ring, as many
    // of the plan's copies as let the ring fit (copies change the speed only)
    mclahe_plan_s q = *p;
    if (q.t.hist_shares > 0) {
        q.t.hist_shares = 0;
        q.t.hist_chunks = 1;
    }
    while (q.t.hist_copies > 1 &&
           hist_smem_bytes(q.g, q.t.hist_copies, q.t.hist_group, 1, q.t.hist_threads) > 220 * 1024)
        q.t.hist_copies >>= 1;
    // elements [e0, r.hi row) of the input into dst, e0 = r.lo row rounded down to 4
    auto first = [&](Rows r) { return (r.lo * row) & ~int64_t(3); };
    auto h2d = [&](float *dst, Rows r) {
        const int64_t e0 = first(r);
        return cudaMemcpyAsync(dst, h_in + e0, sizeof(float) * size_t(r.hi * row - e0),
                               cudaMemcpyHostToDevice, st) == cudaSuccess;
    };

    // 1. global range
    if (g.mode == MCLAHE_RANGE_GLOBAL && !g.has_range) {
        uint32_t *keys = reinterpret_cast<uint32_t *>(ws + p->ws.keys);
        if (cudaMemsetAsync(keys, 0, 2 * sizeof(uint32_t), st) != cudaSuccess) return MCLAHE_ERR_CUDA;
        for (int64_t r0 = 0; r0 < g.d[0].s; r0 += half_rows) {
            const Rows r{r0, std::min<int64_t>(g.d[0].s, r0 + half_rows)};
            if (!h2d(sin, r)) return MCLAHE_ERR_CUDA;
            if (launch_range_buffer(sin, r.hi * row - first(r), keys, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
        }
    }
    // 2. histograms and tables, a run of kernel rows at a time
    const int64_t items_per_row = hist_items(g, q.t.hist_group) / g.d[0].n;
    for (int ka = 0; ka < g.d[0].n;) {
        int kb = ka + 1;
        while (kb < g.d[0].n) {
            const Rows r = kernel_rows(g, ka, kb + 1);
            if (r.hi - r.lo > 2 * half_rows) break;   // the whole staging buffer serves here
            ++kb;
        }
        const Rows r = kernel_rows(g, ka, kb);
        if (!h2d(sin, r)) return MCLAHE_ERR_CUDA;
        if (launch_hist_items(q, shifted(sin, first(r)), ws, d_clip, st, int64_t(ka) * items_per_row,
                              int64_t(kb - ka) * items_per_row) != cudaSuccess)
            return MCLAHE_ERR_CUDA;
        ka = kb;
    }
    // 3. mapping, a run of cell rows at a time
    const int64_t cells_per_row = n_cells(g) / (g.d[0].n - 1);
    for (int ca = 0; ca < g.d[0].n - 1;) {
        int cb = ca + 1;
        while (cb < g.d[0].n - 1) {
            const Rows r = cell_rows(g, ca, cb + 1);
            if (r.hi - r.lo > half_rows) break;
            ++cb;
        }
        const Rows r = cell_rows(g, ca, cb);
        if (r.hi > r.lo) {
            if (!h2d(sin, r)) return MCLAHE_ERR_CUDA;
            const int64_t e0 = first(r);
            if (launch_map_cells(q, shifted(sin, e0), shifted(sout, e0), ws, st, int64_t(ca) * cells_per_row,
                                 int64_t(cb - ca) * cells_per_row) != cudaSuccess)
                return MCLAHE_ERR_CUDA;
            if (cudaMemcpyAsync(h_out + r.lo * row, sout + (r.lo * row - e0),
                                sizeof(float) * size_t((r.hi - r.lo) * row), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess)
                return MCLAHE_ERR_CUDA;
        }
        ca = cb;
    }
    return MCLAHE_OK;
}

extern "C" mclahe_status mclahe_slab_rows(mclahe_plan_t p, mclahe_pass pass, int32_t row0, int32_t row1,
                                          int64_t *first_row, int64_t *end_row) {
    if (!p || !first_row || !end_row || p->g.D < 2 || row0 < 0 || row1 <= row0) return MCLAHE_ERR_INVALID_ARG;
    const Geom &g = p->g;
    Rows r;
    if (pass == MCLAHE_PASS_HIST) {
        if (row1 > g.d[0].n) return MCLAHE_ERR_INVALID_ARG;
        r = kernel_rows(g, row0, row1);
    } else if (pass == MCLAHE_PASS_MAP) {
        if (row1 > g.d[0].n - 1) return MCLAHE_ERR_INVALID_ARG;
        r = cell_rows(g, row0, row1);
    } else if (pass == MCLAHE_PASS_RANGE) {
        if (row1 > g.d[0].s) return MCLAHE_ERR_INVALID_ARG;
        r = Rows{row0, row1};
    } else {
        return MCLAHE_ERR_INVALID_ARG;
    }
    *first_row = r.lo;
    *end_row = r.hi;
    return MCLAHE_OK;
}

extern "C" mclahe_status mclahe_forward_slab(mclahe_plan_t p, mclahe_pass pass, const float *d_slab,
                                             int64_t slab_first, float *d_out_slab, void *d_ws,
                                             size_t ws_bytes, const float *d_clip, int32_t row0,
                                             int32_t row1, mclahe_stream_t stream) {
    if (!p || !d_slab || p->g.D < 2 || slab_first < 0 || (slab_first & 3)) return MCLAHE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_slab) & 15) || (reinterpret_cast<uintptr_t>(d_out_slab) & 15))
        return MCLAHE_ERR_INVALID_ARG;
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & (kWsAlign - 1)) || ws_bytes < p->ws.total)
        return MCLAHE_ERR_WORKSPACE;
    int64_t lo = 0, hi = 0;
    const mclahe_status s = mclahe_slab_rows(p, pass, row0, row1, &lo, &hi);
    if (s != MCLAHE_OK) return s;
    const Geom &g = p->g;
    const int64_t row = g.N / g.d[0].s;
    if (slab_first > lo * row) return MCLAHE_ERR_INVALID_ARG;   // the slab must hold the rows
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    mclahe_plan_s q = *p;
    if (q.t.hist_shares > 0) {
        q.t.hist_shares = 0;
        q.t.hist_chunks = 1;
    }
    while (q.t.hist_copies > 1 &&
           hist_smem_bytes(q.g, q.t.hist_copies, q.t.hist_group, 1, q.t.hist_threads) > 220 * 1024)
        q.t.hist_copies >>= 1;
    cudaError_t e = cudaSuccess;
    if (pass == MCLAHE_PASS_RANGE) {
        if (g.mode != MCLAHE_RANGE_GLOBAL || g.has_range) return MCLAHE_OK;
        // from the row start rounded down to 4 elements (16-byte loads): the few
        // voxels before it belong to the volume too, so the min/max is unchanged
        const int64_t e0 = (lo * row) & ~int64_t(3);
        e = launch_range_buffer(d_slab + (e0 - slab_first), hi * row - e0,
                                reinterpret_cast<uint32_t *>(ws + p->ws.keys), st);
    } else if (pass == MCLAHE_PASS_HIST) {
        const int64_t per = hist_items(g, q.t.hist_group) / g.d[0].n;
        e = launch_hist_items(q, shifted(d_slab, slab_first), ws, d_clip, st, int64_t(row0) * per,
                              int64_t(row1 - row0) * per);
    } else {
        if (!d_out_slab || d_out_slab == d_slab) return MCLAHE_ERR_INVALID_ARG;
        const int64_t per = n_cells(g) / (g.d[0].n - 1);
        e = launch_map_cells(q, shifted(d_slab, slab_first), shifted(d_out_slab, slab_first), ws, st,
                             int64_t(row0) * per, int64_t(row1 - row0) * per);
    }
    return e == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}
