// plan.cu -- host side of the C ABI: plan validation and geometry
// (Sec. III.B, Eq. (1)-(2)), workspace layout, launch-shape heuristic, the
// forward pass orchestration (Algorithm 1) and status reporting.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include <algorithm>

#include "mclahe_internal.cuh"

namespace mclahe {

static size_t align_up(size_t x) { return (x + kWsAlign - 1) / kWsAlign * kWsAlign; }

// Number of SMs of the current device (152 on GB300), cached per process.
int device_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            sms = 152;
    }
    return sms;
}

int64_t n_cells(const Geom &g) {
    int64_t c = 1;
    for (int j = 0; j < g.D; ++j) c *= (g.d[j].n - 1);
    return c;
}

// Default launch shapes (the autotuner may replace them).  Each CTA should
// own enough voxels to amortise its fixed work (zeroing and summing the
// histogram copies, building tables, staging the corner tables), which the
// timed candidates of mclahe_autotune favour over more, smaller CTAs:
//   histogram: G kernels per work item along the last dimension, so that an
//   item's rows span at least 64 elements (256 bytes); R lane copies, at most
//   16, as many as keep the CTA's shared memory within 64 KiB and the copy
//   summation (G * P * R words) small next to the item's voxels; cluster
//   size C, a power of two up to 8, about one CTA per 300 Ki voxels;
//   mapping: about one CTA per 64 Ki voxels of a cell;
//   both raised to give small volumes at least one CTA per SM while every CTA
//   keeps some thousands of voxels.
Tuning default_tuning(const Geom &g) {
    Tuning t;
    t.hist_threads = 256;   // 512 for 4-D below, with the whole-row group
    t.map_threads = 256;
    const Dim &dl = g.d[g.D - 1];
    int G = std::min(dl.n, std::max(1, (64 + dl.b - 1) / dl.b));
    int R = 16;
    while (R > 1 && (hist_smem_bytes(g, R, G, false) > 64 * 1024 ||
                     int64_t(g.P) * R * G > std::max<int64_t>(g.V * G / 2, int64_t(g.P) * G)))
        R >>= 1;
    while (G > 1 && hist_smem_bytes(g, R, G, false) > 100 * 1024) G >>= 1;
    t.hist_group = G;
    t.hist_copies = R;
    if (g.D >= 4 && hist_smem_bytes(g, R, G, 1, 512) <= 220 * 1024) t.hist_threads = 512;
    const int sms = 152;
    const int64_t vitem = g.V * G, items = hist_items(g, G);
    int C = 1;
    // about one CTA per 300 Ki voxels, and at least one CTA per SM while the
    // CTAs keep 16 Ki voxels or more
    while (C < 8 && (vitem / (2 * C) >= 300 * 1024 ||
                     (items * C < sms && vitem / (2 * C) >= 16 * 1024)))
        C <<= 1;
    t.hist_chunks = C;
    // the cluster form (the flat form and TMA rows are autotuner candidates;
    // neither won on the benchmark volumes)
    t.hist_shares = 0;
    int64_t rows = 1, cell_vox = dl.b;   // rows and voxels of an interior cell
    for (int j = 0; j + 1 < g.D; ++j) {
        rows *= g.d[j].b;
        cell_vox *= g.d[j].b;
    }
    const int64_t cells = n_cells(g);
    int64_t mc = (cell_vox + 65535) / 65536;
    while (cells * mc < sms && cell_vox / (mc + 1) >= 8 * 1024) ++mc;
    t.map_chunks = int(std::min<int64_t>(std::max<int64_t>(std::min(mc, rows), 1), 64));
    // TMA tiles for cell rows shorter than a 128-byte line, where per-thread
    // requests would touch a line per 32 bytes
    int bx, by, bz;
    t.map_tma = (map_tma_box(g, bx, by, bz) && dl.b < 32) ? 1 : 0;
    t.map_flat = 0;
    t.hist_walk = 0;
    // the separate range sweep is an autotuner candidate; on the 3-D
    // fluorescence workload it measured slower than the in-pass sweep
    t.range_pass = 0;
    // Backward chunks per cell: about one CTA per SM for one volume (the
    // batched backward fills the GPU with the other volumes; every chunk
    // restages its cell's tables and closes with block barriers, so fewer,
    // longer chunks run faster), a power of two (a cell's rows -- a power of
    // two times the walk's row groups for power-of-two kernels -- then split
    // into whole row groups, so no warp idles at the closing barrier), and
    // enough of them that the adjoint's integer accumulators hold at most
    // 65535 voxels per chunk: ceil(rows / chunks) rows of b_last voxels
    // (b_last <= 65535, checked by mclahe_plan).
    const auto pow2_floor = [](int64_t v) { while (v & (v - 1)) v &= v - 1; return v; };
    const auto pow2_ceil = [](int64_t v) { int64_t p = 1; while (p < v) p <<= 1; return p; };
    const int64_t rows_max = std::max<int64_t>(65535 / dl.b, 1);
    const int64_t bc_min = pow2_ceil((rows + rows_max - 1) / rows_max);
    int64_t bc = pow2_floor(std::min<int64_t>(std::max<int64_t>((sms + cells - 1) / cells, 1),
                                              std::max<int64_t>(rows / 4, 1)));
    bc = std::max<int64_t>(std::min<int64_t>(bc, 32), bc_min);
    t.bwd_chunks = int(bc);
    return t;
}

Layout make_layout(const Geom &g, const Tuning &t) {
    Layout L;
    size_t off = 0;
    L.status = off;
    off = align_up(off + sizeof(uint32_t) * 4);
    // range keys, work-item tickets and histograms are adjacent: the flat
    // histogram pass accumulates all three and clears them with one memset
    L.keys_count = 2 + 2 * size_t(g.K);
    L.keys = off;
    L.tickets = off + sizeof(uint32_t) * L.keys_count;
    off = align_up(L.tickets + sizeof(uint32_t) * size_t(g.K));
    L.hist = off;
    off = align_up(off + sizeof(uint32_t) * size_t(g.K) * g.nb);
    L.lo = off;
    off = align_up(off + sizeof(float) * size_t(g.K));
    L.scale = off;
    off = align_up(off + sizeof(float) * size_t(g.K));
    L.lut = off;
    off = align_up(off + sizeof(float) * size_t(g.K) * g.LS);
    // backward: partial table gradients (2^D corner tables per cell chunk)
    // and per-kernel threshold gradients
    L.scratch = off;
    L.scratch_bytes = bwd_scratch_bytes(g, t.bwd_chunks);
    off = align_up(off + L.scratch_bytes);
    L.total = off;
    return L;
}

mclahe_status check_forward_args(const mclahe_plan_s *p, const void *in, const void *out,
                                 const void *ws, size_t ws_bytes) {
    if (!p || !in || !out) return MCLAHE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return MCLAHE_ERR_INVALID_ARG;
    if (in == out) return MCLAHE_ERR_INVALID_ARG;
    if (!ws || ws_bytes < p->ws.total || (reinterpret_cast<uintptr_t>(ws) & (kWsAlign - 1)))
        return MCLAHE_ERR_WORKSPACE;
    return MCLAHE_OK;
}

mclahe_status run_pass(const mclahe_plan_s &p, int pass, const float *in, float *out,
                       unsigned char *ws, const float *d_clip, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    switch (pass) {
        case MCLAHE_PASS_CLEAR:
            // what later passes accumulate with atomics: the range keys, and
            // in the flat histogram pass the tickets and histograms
            if (p.t.hist_shares > 0)
                e = cudaMemsetAsync(ws + p.ws.keys, 0,
                                    p.ws.hist + sizeof(uint32_t) * size_t(p.g.K) * p.g.nb - p.ws.keys, st);
            else if (uses_range_pass(p))
                e = cudaMemsetAsync(ws + p.ws.keys, 0, (2 + 2 * size_t(p.g.K)) * sizeof(uint32_t), st);
            else if (p.g.mode == MCLAHE_RANGE_GLOBAL && !p.g.has_range)
                e = cudaMemsetAsync(ws + p.ws.keys, 0, 2 * sizeof(uint32_t), st);
            break;
        case MCLAHE_PASS_RANGE:
            e = p.g.mode == MCLAHE_RANGE_ADAPTIVE && p.t.hist_shares > 0 ? launch_hist_range(p, in, ws, st)
                : uses_range_pass(p)                                    ? launch_range_kernels(p, in, ws, st)
                                                                        : launch_range(p, in, ws, st);
            break;
        case MCLAHE_PASS_HIST: e = launch_hist(p, in, ws, d_clip, st); break;
        case MCLAHE_PASS_LUT: break;   // built by the histogram pass's clusters
        case MCLAHE_PASS_MAP: e = launch_map(p, in, out, ws, st); break;
        default: return MCLAHE_ERR_INVALID_ARG;
    }
    return e == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}

mclahe_status forward_impl(const mclahe_plan_s &p, const float *in, float *out, unsigned char *ws,
                           const float *d_clip, cudaStream_t st) {
    for (int pass = MCLAHE_PASS_CLEAR; pass < MCLAHE_N_PASSES; ++pass) {
        mclahe_status s = run_pass(p, pass, in, out, ws, d_clip, st);
        if (s != MCLAHE_OK) return s;
    }
    return MCLAHE_OK;
}

}  // namespace mclahe

using namespace mclahe;

extern "C" {

mclahe_status mclahe_plan(mclahe_plan_t *out, int ndim, const int64_t *shape,
                          const int32_t *kernel_size, int32_t n_bins, float clip_limit,
                          mclahe_range_mode mode, const float *global_range) {
    if (!out) return MCLAHE_ERR_INVALID_ARG;
    *out = nullptr;
    if (ndim < 1 || ndim > kMaxDim || !shape || !kernel_size) return MCLAHE_ERR_INVALID_ARG;
    if (n_bins < 2 || n_bins > kMaxBins) return MCLAHE_ERR_INVALID_ARG;
    if (!(clip_limit >= 0.0f && clip_limit <= 1.0f)) return MCLAHE_ERR_INVALID_ARG;
    if (mode != MCLAHE_RANGE_GLOBAL && mode != MCLAHE_RANGE_ADAPTIVE) return MCLAHE_ERR_INVALID_ARG;
    if (global_range) {
        if (mode != MCLAHE_RANGE_GLOBAL) return MCLAHE_ERR_INVALID_ARG;
        if (!std::isfinite(global_range[0]) || !std::isfinite(global_range[1]) ||
            global_range[1] < global_range[0])
            return MCLAHE_ERR_INVALID_ARG;
    }
    Geom g;
    std::memset(&g, 0, sizeof(g));
    g.D = ndim;
    g.nb = n_bins;
    g.mode = mode;
    g.clip = clip_limit;
    g.has_range = global_range != nullptr;
    g.range_lo = global_range ? global_range[0] : 0.0f;
    g.range_hi = global_range ? global_range[1] : 0.0f;
    g.K = 1;
    g.V = 1;
    g.N = 1;
    int64_t pad[kMaxDim] = {0, 0, 0, 0};
    for (int j = 0; j < ndim; ++j) {
        const int64_t s = shape[j], b = kernel_size[j];
        if (s < 1 || b < 1 || b > s) return MCLAHE_ERR_INVALID_ARG;
        if (s > (int64_t(1) << 30)) return MCLAHE_ERR_UNSUPPORTED;
        if (j == ndim - 1 && b > 65535) return MCLAHE_ERR_UNSUPPORTED;   // backward chunks
        const int64_t p = 2 * b - 1 - ((s - 1) % b);   // Eq. (1)
        Dim &d = g.d[j];
        d.s = int32_t(s);
        d.b = int32_t(b);
        d.p0 = int32_t(p / 2);                          // Eq. (2)
        d.p1 = int32_t((p + 1) / 2);
        d.n = int32_t((s + p) / b);
        pad[j] = p;
        g.K *= d.n;
        g.V *= b;
        g.N *= s;
        if (g.K > (int64_t(1) << 31) || g.V > (int64_t(1) << 31) || g.N > (int64_t(1) << 40))
            return MCLAHE_ERR_UNSUPPORTED;
    }
    // table geometry of the bin quantiser: indices 0..qk, qk = 2^k >= nb - 1
    g.qk = 1;
    while (g.qk < n_bins - 1) g.qk <<= 1;
    g.qkf = float(g.qk);
    g.iqk = 1.0f / float(g.qk);
    g.P = g.qk + 1;
    g.LS = (g.P + 3) & ~3;
    int64_t stride = 1;
    for (int j = ndim - 1; j >= 0; --j) {
        g.d[j].stride = stride;
        stride *= g.d[j].s;
    }
    // the 2^D neighbouring tables and one histogram (one lane copy at the
    // least) must fit in a CTA's shared memory
    if (map_smem_bytes(g) > 220 * 1024 || hist_smem_bytes(g, 1, 1) > 220 * 1024)
        return MCLAHE_ERR_UNSUPPORTED;
    // CTAs per footprint row range: counts must stay in 32 bits
    int64_t foot = 1;
    for (int j = 0; j < ndim; ++j) foot *= std::min<int64_t>(g.d[j].s, 2 * int64_t(g.d[j].b));
    if (foot > (int64_t(1) << 31)) return MCLAHE_ERR_UNSUPPORTED;

    mclahe_plan_s *p = new (std::nothrow) mclahe_plan_s;
    if (!p) return MCLAHE_ERR_NO_MEMORY;
    std::memset(p, 0, sizeof(*p));
    p->g = g;
    p->t = default_tuning(g);
    p->ws = make_layout(g, p->t);
    for (int j = 0; j < kMaxDim; ++j) p->pad[j] = pad[j];
    p->tuned = 0;
    *out = p;
    return MCLAHE_OK;
}

void mclahe_plan_destroy(mclahe_plan_t plan) {
    if (!plan) return;
    batch_forget_plan(plan);
    delete plan;
}

mclahe_status mclahe_plan_query(mclahe_plan_t p, mclahe_plan_info *info) {
    if (!p || !info) return MCLAHE_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    const Geom &g = p->g;
    info->ndim = g.D;
    info->n_bins = g.nb;
    info->mode = g.mode;
    info->clip_limit = g.clip;
    for (int j = 0; j < g.D; ++j) {
        info->shape[j] = g.d[j].s;
        info->kernel_size[j] = g.d[j].b;
        info->pad[j] = p->pad[j];
        info->pad_before[j] = g.d[j].p0;
        info->pad_after[j] = g.d[j].p1;
        info->n_kernels_dim[j] = g.d[j].n;
    }
    info->n_kernels = g.K;
    info->kernel_voxels = g.V;
    info->n_voxels = g.N;
    info->table_stride = g.LS;
    info->ws_status = p->ws.status;
    info->ws_range_keys = p->ws.keys;
    info->ws_hist = p->ws.hist;
    info->ws_lo = p->ws.lo;
    info->ws_scale = p->ws.scale;
    info->ws_lut = p->ws.lut;
    info->ws_scratch = p->ws.scratch;
    info->ws_bytes = p->ws.total;
    info->hist_group = p->t.hist_group;
    info->hist_cluster = p->t.hist_shares > 0 ? 1 : p->t.hist_chunks;
    info->hist_shares = p->t.hist_shares;
    info->hist_ctas = p->t.hist_shares > 0 ? p->flat_ctas : 0;
    info->map_tma = p->t.map_tma;
    info->hist_walk = p->t.hist_walk;
    info->hist_threads = p->t.hist_threads;
    info->map_flat = p->t.map_flat;
    info->hist_copies = p->t.hist_copies;
    info->map_chunks = p->t.map_chunks;
    info->bwd_chunks = p->t.bwd_chunks;
    info->tuned = p->tuned;
    info->range_pass = p->t.range_pass;
    return MCLAHE_OK;
}

mclahe_status mclahe_plan_set_range_pass(mclahe_plan_t p, int32_t separate) {
    if (!p || (separate != 0 && separate != 1)) return MCLAHE_ERR_INVALID_ARG;
    if (separate && !range_pass_fits(p->g)) return MCLAHE_ERR_UNSUPPORTED;
    p->t.range_pass = separate;
    p->tuned = 2;
    batch_forget_plan(p);   // graphs captured with the old passes
    return MCLAHE_OK;
}

mclahe_status mclahe_plan_set_shapes(mclahe_plan_t p, int32_t hist_group, int32_t hist_cluster,
                                     int32_t hist_copies, int32_t hist_shares, int32_t hist_walk,
                                     int32_t hist_threads, int32_t map_chunks, int32_t map_tma,
                                     int32_t map_flat) {
    if (!p) return MCLAHE_ERR_INVALID_ARG;
    auto pow2 = [](int32_t v, int32_t hi) { return v >= 1 && v <= hi && (v & (v - 1)) == 0; };
    const Geom &g = p->g;
    if (hist_group < 1 || hist_group > g.d[g.D - 1].n) return MCLAHE_ERR_INVALID_ARG;
    if (!pow2(hist_cluster, 8) || !pow2(hist_copies, 32)) return MCLAHE_ERR_INVALID_ARG;
    if (hist_shares < 0 || hist_shares > 4096 || (hist_shares > 0 && hist_cluster != 1))
        return MCLAHE_ERR_INVALID_ARG;
    if (map_chunks < 1 || map_chunks > 64) return MCLAHE_ERR_INVALID_ARG;
    int bx, by, bz;
    if (map_tma != 0 && (map_tma != 1 || !map_tma_box(g, bx, by, bz))) return MCLAHE_ERR_INVALID_ARG;
    if (map_flat != 0 && (map_flat != 1 || map_tma != 0)) return MCLAHE_ERR_INVALID_ARG;
    if (hist_walk < 0 || hist_walk > 3 || (hist_walk == 1 && !hist_tma_box(g, hist_group, bx, by)))
        return MCLAHE_ERR_INVALID_ARG;
    if (hist_threads != 256 && !(hist_threads == 512 && g.D >= 4)) return MCLAHE_ERR_INVALID_ARG;
    if (hist_walk == 3) {
        // one kernel per cluster of 256-thread CTAs, its footprint in shared memory
        if (hist_group != 1 || hist_shares != 0 || hist_threads != 256 ||
            !hist_staged_fits(g, hist_copies, hist_cluster, nullptr))
            return MCLAHE_ERR_INVALID_ARG;
    } else if (hist_smem_bytes(g, hist_copies, hist_group, hist_walk_code(hist_walk), hist_threads) >
               220 * 1024) {
        return MCLAHE_ERR_INVALID_ARG;
    }
    p->t.hist_group = hist_group;
    p->t.hist_chunks = hist_cluster;
    p->t.hist_copies = hist_copies;
    p->t.hist_shares = hist_shares;
    p->t.map_chunks = map_chunks;
    p->t.map_tma = map_tma;
    p->t.map_flat = map_flat;
    p->t.hist_walk = hist_walk;
    p->t.hist_threads = hist_threads;
    p->tuned = 2;
    batch_forget_plan(p);   // batched graphs captured with the old shapes
    return MCLAHE_OK;
}

size_t mclahe_workspace_bytes(mclahe_plan_t p) { return p ? p->ws.total : 0; }

mclahe_status mclahe_forward(mclahe_plan_t p, const float *d_in, float *d_out, void *d_ws,
                             size_t ws_bytes, const float *d_clip, mclahe_stream_t stream) {
    mclahe_status s = check_forward_args(p, d_in, d_out, d_ws, ws_bytes);
    if (s != MCLAHE_OK) return s;
    return forward_impl(*p, d_in, d_out, static_cast<unsigned char *>(d_ws), d_clip,
                        reinterpret_cast<cudaStream_t>(stream));
}

mclahe_status mclahe_forward_pass(mclahe_plan_t p, mclahe_pass pass, const float *d_in,
                                  float *d_out, void *d_ws, size_t ws_bytes, const float *d_clip,
                                  mclahe_stream_t stream) {
    if (pass < MCLAHE_PASS_CLEAR || pass >= MCLAHE_N_PASSES) return MCLAHE_ERR_INVALID_ARG;
    mclahe_status s;
    if (pass == MCLAHE_PASS_MAP) {
        s = check_forward_args(p, d_in, d_out, d_ws, ws_bytes);
    } else {
        // a 16-aligned dummy stands in for the unused output
        s = check_forward_args(p, d_in, reinterpret_cast<const void *>(uintptr_t(16)), d_ws, ws_bytes);
        if (s == MCLAHE_OK && d_out && (reinterpret_cast<uintptr_t>(d_out) & 15))
            s = MCLAHE_ERR_INVALID_ARG;
    }
    if (s != MCLAHE_OK) return s;
    return run_pass(*p, pass, d_in, d_out, static_cast<unsigned char *>(d_ws), d_clip,
                    reinterpret_cast<cudaStream_t>(stream));
}

int mclahe_pass_launches(mclahe_plan_t p, mclahe_pass pass) {
    if (!p) return 0;
    switch (pass) {
        case MCLAHE_PASS_RANGE:
            if (p->g.mode == MCLAHE_RANGE_ADAPTIVE) return p->t.hist_shares > 0 || uses_range_pass(*p) ? 1 : 0;
            return p->g.has_range ? 0 : 1;
        case MCLAHE_PASS_HIST:
        case MCLAHE_PASS_MAP: return 1;
        default: return 0;
    }
}

mclahe_status mclahe_sync_status(void *d_ws, mclahe_stream_t stream) {
    if (!d_ws) return MCLAHE_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    if (cudaMemcpyAsync(&word, d_ws, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MCLAHE_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    if (word != 0) {
        if (cudaMemsetAsync(d_ws, 0, sizeof(word), st) != cudaSuccess) return MCLAHE_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return MCLAHE_ERR_CUDA;
        return word <= MCLAHE_ERR_DEVICE ? mclahe_status(word) : MCLAHE_ERR_DEVICE;
    }
    return MCLAHE_OK;
}

const char *mclahe_status_string(mclahe_status s) {
    switch (s) {
        case MCLAHE_OK: return "ok";
        case MCLAHE_ERR_INVALID_ARG: return "invalid argument";
        case MCLAHE_ERR_UNSUPPORTED: return "unsupported size or parameter";
        case MCLAHE_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case MCLAHE_ERR_CUDA: return "CUDA runtime error";
        case MCLAHE_ERR_TIMEOUT: return "bounded device wait timed out";
        case MCLAHE_ERR_NO_MEMORY: return "host allocation failed";
        case MCLAHE_ERR_DEVICE: return "device code reported an error";
    }
    return "unknown status";
}

int mclahe_version(void) { return 100; }

}  // extern "C"
