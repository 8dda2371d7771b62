// autotune.cu -- mclahe_autotune: pick the launch shapes of a plan's passes by
// timing candidates on the caller's buffers (no counterpart in the paper).
//
// Histogram pass: kernels per work item G in {1, 2, 4, ...} and the whole
// last dimension x lane copies R in {2, 4, 8, 16, 32} (shared memory with the
// row ring at most 200 KiB) x form: a cluster of C in {1, 2, 4, 8} CTAs per
// item, or the flat form with S in {1, 2, 4, ..., 256} shares per item (with
// its range pass, under the adaptive range) x row walk: the cp.async ring or
// TMA tiles (where the geometry allows); and the staged walk (one kernel per
// cluster of C in {1, 2, 4, 8} CTAs, its footprint in shared memory, where it
// fits); for an adaptive range, the cluster form with and without the separate
// streaming range pass.  Mapping pass: per-thread loads
// or TMA tiles (where the geometry allows) x CTAs per cell in {1, 2, 4, ...,
// 64} (at most one row per CTA).  Each candidate runs twice
// after one warm-up and keeps its faster time; results are cached per
// (shape, kernel size, n_bins, range mode, given range) for the process, so a
// later plan of the same problem takes them without timing.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mclahe_internal.cuh"

namespace mclahe {

mclahe_status run_pass(const mclahe_plan_s &p, int pass, const float *in, float *out,
                       unsigned char *ws, const float *d_clip, cudaStream_t st);

namespace {

using TuneKey = std::tuple<int, std::vector<int64_t>, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, Tuning> g_tuned;

TuneKey tune_key(const mclahe_plan_s &p) {
    std::vector<int64_t> dims;
    for (int j = 0; j < p.g.D; ++j) {
        dims.push_back(p.g.d[j].s);
        dims.push_back(p.g.d[j].b);
    }
    return TuneKey(p.g.D, dims, p.g.nb, p.g.mode, p.g.has_range);
}

// Milliseconds of the best of two timed runs of passes [p0, p1] (after a
// warm-up), or a negative value if a launch fails.
float time_passes(mclahe_plan_s &p, int p0, int p1, const float *in, float *out,
                  unsigned char *ws, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    auto run = [&]() {
        for (int pass = p0; pass <= p1; ++pass)
            if (run_pass(p, pass, in, out, ws, nullptr, st) != MCLAHE_OK) return false;
        return true;
    };
    if (!run()) return -1.0f;
    float best = 1e30f;
    for (int r = 0; r < 2; ++r) {
        cudaEventRecord(e0, st);
        if (!run()) return -1.0f;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = ms < best ? ms : best;
    }
    return best;
}

}  // namespace

}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_autotune(mclahe_plan_t p, const float *d_in, float *d_out,
                                         void *d_ws, size_t ws_bytes, mclahe_stream_t stream) {
    mclahe_status s = check_forward_args(p, d_in, d_out, d_ws, ws_bytes);
    if (s != MCLAHE_OK) return s;
    const TuneKey key = tune_key(*p);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            const int bwd = p->t.bwd_chunks;   // fixed by the workspace layout
            p->t = it->second;
            p->t.bwd_chunks = bwd;
            p->tuned = 1;
            batch_forget_plan(p);
            return MCLAHE_OK;
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MCLAHE_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MCLAHE_ERR_CUDA;
    }
    const Tuning t0 = p->t;
    Tuning best = t0;
    s = MCLAHE_OK;
    float best_ms = 1e30f;
    std::vector<int> groups;
    const int nl = p->g.d[p->g.D - 1].n;
    for (int G = 1; G < nl; G <<= 1) groups.push_back(G);
    groups.push_back(nl);
    // every candidate is timed with the passes that feed it (the clear, and
    // the range pass: the flat form's adaptive range is its own pass)
    int64_t item_rows = 1;
    for (int j = 0; j + 1 < p->g.D; ++j) item_rows *= p->g.d[j].b;
    // candidates: G x R x threads per CTA (512 only for 4-D) x walk x form
    struct Cand {
        int G, R, th, walk, C, S, rp;
    };
    const bool rp_ok = range_pass_fits(p->g);
    std::vector<Cand> cands;
    for (int G : groups)
        for (int R = 2; R <= 32; R <<= 1)
            for (int th = 256; th <= (p->g.D >= 4 ? 512 : 256); th *= 2) {
                int bx, by;
                const bool tma_ok = hist_tma_box(p->g, G, bx, by);
                for (int walk = 0; walk < 3; ++walk) {
                    if (walk == 1 && !tma_ok) continue;
                    if (hist_smem_bytes(p->g, R, G, hist_walk_code(walk), th) > 200 * 1024) continue;
                    for (int C = 1; C <= 8; C <<= 1) {
                        cands.push_back({G, R, th, walk, C, 0, 0});
                        if (rp_ok) cands.push_back({G, R, th, walk, C, 0, 1});
                    }
                    for (int S = 1; S <= 256 && S <= item_rows; S <<= 1)
                        cands.push_back({G, R, th, walk, 1, S, 0});
                }
            }
    // the staged walk: one kernel per cluster of 1..8 CTAs
    for (int R = 2; R <= 32; R <<= 1)
        for (int C = 1; C <= 8; C <<= 1)
            if (hist_staged_fits(p->g, R, C, nullptr)) cands.push_back({1, R, 256, 3, C, 0, 0});
    for (const Cand &c : cands) {
        if (s != MCLAHE_OK) break;
        p->t.hist_group = c.G;
        p->t.hist_copies = c.R;
        p->t.hist_threads = c.th;
        p->t.hist_walk = c.walk;
        p->t.hist_chunks = c.C;
        p->t.hist_shares = c.S;
        p->t.range_pass = c.rp;
        const float ms = time_passes(*p, MCLAHE_PASS_CLEAR, MCLAHE_PASS_HIST, d_in, d_out, ws, st, e0, e1);
        if (ms < 0.0f) continue;   // e.g. a cluster shape the device cannot schedule
        if (ms < best_ms) {
            best_ms = ms;
            best.hist_group = c.G;
            best.hist_copies = c.R;
            best.hist_threads = c.th;
            best.hist_walk = c.walk;
            best.hist_chunks = c.C;
            best.hist_shares = c.S;
            best.range_pass = c.rp;
        }
    }
    cudaGetLastError();   // clear a failed candidate's launch error
    if (s == MCLAHE_OK && best_ms >= 1e30f) s = MCLAHE_ERR_CUDA;
    if (s == MCLAHE_OK) {
        p->t = best;
        // tables for the mapping candidates
        for (int pass = MCLAHE_PASS_CLEAR; pass <= MCLAHE_PASS_HIST; ++pass)
            if (run_pass(*p, pass, d_in, d_out, ws, nullptr, st) != MCLAHE_OK) s = MCLAHE_ERR_CUDA;
        int64_t rows = 1;
        for (int j = 0; j + 1 < p->g.D; ++j) rows *= p->g.d[j].b;
        best_ms = 1e30f;
        int bx, by, bz;
        const int n_walks = map_tma_box(p->g, bx, by, bz) ? 2 : 1;
        // walks: per-thread (per-cell grid), per-thread (flat grid), TMA tiles
        for (int walk = 0; walk < 2 + (n_walks > 1 ? 1 : 0); ++walk) {
            p->t.map_tma = walk == 2 ? 1 : 0;
            p->t.map_flat = walk == 1 ? 1 : 0;
            for (int mc = 1; mc <= 64 && mc <= rows && s == MCLAHE_OK; mc <<= 1) {
                p->t.map_chunks = mc;
                const float ms =
                    time_passes(*p, MCLAHE_PASS_MAP, MCLAHE_PASS_MAP, d_in, d_out, ws, st, e0, e1);
                if (ms >= 0.0f && ms < best_ms) {
                    best_ms = ms;
                    best.map_chunks = mc;
                    best.map_tma = p->t.map_tma;
                    best.map_flat = p->t.map_flat;
                }
            }
        }
        cudaGetLastError();
        if (best_ms >= 1e30f) s = MCLAHE_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MCLAHE_OK) {
        p->t = t0;
        return s;
    }
    p->t = best;
    p->tuned = 1;
    batch_forget_plan(p);   // batched graphs captured with the old shapes
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = best;
    return MCLAHE_OK;
}
