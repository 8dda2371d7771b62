// batch.cu -- many volumes in one persistent launch per kind of volume
// (mclahe_batch; no counterpart in the paper), and the launch-shape autotuner
// (mclahe_autotune).
//
// Volumes are grouped by (dimensionality, range mode), which fix the code a
// tile runs.  Each group runs as ONE persistent launch of
// thread-block clusters that pull tiles from a work list through a global
// counter:
//   range tiles  slabs of a volume whose global range must be found;
//   kernel tiles a group of kernels of one volume along its last dimension:
//                histograms and mapping tables (Algorithm 1; the cluster
//                code of hist_impl.cuh);
//   cell tiles   one inter-kernel cell (or a part of it) of one volume:
//                multilinear mapping (Sec. III.C; map_impl.cuh), the
//                cluster's CTAs splitting the cell's rows.
// The list is ordered so that a volume's kernel tiles follow its range tiles
// and its cell tiles follow its kernel tiles, with the volumes interleaved
// (cell tiles of volume v are queued after the kernel tiles of volume v + 1)
// so that the phases of different volumes overlap.  Per-volume ready counters
// order the phases: a kernel tile of v waits until all range tiles of v are
// done, a cell tile until all kernel tiles of v are done.  Every wait depends
// only on tiles handed out earlier, which are held by running clusters, so the
// launch makes progress whatever the residency; each wait is still bounded and
// records MCLAHE_ERR_TIMEOUT in the batch status word when it gives up.
//
// One-dimensional volumes and tables of more than 1280 entries (n_bins > 1024)
// run one mclahe_forward each after the persistent launches.  With use_graph
// the memset of the control block and all launches are captured once into a
// CUDA graph, cached per (plans, pointers), and replayed.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <new>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch_impl.cuh"

namespace mclahe {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

size_t align_ws(size_t x) { return (x + kWsAlign - 1) / kWsAlign * kWsAlign; }

// mclahe_batch_set_wait: polls before a wait gives up, and whether every wait
// target is raised out of reach (testing of the timeout path only)
std::atomic<uint32_t> g_wait_polls{kWaitSpins};
std::atomic<uint32_t> g_wait_unreachable{0};

// Control block: status (16 B), then per launch group a work counter, then
// per volume 2 done counters and 2 range keys.
struct BatchLayout {
    size_t next, done, keys, control, vol0, total;
    std::vector<size_t> vol;    // offset of each volume's forward workspace
};

BatchLayout batch_layout(int n_vol, const mclahe_plan_t *plans) {
    BatchLayout L;
    L.next = 16;
    L.done = L.next + 8 * size_t(n_vol);           // at most one group per volume
    L.keys = L.done + 8 * size_t(n_vol);
    L.control = align_ws(L.keys + 8 * size_t(n_vol));
    size_t off = L.control;
    L.vol0 = off;
    L.vol.resize(n_vol);
    for (int v = 0; v < n_vol; ++v) {
        L.vol[v] = off;
        off = align_ws(off + plans[v]->ws.scratch);   // forward part of the layout
    }
    L.total = off;
    return L;
}

bool same_group(const Geom &a, const Geom &b) { return a.D == b.D && a.mode == b.mode; }

cudaError_t launch_group(const BParams &bp, int D, bool A, int C, size_t smem, cudaStream_t st) {
    switch (D) {
        case 2: return launch_batch_d2(bp, A, C, smem, st);
        case 3: return launch_batch_d3(bp, A, C, smem, st);
        case 4: return launch_batch_d4(bp, A, C, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

// Volumes the persistent kernels take: 2 to 4 dimensions with the replicated
// table layout (at most 1280 table entries); others run one forward each.
bool batchable(const Geom &g) { return g.D >= 2 && map_repl_fits(g.P); }

// Records the whole batch (control memset + one launch per group) on st.
mclahe_status enqueue_batch(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                            float *const *d_out, unsigned char *ws, const float *d_clip,
                            cudaStream_t st) {
    const BatchLayout L = batch_layout(n_vol, plans);
    if (cudaMemsetAsync(ws, 0, L.control, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    // batchable volumes by group, larger volumes first inside a group
    std::vector<int> order;
    for (int v = 0; v < n_vol; ++v)
        if (batchable(plans[v]->g)) order.push_back(v);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const Geom &ga = plans[a]->g, &gb = plans[b]->g;
        if (ga.D != gb.D) return ga.D < gb.D;
        if (ga.mode != gb.mode) return ga.mode < gb.mode;
        return ga.N > gb.N;
    });
    int launch = 0;
    for (size_t i0 = 0; i0 < order.size();) {
        size_t i1 = i0 + 1;
        while (i1 < order.size() && int(i1 - i0) < kGroupVol &&
               same_group(plans[order[i0]]->g, plans[order[i1]]->g))
            ++i1;
        const int nv = int(i1 - i0);
        BParams *bp = new (std::nothrow) BParams;
        if (!bp) return MCLAHE_ERR_NO_MEMORY;
        std::memset(bp, 0, sizeof(*bp));
        bp->n_vol = nv;
        bp->next = reinterpret_cast<unsigned long long *>(ws + L.next + 8 * size_t(launch));
        bp->status = reinterpret_cast<uint32_t *>(ws);
        bp->wait_polls = g_wait_polls.load();
        bp->target_bias = g_wait_unreachable.load() ? 0x80000000u : 0u;
        // cluster size: the most common histogram cluster size of the group
        int C = 1;
        {
            int cnt[4] = {0, 0, 0, 0};
            for (int i = 0; i < nv; ++i) {
                const int c = plans[order[i0 + i]]->t.hist_chunks;
                cnt[c >= 8 ? 3 : c >= 4 ? 2 : c >= 2 ? 1 : 0]++;
            }
            int best = 0;
            for (int j = 1; j < 4; ++j)
                if (cnt[j] > cnt[best]) best = j;
            C = 1 << best;
        }
        size_t smem = 0;
        int64_t nr[kGroupVol], nk[kGroupVol], nc[kGroupVol];
        for (int i = 0; i < nv; ++i) {
            const int v = order[i0 + i];
            const mclahe_plan_s &p = *plans[v];
            unsigned char *vws = ws + L.vol[v];
            BVol &B = bp->v[i];
            B.g = p.g;
            B.in = d_in[v];
            B.out = d_out[v];
            B.hist = reinterpret_cast<uint32_t *>(vws + p.ws.hist);
            B.lut = reinterpret_cast<float *>(vws + p.ws.lut);
            B.lo = reinterpret_cast<float *>(vws + p.ws.lo);
            B.scale = reinterpret_cast<float *>(vws + p.ws.scale);
            B.keys = reinterpret_cast<uint32_t *>(ws + L.keys + 8 * size_t(v));
            B.clip = d_clip ? d_clip + v : nullptr;
            B.R = p.t.hist_copies;
            B.G = p.t.hist_group;
            B.n_hist = hist_items(p.g, B.G);
            B.mgroups = std::max(1, (p.t.map_chunks + C - 1) / C);
            const bool need_range = p.g.mode == MCLAHE_RANGE_GLOBAL && !p.g.has_range;
            B.range_len = int64_t(1) << 20;
            B.n_range = need_range ? (p.g.N + B.range_len - 1) / B.range_len : 0;
            nr[i] = B.n_range;
            nk[i] = B.n_hist;
            nc[i] = n_cells(p.g) * B.mgroups;
            smem = std::max(smem, std::max(hist_smem_bytes(p.g, B.R, B.G, false), map_smem_for(p.g.D, p.g.P, false)));
        }
        // the group's counters: 2 per volume, by group-local index
        bp->done = reinterpret_cast<uint32_t *>(ws + L.done + 8 * i0);
        // stages: all range tiles, then kernel tiles of v0, v1, cell tiles of v0,
        // kernel tiles of v2, cell tiles of v1, ...
        int s = 0;
        int64_t at = 0;
        auto add = [&](int kind, int vi, int64_t n) {
            if (n <= 0) return;
            bp->stage_start[s] = at;
            bp->stage_kind[s] = kind;
            bp->stage_vol[s] = vi;
            at += n;
            ++s;
        };
        for (int i = 0; i < nv; ++i) add(0, i, nr[i]);
        for (int i = 0; i <= nv; ++i) {
            if (i < nv) add(1, i, nk[i]);
            if (i >= 1) add(2, i - 1, nc[i - 1]);
        }
        bp->n_stage = s;
        bp->stage_start[s] = at;
        const Geom &g0 = plans[order[i0]]->g;
        const cudaError_t e = launch_group(*bp, g0.D, g0.mode == MCLAHE_RANGE_ADAPTIVE, C, smem, st);
        delete bp;
        if (e != cudaSuccess) return MCLAHE_ERR_CUDA;
        ++launch;
        i0 = i1;
    }
    for (int v = 0; v < n_vol; ++v) {   // the others, one forward pass each
        if (batchable(plans[v]->g)) continue;
        const mclahe_status s = forward_impl(*plans[v], d_in[v], d_out[v], ws + L.vol[v],
                                             d_clip ? d_clip + v : nullptr, st);
        if (s != MCLAHE_OK) return s;
    }
    return MCLAHE_OK;
}

// graph cache: (plans, pointers) -> executable graph
struct GraphKey {
    std::vector<const void *> ptrs;
    bool operator<(const GraphKey &o) const { return ptrs < o.ptrs; }
};
std::mutex g_graph_mutex;
std::map<GraphKey, cudaGraphExec_t> g_graphs;

// Replay the graph cached under key (plus the current device) on st; on the
// first call capture enqueue(capture stream) into it.
template <typename Enqueue>
mclahe_status replay_cached(GraphKey key, cudaStream_t st, Enqueue &&enqueue) {
    int dev = 0;
    cudaGetDevice(&dev);
    key.ptrs.push_back(reinterpret_cast<const void *>(intptr_t(dev)));
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_graph_mutex);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) exec = it->second;
    }
    if (!exec) {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return MCLAHE_ERR_CUDA;
        cudaGraph_t graph = nullptr;
        mclahe_status s = MCLAHE_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            s = MCLAHE_ERR_CUDA;
        } else {
            s = enqueue(cap);
            if (cudaStreamEndCapture(cap, &graph) != cudaSuccess && s == MCLAHE_OK) s = MCLAHE_ERR_CUDA;
        }
        if (s == MCLAHE_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) s = MCLAHE_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (s != MCLAHE_OK) return s;
        std::lock_guard<std::mutex> lock(g_graph_mutex);
        auto ins = g_graphs.emplace(key, exec);
        if (!ins.second) {   // another thread cached the same graph meanwhile
            cudaGraphExecDestroy(exec);
            exec = ins.first->second;
        }
    }
    return cudaGraphLaunch(exec, st) == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}

// Side streams and events for the concurrent form, per device, created once
// and kept for the process (a captured graph's branches must outlive the capture).
constexpr int kMaxBranches = 16;
struct BranchPool {
    cudaStream_t s[kMaxBranches] = {};
    cudaEvent_t fork = nullptr, join[kMaxBranches] = {};
    bool ok = false;
};
std::mutex g_pool_mutex;
std::map<int, BranchPool> g_pools;

BranchPool *branch_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    BranchPool &p = g_pools[dev];
    if (!p.ok) {
        if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        for (int i = 0; i < kMaxBranches; ++i)
            if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess)
                return nullptr;
        p.ok = true;
    }
    return &p;
}

// Every volume's own forward pass (its plan's launch shapes and walks, its
// own workspace ws[v]) on one of `branches` parallel branches forked from st
// and joined back into it; volumes are dealt longest first to the least
// loaded branch.  The pool's streams and events are shared by the process, so
// one enqueue runs at a time.
std::mutex g_enqueue_mutex;

mclahe_status enqueue_concurrent_ws(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                                    float *const *d_out, unsigned char *const *ws, const float *d_clip,
                                    cudaStream_t st, int branches) {
    BranchPool *pool = branch_pool();
    if (!pool) return MCLAHE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_enqueue_mutex);
    branches = std::max(1, std::min({branches, kMaxBranches, n_vol}));
    std::vector<int> order(n_vol);
    for (int v = 0; v < n_vol; ++v) order[v] = v;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return plans[a]->g.N > plans[b]->g.N; });
    std::vector<int64_t> load(branches, 0);
    std::vector<std::vector<int>> lists(branches);
    for (int v : order) {
        const int b = int(std::min_element(load.begin(), load.end()) - load.begin());
        lists[b].push_back(v);
        load[b] += plans[v]->g.N;
    }
    if (cudaEventRecord(pool->fork, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    for (int b = 0; b < branches; ++b) {
        cudaStream_t sb = pool->s[b];
        if (cudaStreamWaitEvent(sb, pool->fork, 0) != cudaSuccess) return MCLAHE_ERR_CUDA;
        for (int v : lists[b]) {
            const mclahe_status s = forward_impl(*plans[v], d_in[v], d_out[v], ws[v],
                                                 d_clip ? d_clip + v : nullptr, sb);
            if (s != MCLAHE_OK) return s;
        }
        if (cudaEventRecord(pool->join[b], sb) != cudaSuccess) return MCLAHE_ERR_CUDA;
        if (cudaStreamWaitEvent(st, pool->join[b], 0) != cudaSuccess) return MCLAHE_ERR_CUDA;
    }
    return MCLAHE_OK;
}

mclahe_status enqueue_concurrent(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                                 float *const *d_out, unsigned char *ws, const float *d_clip,
                                 cudaStream_t st, int branches) {
    const BatchLayout L = batch_layout(n_vol, plans);
    std::vector<unsigned char *> wsv(n_vol);
    for (int v = 0; v < n_vol; ++v) wsv[v] = ws + L.vol[v];
    return enqueue_concurrent_ws(n_vol, plans, d_in, d_out, wsv.data(), d_clip, st, branches);
}

}  // namespace

void batch_forget_plan(const mclahe_plan_s *p) {
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (std::find(it->first.ptrs.begin(), it->first.ptrs.end(), static_cast<const void *>(p)) !=
            it->first.ptrs.end()) {
            cudaGraphExecDestroy(it->second);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace mclahe

using namespace mclahe;

extern "C" {

size_t mclahe_batch_workspace_bytes(int n_vol, const mclahe_plan_t *plans) {
    if (n_vol < 1 || !plans) return 0;
    for (int v = 0; v < n_vol; ++v)
        if (!plans[v]) return 0;
    return batch_layout(n_vol, plans).total;
}

mclahe_status mclahe_batch(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                           float *const *d_out, void *d_ws, size_t ws_bytes, const float *d_clip,
                           mclahe_stream_t stream, int use_graph) {
    if (n_vol < 1 || !plans || !d_in || !d_out) return MCLAHE_ERR_INVALID_ARG;
    for (int v = 0; v < n_vol; ++v) {
        if (!plans[v] || !d_in[v] || !d_out[v] || d_in[v] == d_out[v]) return MCLAHE_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(d_in[v]) & 15) || (reinterpret_cast<uintptr_t>(d_out[v]) & 15))
            return MCLAHE_ERR_INVALID_ARG;
    }
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & (kWsAlign - 1)) ||
        ws_bytes < mclahe_batch_workspace_bytes(n_vol, plans))
        return MCLAHE_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    if (!use_graph) return enqueue_batch(n_vol, plans, d_in, d_out, ws, d_clip, st);

    GraphKey key;
    for (int v = 0; v < n_vol; ++v) {
        key.ptrs.push_back(plans[v]);
        key.ptrs.push_back(d_in[v]);
        key.ptrs.push_back(d_out[v]);
    }
    key.ptrs.push_back(d_ws);
    key.ptrs.push_back(d_clip);
    // the wait setting is captured into the graph's launch parameters
    key.ptrs.push_back(reinterpret_cast<const void *>(uintptr_t(g_wait_polls.load())));
    key.ptrs.push_back(reinterpret_cast<const void *>(uintptr_t(g_wait_unreachable.load())));
    return replay_cached(key, st, [&](cudaStream_t cap) {
        return enqueue_batch(n_vol, plans, d_in, d_out, ws, d_clip, cap);
    });
}

mclahe_status mclahe_batch_concurrent(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                                      float *const *d_out, void *d_ws, size_t ws_bytes,
                                      const float *d_clip, mclahe_stream_t stream, int branches,
                                      int use_graph) {
    if (n_vol < 1 || !plans || !d_in || !d_out || branches < 1) return MCLAHE_ERR_INVALID_ARG;
    for (int v = 0; v < n_vol; ++v) {
        if (!plans[v] || !d_in[v] || !d_out[v] || d_in[v] == d_out[v]) return MCLAHE_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(d_in[v]) & 15) || (reinterpret_cast<uintptr_t>(d_out[v]) & 15))
            return MCLAHE_ERR_INVALID_ARG;
    }
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & (kWsAlign - 1)) ||
        ws_bytes < mclahe_batch_workspace_bytes(n_vol, plans))
        return MCLAHE_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    if (!use_graph) return enqueue_concurrent(n_vol, plans, d_in, d_out, ws, d_clip, st, branches);
    GraphKey key;
    // a tag no other key has in its first slot, then the plans and pointers
    key.ptrs.push_back(reinterpret_cast<const void *>(uintptr_t(2)));
    for (int v = 0; v < n_vol; ++v) {
        key.ptrs.push_back(plans[v]);
        key.ptrs.push_back(d_in[v]);
        key.ptrs.push_back(d_out[v]);
    }
    key.ptrs.push_back(d_ws);
    key.ptrs.push_back(d_clip);
    key.ptrs.push_back(reinterpret_cast<const void *>(uintptr_t(branches)));
    return replay_cached(key, st, [&](cudaStream_t cap) {
        return enqueue_concurrent(n_vol, plans, d_in, d_out, ws, d_clip, cap, branches);
    });
}

mclahe_status mclahe_forward_batch(mclahe_plan_t plan, int n_vol, const float *const *d_in,
                                   float *const *d_out, void *const *d_ws, size_t ws_bytes,
                                   const float *d_clip, mclahe_stream_t stream, int branches) {
    if (!plan || n_vol < 0 || branches < 1 || (n_vol > 0 && (!d_in || !d_out || !d_ws)))
        return MCLAHE_ERR_INVALID_ARG;
    if (d_clip && (reinterpret_cast<uintptr_t>(d_clip) & 3)) return MCLAHE_ERR_INVALID_ARG;
    for (int v = 0; v < n_vol; ++v) {
        const mclahe_status s = check_forward_args(plan, d_in[v], d_out[v], d_ws[v], ws_bytes);
        if (s != MCLAHE_OK) return s;
        for (int u = 0; u < v; ++u)
            if (d_ws[u] == d_ws[v] || d_out[u] == d_out[v] || d_out[u] == d_in[v] ||
                d_in[u] == d_out[v])
                return MCLAHE_ERR_INVALID_ARG;
    }
    if (n_vol == 0) return MCLAHE_OK;
    std::vector<mclahe_plan_t> plans(n_vol, plan);
    return enqueue_concurrent_ws(n_vol, plans.data(), d_in, d_out,
                                 reinterpret_cast<unsigned char *const *>(d_ws), d_clip,
                                 reinterpret_cast<cudaStream_t>(stream), branches);
}

mclahe_status mclahe_batch_set_wait(uint32_t max_polls, int unreachable) {
    g_wait_polls.store(max_polls ? max_polls : kWaitSpins);
    g_wait_unreachable.store(unreachable ? 1u : 0u);
    return MCLAHE_OK;
}

mclahe_status mclahe_forward_graph(mclahe_plan_t p, const float *d_in, float *d_out, void *d_ws,
                                   size_t ws_bytes, const float *d_clip, mclahe_stream_t stream) {
    mclahe_status s = check_forward_args(p, d_in, d_out, d_ws, ws_bytes);
    if (s != MCLAHE_OK) return s;
    GraphKey key;
    // the forward's key carries a tag that no batch key has in that slot
    key.ptrs = {reinterpret_cast<const void *>(uintptr_t(1)), p, d_in, d_out, d_ws, d_clip};
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    return replay_cached(key, reinterpret_cast<cudaStream_t>(stream), [&](cudaStream_t cap) {
        return forward_impl(*p, d_in, d_out, ws, d_clip, cap);
    });
}

}  // extern "C"
