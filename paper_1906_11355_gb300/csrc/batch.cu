// batch.cu -- many volumes in one persistent launch per kind of volume
// (mclahe_batch; no counterpart in the paper), and the launch-shape autotuner
// (mclahe_autotune).
//
// Volumes are grouped by (dimensionality, range mode, table layout), which fix
// the code a tile runs.  Each group runs as ONE persistent launch of
// thread-block clusters that pull tiles from a work list through a global
// counter:
//   range tiles  slabs of a volume whose global range must be found;
//   kernel tiles one kernel of one volume: histogram and mapping table
//                (Algorithm 1; the cluster code of hist_impl.cuh);
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
// With use_graph the memset of the control block and the group launches are
// captured once into a CUDA graph, cached per (plans, pointers), and replayed.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <mutex>
#include <tuple>
#include <vector>

#include "hist_impl.cuh"
#include "map_impl.cuh"

namespace mclahe {

constexpr int kGroupVol = 64;                 // volumes per persistent launch
constexpr int kMaxStage = 3 * kGroupVol;
constexpr uint32_t kWaitSpins = 1u << 22;     // ~ seconds with the back-off below

struct BVol {
    Geom g;
    const float *in;
    float *out;
    uint32_t *hist;
    float *lut, *lo, *scale;
    uint32_t *keys;          // global range keys (min complemented, max)
    const float *clip;       // nullable
    int32_t R;               // histogram lane copies
    int32_t mgroups;         // cell tiles per cell (each split over the cluster)
    int64_t n_range;         // range tiles (0: no range pass)
    int64_t range_len;       // voxels per range tile
};

struct BParams {
    int n_vol, n_stage;
    unsigned long long *next;   // work counter
    uint32_t *done;             // per volume: range tiles done, kernel tiles done
    uint32_t *status;           // batch status word
    int64_t stage_start[kMaxStage + 1];
    int32_t stage_kind[kMaxStage];   // 0 range, 1 kernel, 2 cell
    int32_t stage_vol[kMaxStage];
    BVol v[kGroupVol];
};

static_assert(sizeof(BParams) <= 32000, "batch parameters must fit the kernel parameter space");

// Thread 0 waits (bounded) until *ctr >= target; then the block proceeds.
__device__ __forceinline__ void wait_ready(const uint32_t *ctr, uint32_t target, uint32_t *status) {
    if (threadIdx.x == 0) {
        uint32_t spins = 0, ns = 32;
        for (;;) {
            if (*reinterpret_cast<volatile uint32_t *>(status) != 0) break;   // an earlier give-up
            uint32_t v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (++spins > kWaitSpins) {
                atomicCAS(status, 0u, uint32_t(MCLAHE_ERR_TIMEOUT));
                break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
        }
    }
    __syncthreads();
}

// Publish one finished tile: every thread's global writes are done first.
__device__ __forceinline__ void signal_done(uint32_t *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

__device__ __forceinline__ void range_tile(const BVol &V, int64_t idx, int rank, int C) {
    __shared__ float s_mn[32], s_mx[32];
    const int64_t a0 = idx * V.range_len, a1 = min(V.g.N, a0 + V.range_len);
    const int64_t len = a1 - a0;
    const int64_t b0 = a0 + (len * rank) / C, b1 = a0 + (len * (rank + 1)) / C;
    float mn = INFINITY, mx = -INFINITY;
    // aligned middle in 128-bit loads, ends element by element
    const int64_t q0 = (b0 + 3) & ~int64_t(3), q1 = max(q0, b1 & ~int64_t(3));
    for (int64_t i = q0 + 4 * int64_t(threadIdx.x); i < q1; i += 4 * int64_t(blockDim.x)) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(V.in + i));
        mn = min3f(mn, v.x, v.y);
        mn = min3f(mn, v.z, v.w);
        mx = max3f(mx, v.x, v.y);
        mx = max3f(mx, v.z, v.w);
    }
    for (int64_t i = b0 + threadIdx.x; i < min(q0, b1); i += blockDim.x) {
        mn = fminf(mn, V.in[i]);
        mx = fmaxf(mx, V.in[i]);
    }
    for (int64_t i = max(q1, b0) + threadIdx.x; i < b1; i += blockDim.x) {
        mn = fminf(mn, V.in[i]);
        mx = fmaxf(mx, V.in[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_mn[warp] = mn;
        s_mx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < int(blockDim.x >> 5); ++w) {
            mn = fminf(mn, s_mn[w]);
            mx = fmaxf(mx, s_mx[w]);
        }
        if (b1 > b0) {
            atomicMax(&V.keys[0], ~float_key(mn));
            atomicMax(&V.keys[1], float_key(mx));
        }
    }
}

template <int D, bool ADAPTIVE, bool REPL>
__global__ void __launch_bounds__(256, D <= 2 ? 3 : ((D >= 4 && ADAPTIVE) ? 1 : 2)) k_batch(const __grid_constant__ BParams bp) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ unsigned long long s_item;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int64_t total = bp.stage_start[bp.n_stage];
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(bp.next, 1ull);
        cluster.sync();
        const int64_t item = int64_t(*cluster.map_shared_rank(&s_item, 0));
        cluster.sync();   // every CTA has read the tile before rank 0 takes the next
        if (item >= total) break;
        int lo = 0, hi = bp.n_stage - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.stage_start[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int vi = bp.stage_vol[lo];
        const BVol &V = bp.v[vi];
        const int64_t idx = item - bp.stage_start[lo];
        switch (bp.stage_kind[lo]) {
            case 0:
                range_tile(V, idx, rank, C);
                signal_done(&bp.done[2 * vi]);
                break;
            case 1:
                if (V.n_range > 0) wait_ready(&bp.done[2 * vi], uint32_t(V.n_range * C), bp.status);
                hist_kernel<D, ADAPTIVE>(V.g, V.in, V.keys, V.clip, V.hist, V.lut, V.lo, V.scale, idx,
                                         V.R, smem);
                if (rank == 0) signal_done(&bp.done[2 * vi + 1]);
                break;
            default: {
                wait_ready(&bp.done[2 * vi + 1], uint32_t(V.g.K), bp.status);
                const int64_t cell = idx / V.mgroups;
                const int grp = int(idx - cell * V.mgroups);
                map_cell<D, ADAPTIVE, REPL>(V.g, V.in, V.out, V.lut, V.lo, V.scale, cell,
                                            grp * C + rank, V.mgroups * C,
                                            reinterpret_cast<float *>(smem));
                break;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

size_t align_ws(size_t x) { return (x + kWsAlign - 1) / kWsAlign * kWsAlign; }

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

bool same_group(const Geom &a, const Geom &b) {
    return a.D == b.D && a.mode == b.mode && map_repl_fits(a.P) == map_repl_fits(b.P);
}

template <int D, bool A, bool R>
cudaError_t launch_group_t(const BParams &bp, int C, size_t smem, cudaStream_t st) {
    auto kern = k_batch<D, A, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C);
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    const int64_t items = bp.stage_start[bp.n_stage];
    const int64_t grid_clusters = std::min<int64_t>(nclusters, std::max<int64_t>(items, 1));
    cfg.gridDim = dim3(unsigned(grid_clusters * C));
    return cudaLaunchKernelEx(&cfg, kern, bp);
}

cudaError_t launch_group(const BParams &bp, int D, bool A, bool R, int C, size_t smem,
                         cudaStream_t st) {
#define MCLAHE_GROUP(d)                                                              \
    case d:                                                                          \
        if (A) return R ? launch_group_t<d, true, true>(bp, C, smem, st)             \
                        : launch_group_t<d, true, false>(bp, C, smem, st);           \
        return R ? launch_group_t<d, false, true>(bp, C, smem, st)                   \
                 : launch_group_t<d, false, false>(bp, C, smem, st);
    switch (D) {
        MCLAHE_GROUP(1)
        MCLAHE_GROUP(2)
        MCLAHE_GROUP(3)
        MCLAHE_GROUP(4)
        default: return cudaErrorInvalidValue;
    }
#undef MCLAHE_GROUP
}

// Records the whole batch (control memset + one launch per group) on st.
mclahe_status enqueue_batch(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                            float *const *d_out, unsigned char *ws, const float *d_clip,
                            cudaStream_t st) {
    const BatchLayout L = batch_layout(n_vol, plans);
    if (cudaMemsetAsync(ws, 0, L.control, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    // volumes by group, larger volumes first inside a group
    std::vector<int> order(n_vol);
    for (int v = 0; v < n_vol; ++v) order[v] = v;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const Geom &ga = plans[a]->g, &gb = plans[b]->g;
        if (ga.D != gb.D) return ga.D < gb.D;
        if (ga.mode != gb.mode) return ga.mode < gb.mode;
        if (map_repl_fits(ga.P) != map_repl_fits(gb.P)) return map_repl_fits(ga.P);
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
            B.mgroups = std::max(1, (p.t.map_chunks + C - 1) / C);
            const bool need_range = p.g.mode == MCLAHE_RANGE_GLOBAL && !p.g.has_range;
            B.range_len = int64_t(1) << 20;
            B.n_range = need_range ? (p.g.N + B.range_len - 1) / B.range_len : 0;
            nr[i] = B.n_range;
            nk[i] = p.g.K;
            nc[i] = n_cells(p.g) * B.mgroups;
            smem = std::max(smem, std::max(hist_smem_bytes(p.g, B.R), map_smem_bytes(p.g)));
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
        const cudaError_t e = launch_group(*bp, g0.D, g0.mode == MCLAHE_RANGE_ADAPTIVE,
                                           map_repl_fits(g0.P), C, smem, st);
        delete bp;
        if (e != cudaSuccess) return MCLAHE_ERR_CUDA;
        ++launch;
        i0 = i1;
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
            s = enqueue_batch(n_vol, plans, d_in, d_out, ws, d_clip, cap);
            if (cudaStreamEndCapture(cap, &graph) != cudaSuccess && s == MCLAHE_OK) s = MCLAHE_ERR_CUDA;
        }
        if (s == MCLAHE_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) s = MCLAHE_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (s != MCLAHE_OK) return s;
        std::lock_guard<std::mutex> lock(g_graph_mutex);
        auto ins = g_graphs.emplace(key, exec);
        if (!ins.second) {   // another thread cached the same batch meanwhile
            cudaGraphExecDestroy(exec);
            exec = ins.first->second;
        }
    }
    return cudaGraphLaunch(exec, st) == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}

}  // extern "C"
