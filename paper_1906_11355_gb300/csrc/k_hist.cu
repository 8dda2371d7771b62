// k_hist.cu -- launchers of the histogram pass of one volume (Algorithm 1;
// the work on one group of kernels along the last dimension is in
// hist_impl.cuh).  Two forms:
//   cluster: one thread-block cluster per group builds its histograms and
//            mapping tables;
//   flat:    every group is cut into equal shares of its rows, and the shares
//            of all groups are dealt out in order to a persistent grid (one
//            wave), so every CTA does the same work; counts meet in the
//            global histograms and the last CTA of a group builds its tables.
//            With the adaptive range a flat range pass of the same shape
//            first leaves every kernel's min/max.
#include <algorithm>

#include "hist_impl.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(256, D >= 4 ? 2 : 3) k_hist(Geom g, const float *__restrict__ in,
                                              const uint32_t *__restrict__ keys,
                                              const float *__restrict__ d_clip,
                                              uint32_t *__restrict__ hist, float *__restrict__ lut,
                                              float *__restrict__ lo_out,
                                              float *__restrict__ scale_out, int G, int R) {
    extern __shared__ __align__(16) uint32_t sh[];
    const int64_t item = blockIdx.x / cg::this_cluster().num_blocks();
    hist_group<D, ADAPTIVE, kHistCluster, true>(g, in, keys, d_clip, hist, lut, lo_out, scale_out,
                                                item, G, R, sh);
}

// Flat forms: CTA b takes shares [total * b / grid, total * (b + 1) / grid)
// of the work items' S shares each, item by item.
template <int D, bool ADAPTIVE, int MODE>
__global__ void __launch_bounds__(256, D >= 4 ? 2 : 3)
    k_hist_flat(Geom g, const float *__restrict__ in, const uint32_t *__restrict__ keys,
                const float *__restrict__ d_clip, uint32_t *__restrict__ hist,
                float *__restrict__ lut, float *__restrict__ lo_out, float *__restrict__ scale_out,
                uint32_t *__restrict__ kkeys, uint32_t *__restrict__ tickets, int G, int R, int S,
                int64_t total) {
    extern __shared__ __align__(16) uint32_t sh[];
    const int64_t b0 = total * blockIdx.x / gridDim.x;
    const int64_t b1 = total * (blockIdx.x + 1) / gridDim.x;
    for (int64_t s = b0; s < b1;) {
        const int64_t item = s / S;
        const int c0 = int(s - item * S);
        const int64_t rest = b1 - item * S;
        const int c1 = rest < S ? int(rest) : S;
        hist_group<D, ADAPTIVE, MODE, true>(g, in, keys, d_clip, hist, lut, lo_out, scale_out, item,
                                            G, R, sh, c0, c1, S, tickets, kkeys);
        s = item * S + c1;
        __syncthreads();   // shared memory is reused by the next item
    }
}

size_t hist_smem_bytes(const Geom &g, int copies, int group, bool ring) {
    const size_t words = hist_smem_words(g.P, copies, group);
    return ring ? hist_ring_offset_words(words) * sizeof(uint32_t) + hist_ring_bytes(256)
                : words * sizeof(uint32_t);
}

// The range pass of the flat form keeps only keys and ranges, plus the ring.
static size_t hist_range_smem_bytes(int group) {
    return hist_ring_offset_words(5 * size_t(group)) * sizeof(uint32_t) + hist_ring_bytes(256);
}

int64_t hist_items(const Geom &g, int group) {
    const int n = g.d[g.D - 1].n;
    return (g.K / n) * ((n + group - 1) / group);
}

template <int D, bool ADAPTIVE>
static cudaError_t launch_hist_dm(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                  const float *d_clip, cudaStream_t st) {
    const Geom &g = p.g;
    const int C = p.t.hist_chunks;
    const size_t smem = hist_smem_bytes(g, p.t.hist_copies, p.t.hist_group);
    cudaError_t e = cudaFuncSetAttribute(k_hist<D, ADAPTIVE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(hist_items(g, p.t.hist_group) * C));
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
    return cudaLaunchKernelEx(&cfg, k_hist<D, ADAPTIVE>, g, in,
                              reinterpret_cast<const uint32_t *>(ws + p.ws.keys), d_clip,
                              reinterpret_cast<uint32_t *>(ws + p.ws.hist),
                              reinterpret_cast<float *>(ws + p.ws.lut),
                              reinterpret_cast<float *>(ws + p.ws.lo),
                              reinterpret_cast<float *>(ws + p.ws.scale), p.t.hist_group,
                              p.t.hist_copies);
}

static int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
        return 0;
    return n;
}

// One launch of a flat form: a persistent grid of as many CTAs as fit on the
// device at once (at most one per share).
template <int D, bool ADAPTIVE, int MODE>
static cudaError_t launch_flat(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                               const float *d_clip, cudaStream_t st) {
    const Geom &g = p.g;
    const int G = p.t.hist_group, R = p.t.hist_copies, S = p.t.hist_shares;
    const size_t smem = MODE == kHistMinMax ? hist_range_smem_bytes(G) : hist_smem_bytes(g, R, G);
    auto kern = k_hist_flat<D, ADAPTIVE, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.t.hist_threads, smem);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    if (per_sm < 1 || sms < 1) return cudaErrorInvalidConfiguration;
    const int64_t total = hist_items(g, G) * S;
    const int grid = int(std::min<int64_t>(total, int64_t(per_sm) * sms));
    p.flat_ctas = grid;
    uint32_t *kkeys = reinterpret_cast<uint32_t *>(ws + p.ws.keys) + 2;
    kern<<<grid, p.t.hist_threads, smem, st>>>(
        g, in, reinterpret_cast<const uint32_t *>(ws + p.ws.keys), d_clip,
        reinterpret_cast<uint32_t *>(ws + p.ws.hist), reinterpret_cast<float *>(ws + p.ws.lut),
        reinterpret_cast<float *>(ws + p.ws.lo), reinterpret_cast<float *>(ws + p.ws.scale), kkeys,
        reinterpret_cast<uint32_t *>(ws + p.ws.tickets), G, R, S, total);
    return cudaGetLastError();
}

// The adaptive range of the flat form (the range pass).
template <int D>
static cudaError_t launch_hist_range_d(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                       cudaStream_t st) {
    return launch_flat<D, true, kHistMinMax>(p, in, ws, nullptr, st);
}

cudaError_t launch_hist_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                              cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_hist_range_d<1>(p, in, ws, st);
        case 2: return launch_hist_range_d<2>(p, in, ws, st);
        case 3: return launch_hist_range_d<3>(p, in, ws, st);
        case 4: return launch_hist_range_d<4>(p, in, ws, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int D>
static cudaError_t launch_hist_d(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                 const float *d_clip, cudaStream_t st) {
    const bool adaptive = p.g.mode == MCLAHE_RANGE_ADAPTIVE;
    if (p.t.hist_shares > 0)
        return adaptive ? launch_flat<D, true, kHistFlat>(p, in, ws, d_clip, st)
                        : launch_flat<D, false, kHistFlat>(p, in, ws, d_clip, st);
    if (adaptive) return launch_hist_dm<D, true>(p, in, ws, d_clip, st);
    return launch_hist_dm<D, false>(p, in, ws, d_clip, st);
}

cudaError_t launch_hist(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                        const float *d_clip, cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_hist_d<1>(p, in, ws, d_clip, st);
        case 2: return launch_hist_d<2>(p, in, ws, d_clip, st);
        case 3: return launch_hist_d<3>(p, in, ws, d_clip, st);
        case 4: return launch_hist_d<4>(p, in, ws, d_clip, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
