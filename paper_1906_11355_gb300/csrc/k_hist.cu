// k_hist.cu -- launcher of the histogram pass of one volume: one thread-block
// cluster per group of kernels along the last dimension builds their
// histograms and mapping tables (Algorithm 1; the work of a cluster is in
// hist_impl.cuh).
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
    hist_group<D, ADAPTIVE>(g, in, keys, d_clip, hist, lut, lo_out, scale_out, item, G, R, sh);
}

size_t hist_smem_bytes(const Geom &g, int copies, int group) {
    return hist_smem_words(g.P, copies, group) * sizeof(uint32_t);
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

template <int D>
static cudaError_t launch_hist_d(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                 const float *d_clip, cudaStream_t st) {
    if (p.g.mode == MCLAHE_RANGE_ADAPTIVE) return launch_hist_dm<D, true>(p, in, ws, d_clip, st);
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
