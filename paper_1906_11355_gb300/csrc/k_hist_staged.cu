// k_hist_staged.cu -- launches of the histogram pass with every kernel's
// footprint staged in shared memory (one cluster per kernel; the work is in
// hist_staged.cuh).  2- to 4-D volumes whose rows start on 16-byte boundaries
// (last extent a multiple of 4), one kernel per work item, the cluster form.
#include <algorithm>

#include "hist_staged.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE, typename T>
__global__ void __launch_bounds__(256, 2)
    k_hist_staged(Geom g, const T *__restrict__ in, const uint32_t *__restrict__ keys,
                  const float *__restrict__ d_clip, uint32_t *__restrict__ hist,
                  float *__restrict__ lut, float *__restrict__ lo_out, float *__restrict__ scale_out,
                  int R) {
    extern __shared__ __align__(128) uint32_t sh[];
    const int64_t k = blockIdx.x / cg::this_cluster().num_blocks();
    hist_staged<D, ADAPTIVE, T>(g, in, keys, d_clip, hist, lut, lo_out, scale_out, k, R, sh);
}

// The widest footprint box over all kernels: rows (the product over all dims
// but the last of the largest extent) and quads per row (from the row's
// 16-byte boundary).
static StagedShape staged_shape(const Geom &g) {
    StagedShape s{1, 1};
    for (int j = 0; j < g.D; ++j) {
        int ext = 1, q = 1;
        for (int k = 0; k < g.d[j].n; ++k) {
            const Foot f = footprint(g.d[j], k);
            ext = std::max(ext, f.hi - f.lo);
            q = std::max(q, ((f.lo & 3) + (f.hi - f.lo) + 3) >> 2);
        }
        if (j + 1 < g.D) s.rows_max *= ext;
        else s.Q = q;
    }
    return s;
}

bool hist_staged_fits(const Geom &g, int R, int C, size_t *bytes) {
    if (g.D < 2 || g.d[g.D - 1].s % 4 != 0) return false;
    const StagedShape sh = staged_shape(g);
    if (sh.Q > 32 * kStagedQmax) return false;   // rows of at most kStagedQmax slots per lane
    const size_t b = staged_smem_bytes(g.P, R, C, sh);
    if (bytes) *bytes = b;
    return b <= 220 * 1024;
}

template <int D, bool ADAPTIVE, typename T>
static cudaError_t launch_staged_t(const mclahe_plan_s &p, const T *in, unsigned char *ws,
                                   const float *d_clip, cudaStream_t st, size_t smem) {
    auto kern = k_hist_staged<D, ADAPTIVE, T>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    const int C = p.t.hist_chunks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(p.g.K * C));
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
    return cudaLaunchKernelEx(&cfg, kern, p.g, in, reinterpret_cast<const uint32_t *>(ws + p.ws.keys),
                              d_clip, reinterpret_cast<uint32_t *>(ws + p.ws.hist),
                              reinterpret_cast<float *>(ws + p.ws.lut),
                              reinterpret_cast<float *>(ws + p.ws.lo),
                              reinterpret_cast<float *>(ws + p.ws.scale), p.t.hist_copies);
}

template <typename T>
static cudaError_t launch_staged_any(const mclahe_plan_s &p, const T *in, unsigned char *ws,
                                     const float *d_clip, cudaStream_t st) {
    size_t smem = 0;
    if (!hist_staged_fits(p.g, p.t.hist_copies, p.t.hist_chunks, &smem)) return cudaErrorInvalidValue;
    const bool a = p.g.mode == MCLAHE_RANGE_ADAPTIVE;
    switch (p.g.D) {
        case 2: return a ? launch_staged_t<2, true, T>(p, in, ws, d_clip, st, smem)
                         : launch_staged_t<2, false, T>(p, in, ws, d_clip, st, smem);
        case 3: return a ? launch_staged_t<3, true, T>(p, in, ws, d_clip, st, smem)
                         : launch_staged_t<3, false, T>(p, in, ws, d_clip, st, smem);
        case 4: return a ? launch_staged_t<4, true, T>(p, in, ws, d_clip, st, smem)
                         : launch_staged_t<4, false, T>(p, in, ws, d_clip, st, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_hist_staged(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                               const float *d_clip, cudaStream_t st) {
    return launch_staged_any(p, in, ws, d_clip, st);
}
cudaError_t launch_hist_staged_u16(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws,
                                   const float *d_clip, cudaStream_t st) {
    return launch_staged_any(p, in, ws, d_clip, st);
}
cudaError_t launch_hist_staged_u8(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws,
                                  const float *d_clip, cudaStream_t st) {
    return launch_staged_any(p, in, ws, d_clip, st);
}

}  // namespace mclahe
