// typed.cu -- mclahe_forward_typed: Algorithm 1 on volumes stored as float32,
// uint16 or uint8.  An integer voxel's intensity is the integer itself
// (converted to fp32, which is exact below 2^24), so the result equals
// mclahe_forward on the float32 volume of those values; reading 2 or 1 bytes
// per voxel instead of 4 is what the integer forms save.
#include <algorithm>
#include <cstring>

#include "mclahe_internal.cuh"

namespace mclahe {

cudaError_t launch_range_u16(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws, cudaStream_t st);
cudaError_t launch_range_u8(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws, cudaStream_t st);
cudaError_t launch_hist_u16_global(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws,
                                   const float *d_clip, cudaStream_t st);
cudaError_t launch_hist_u16_adaptive(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws,
                                     const float *d_clip, cudaStream_t st);
cudaError_t launch_hist_u8_global(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws,
                                  const float *d_clip, cudaStream_t st);
cudaError_t launch_hist_u8_adaptive(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws,
                                    const float *d_clip, cudaStream_t st);
cudaError_t launch_hist_staged_u16(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws,
                                   const float *d_clip, cudaStream_t st);
cudaError_t launch_hist_staged_u8(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws,
                                  const float *d_clip, cudaStream_t st);
cudaError_t launch_map_u16(const mclahe_plan_s &p, const uint16_t *in, float *out,
                           const unsigned char *ws, cudaStream_t st);
cudaError_t launch_map_u8(const mclahe_plan_s &p, const uint8_t *in, float *out,
                          const unsigned char *ws, cudaStream_t st);

namespace {

cudaError_t range_of(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws, cudaStream_t st) {
    return launch_range_u16(p, in, ws, st);
}
cudaError_t range_of(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws, cudaStream_t st) {
    return launch_range_u8(p, in, ws, st);
}
// The plan's shapes for the ring walk of an integer volume: the cluster form
// (a flat plan runs as one-CTA clusters with the same groups) with as many of
// the plan's lane copies as let the row ring fit; copies change the speed, never
// the counts.
mclahe_plan_s ring_plan(const mclahe_plan_s &p) {
    mclahe_plan_s q = p;
    q.t.range_pass = 0;   // integer volumes sweep each footprint's range inside the pass
    while (q.t.hist_copies > 1 &&
           hist_smem_bytes(q.g, q.t.hist_copies, q.t.hist_group, 1, q.t.hist_threads) > 220 * 1024)
        q.t.hist_copies >>= 1;
    return q;
}
cudaError_t hist_of(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws, const float *c,
                    cudaStream_t st) {
    if (p.t.hist_walk == 3 && hist_staged_fits(p.g, p.t.hist_copies, p.t.hist_chunks, nullptr))
        return launch_hist_staged_u16(p, in, ws, c, st);
    const mclahe_plan_s q = ring_plan(p);
    return p.g.mode == MCLAHE_RANGE_ADAPTIVE ? launch_hist_u16_adaptive(q, in, ws, c, st)
                                             : launch_hist_u16_global(q, in, ws, c, st);
}
cudaError_t hist_of(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws, const float *c,
                    cudaStream_t st) {
    if (p.t.hist_walk == 3 && hist_staged_fits(p.g, p.t.hist_copies, p.t.hist_chunks, nullptr))
        return launch_hist_staged_u8(p, in, ws, c, st);
    const mclahe_plan_s q = ring_plan(p);
    return p.g.mode == MCLAHE_RANGE_ADAPTIVE ? launch_hist_u8_adaptive(q, in, ws, c, st)
                                             : launch_hist_u8_global(q, in, ws, c, st);
}
cudaError_t map_of(const mclahe_plan_s &p, const uint16_t *in, float *out, const unsigned char *ws,
                   cudaStream_t st) {
    return launch_map_u16(p, in, out, ws, st);
}
cudaError_t map_of(const mclahe_plan_s &p, const uint8_t *in, float *out, const unsigned char *ws,
                   cudaStream_t st) {
    return launch_map_u8(p, in, out, ws, st);
}

// The passes of mclahe_forward for an integer volume: clear the global range
// keys, the global range (unless given), the histogram pass in its cluster
// form (a flat plan runs as one-CTA clusters with the same groups and copies)
// or the staged walk, and the mapping pass (per-thread walks; the TMA tile
// walk maps float32 tiles in place).
template <typename T>
mclahe_status forward_int(const mclahe_plan_s &p, const T *in, float *out, unsigned char *ws,
                          const float *d_clip, cudaStream_t st) {
    if (p.g.mode == MCLAHE_RANGE_GLOBAL && !p.g.has_range) {
        if (cudaMemsetAsync(ws + p.ws.keys, 0, 2 * sizeof(uint32_t), st) != cudaSuccess)
            return MCLAHE_ERR_CUDA;
        if (range_of(p, in, ws, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    }
    if (hist_of(p, in, ws, d_clip, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    // the per-cell mapping grid: a flat plan's shares per cell would each restage
    // the corner tables, so at least about two CTAs per SM in all, and chunks of
    // at most 64 Ki voxels of a cell (large 4-D cells: 4 chunks per cell measured
    // 5 % faster than 1 on 128x128x256x32 uint8; 3-D unchanged)
    mclahe_plan_s q = p;
    if (q.t.map_flat || q.t.map_tma) {
        const int64_t cells = n_cells(q.g);
        int64_t cell_vox = 1;
        for (int j = 0; j < q.g.D; ++j) cell_vox *= q.g.d[j].b;
        q.t.map_chunks = int(std::min<int64_t>(
            64, std::max<int64_t>({int64_t(1), (2 * int64_t(device_sms()) + cells - 1) / cells,
                                   (cell_vox + 65535) / 65536})));
        q.t.map_flat = 0;
        q.t.map_tma = 0;
    }
    if (map_of(q, in, out, ws, st) != cudaSuccess) return MCLAHE_ERR_CUDA;
    return MCLAHE_OK;
}

}  // namespace

}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_forward_typed(mclahe_plan_t p, mclahe_dtype dtype, const void *d_in,
                                              float *d_out, void *d_ws, size_t ws_bytes,
                                              const float *d_clip, mclahe_stream_t stream) {
    const mclahe_status s = check_forward_args(p, d_in, d_out, d_ws, ws_bytes);
    if (s != MCLAHE_OK) return s;
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (dtype) {
        case MCLAHE_F32: return forward_impl(*p, static_cast<const float *>(d_in), d_out, ws, d_clip, st);
        case MCLAHE_U16: return forward_int(*p, static_cast<const uint16_t *>(d_in), d_out, ws, d_clip, st);
        case MCLAHE_U8: return forward_int(*p, static_cast<const uint8_t *>(d_in), d_out, ws, d_clip, st);
        default: return MCLAHE_ERR_INVALID_ARG;
    }
}
