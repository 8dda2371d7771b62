// k_hist_tma.cu -- launches of the histogram pass with TMA box tiles (the
// kernels are in k_hist_impl.cuh; shapes and the box in k_hist.cu).
#include <type_traits>

#include "k_hist_impl.cuh"

namespace mclahe {

cudaError_t launch_hist_tma(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                            const float *d_clip, cudaStream_t st, bool range, int bx, int by) {
    HistTmaArgs ta;
    ta.bx = bx;
    ta.by = by;
    int box[4] = {bx, by, 1, 1};
    const cudaError_t e = encode_tensor_map(&ta.map, in, p.g, box);
    if (e != cudaSuccess) return e;
    return launch_hist_walk<kHistTma>(p, in, ws, d_clip, st, ta, range);
}

}  // namespace mclahe
