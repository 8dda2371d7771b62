// k_hist_lsu.cu -- launches of the histogram pass with per-thread 128-bit
// loads into registers (no row buffer in shared memory, so more CTAs fit on an
// SM when the histograms are large); kernels in k_hist_impl.cuh.
#include <cstring>
#include <type_traits>

#include "k_hist_impl.cuh"

namespace mclahe {

cudaError_t launch_hist_lsu(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                            const float *d_clip, cudaStream_t st, bool range) {
    HistTmaArgs none;
    std::memset(&none.map, 0, sizeof(none.map));
    return launch_hist_walk<kHistLsu>(p, in, ws, d_clip, st, none, range);
}

}  // namespace mclahe
