// k_hist_u16a.cu -- the histogram pass (cluster form, cp.async row ring) of one
// uint16 volume with a per-kernel adaptive range: intensities are the integers,
// converted to fp32 exactly (kernels in k_hist_impl.cuh).
#include "k_hist_impl.cuh"

namespace mclahe {

cudaError_t launch_hist_u16_adaptive(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws,
                          const float *d_clip, cudaStream_t st) {
    HistTmaArgs none;
    std::memset(&none.map, 0, sizeof(none.map));
    auto go = [&](auto dtag) -> cudaError_t {
        constexpr int D = decltype(dtag)::value;
        return launch_hist_cluster<D, true, kHistRing, uint16_t>(p, in, ws, d_clip, st, none);
    };
    switch (p.g.D) {
        case 1: return go(std::integral_constant<int, 1>{});
        case 2: return go(std::integral_constant<int, 2>{});
        case 3: return go(std::integral_constant<int, 3>{});
        case 4: return go(std::integral_constant<int, 4>{});
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
