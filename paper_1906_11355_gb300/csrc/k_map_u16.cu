// k_map_u16.cu -- the mapping pass of one uint16 volume (intensities are the
// integers, converted to fp32 exactly; kernels in k_map_impl.cuh).
#include "k_map_impl.cuh"

namespace mclahe {

cudaError_t launch_map_u16(const mclahe_plan_s &p, const uint16_t *in, float *out,
                          const unsigned char *ws, cudaStream_t st) {
    return launch_map_any(p, in, out, ws, st);
}

}  // namespace mclahe
