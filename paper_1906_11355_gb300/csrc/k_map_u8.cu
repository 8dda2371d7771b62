// k_map_u8.cu -- the mapping pass of one uint8 volume (intensities are the
// integers, converted to fp32 exactly; kernels in k_map_impl.cuh).
#include "k_map_impl.cuh"

namespace mclahe {

cudaError_t launch_map_u8(const mclahe_plan_s &p, const uint8_t *in, float *out,
                          const unsigned char *ws, cudaStream_t st) {
    return launch_map_any(p, in, out, ws, st);
}

}  // namespace mclahe
