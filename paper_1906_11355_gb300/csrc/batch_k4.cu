// batch_k4.cu -- the persistent batch kernel for 4-dimensional volumes.
#include "batch_impl.cuh"

namespace mclahe {

cudaError_t launch_batch_d4(const BParams &bp, bool adaptive, int C, size_t smem, cudaStream_t st) {
    return adaptive ? launch_batch_t<4, true>(bp, C, smem, st) : launch_batch_t<4, false>(bp, C, smem, st);
}

}  // namespace mclahe
