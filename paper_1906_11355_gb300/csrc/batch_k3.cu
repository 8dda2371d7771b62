// batch_k3.cu -- the persistent batch kernel for 3-dimensional volumes.
#include "batch_impl.cuh"

namespace mclahe {

cudaError_t launch_batch_d3(const BParams &bp, bool adaptive, int C, size_t smem, cudaStream_t st) {
    return adaptive ? launch_batch_t<3, true>(bp, C, smem, st) : launch_batch_t<3, false>(bp, C, smem, st);
}

}  // namespace mclahe
