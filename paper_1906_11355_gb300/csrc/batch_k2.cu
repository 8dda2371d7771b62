// batch_k2.cu -- the persistent batch kernel for 2-dimensional volumes.
#include "batch_impl.cuh"

namespace mclahe {

cudaError_t launch_batch_d2(const BParams &bp, bool adaptive, int C, size_t smem, cudaStream_t st) {
    return adaptive ? launch_batch_t<2, true>(bp, C, smem, st) : launch_batch_t<2, false>(bp, C, smem, st);
}

}  // namespace mclahe
