// tma_host.cu -- tensor maps (TMA descriptors) of float32 volumes, encoded
// with the CUDA driver API's cuTensorMapEncodeTiled, reached through the
// runtime's entry-point lookup (the library does not link libcuda).
#include "mclahe_internal.cuh"

namespace mclahe {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Dims innermost first (dim i of the map = volume dim D-1-i), byte strides
// of the outer dims, the tile box, no swizzle, zero fill out of bounds.
cudaError_t encode_tensor_map(CUtensorMap *m, const float *ptr, const Geom &g, const int *box) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const int D = g.D;
    cuuint64_t dims[4], strides[3];
    cuuint32_t bx[4], es[4] = {1, 1, 1, 1};
    for (int i = 0; i < D; ++i) {
        dims[i] = cuuint64_t(g.d[D - 1 - i].s);
        bx[i] = cuuint32_t(box[i]);
    }
    for (int i = 1; i < D; ++i) strides[i - 1] = cuuint64_t(g.d[D - 1 - i].stride) * sizeof(float);
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, cuuint32_t(D), const_cast<float *>(ptr),
                           dims, strides, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace mclahe
