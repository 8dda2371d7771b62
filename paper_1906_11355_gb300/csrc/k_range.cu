// k_range.cu -- histogram ranges (Sec. III.D).
//   GHR: min and max of the whole input (the mirror padding of Sec. III.B
//        repeats voxels, so it changes neither).
//   (The per-kernel ranges of AHR are computed inside the histogram pass.)
// Results are order-preserving uint32 keys combined with atomicMax; the min
// is stored complemented so that every key starts at 0 (one memset).
#include <algorithm>

#include "mclahe_internal.cuh"

namespace mclahe {

__device__ __forceinline__ void warp_minmax(float &mn, float &mx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
}

// Block-wide min/max; the result is valid in thread 0.
__device__ __forceinline__ void block_minmax(float &mn, float &mx) {
    __shared__ float smn[32], smx[32];
    warp_minmax(mn, mx);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        smn[w] = mn;
        smx[w] = mx;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        mn = l < nw ? smn[l] : INFINITY;
        mx = l < nw ? smx[l] : -INFINITY;
        warp_minmax(mn, mx);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_range_global(const T *__restrict__ in, int64_t n,
                                                      uint32_t *__restrict__ keys) {
    float mn = INFINITY, mx = -INFINITY;
    const int64_t nq = n >> 2;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < nq; i += 4 * stride) {   // four loads in flight
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ldq(in + 4 * (i + u * stride), true);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            mn = fminf(mn, fminf(fminf(v[u].x, v[u].y), fminf(v[u].z, v[u].w)));
            mx = fmaxf(mx, fmaxf(fmaxf(v[u].x, v[u].y), fmaxf(v[u].z, v[u].w)));
        }
    }
    for (; i < nq; i += stride) {
        const float4 v = ldq(in + 4 * i, true);
        mn = fminf(mn, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
        mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
    }
    for (int64_t t = (nq << 2) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride) {
        const float v = ld1(in + t);
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    block_minmax(mn, mx);
    if (threadIdx.x == 0) {
        atomicMax(&keys[0], ~float_key(mn));
        atomicMax(&keys[1], float_key(mx));
    }
}

template <typename T>
static cudaError_t launch_range_t(const mclahe_plan_s &p, const T *in, unsigned char *ws,
                                  cudaStream_t st) {
    const Geom &g = p.g;
    uint32_t *keys = reinterpret_cast<uint32_t *>(ws + p.ws.keys);
    if (g.mode == MCLAHE_RANGE_GLOBAL) {
        if (g.has_range) return cudaSuccess;
        int64_t nq = (g.N >> 2) + 1;
        int blocks = int(std::min<int64_t>((nq + 255) / 256, int64_t(device_sms()) * 4));
        k_range_global<T><<<blocks, 256, 0, st>>>(in, g.N, keys);
        return cudaGetLastError();
    }
    return cudaSuccess;   // the adaptive range is fused into the histogram pass
}

cudaError_t launch_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                         cudaStream_t st) {
    return launch_range_t(p, in, ws, st);
}

// min/max of n contiguous values of a buffer, added to the global range keys
// (the slabs of mclahe_forward_chunked)
cudaError_t launch_range_buffer(const float *buf, int64_t n, uint32_t *keys, cudaStream_t st) {
    const int64_t nq = (n >> 2) + 1;
    const int blocks = int(std::min<int64_t>((nq + 255) / 256, int64_t(device_sms()) * 4));
    k_range_global<float><<<blocks, 256, 0, st>>>(buf, n, keys);
    return cudaGetLastError();
}
cudaError_t launch_range_u16(const mclahe_plan_s &p, const uint16_t *in, unsigned char *ws,
                             cudaStream_t st) {
    return launch_range_t(p, in, ws, st);
}
cudaError_t launch_range_u8(const mclahe_plan_s &p, const uint8_t *in, unsigned char *ws,
                            cudaStream_t st) {
    return launch_range_t(p, in, ws, st);
}

}  // namespace mclahe
