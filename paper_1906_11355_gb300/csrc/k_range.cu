// k_range.cu -- histogram ranges (Sec. III.D).
//   GHR: min and max of the whole input (the mirror padding of Sec. III.B
//        repeats voxels, so it changes neither).
//   AHR: min and max of every kernel of the padded volume, read through the
//        kernel's footprint in the original volume.
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

__global__ void __launch_bounds__(256) k_range_global(const float *__restrict__ in, int64_t n,
                                                      uint32_t *__restrict__ keys) {
    float mn = INFINITY, mx = -INFINITY;
    const int64_t nq = n >> 2;
    const float4 *in4 = reinterpret_cast<const float4 *>(in);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < nq; i += 4 * stride) {   // four loads in flight
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(in4 + i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            mn = fminf(mn, fminf(fminf(v[u].x, v[u].y), fminf(v[u].z, v[u].w)));
            mx = fmaxf(mx, fmaxf(fmaxf(v[u].x, v[u].y), fmaxf(v[u].z, v[u].w)));
        }
    }
    for (; i < nq; i += stride) {
        float4 v = __ldcs(in4 + i);
        mn = fminf(mn, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
        mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
    }
    for (int64_t t = (nq << 2) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride) {
        float v = in[t];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    block_minmax(mn, mx);
    if (threadIdx.x == 0) {
        atomicMax(&keys[0], ~float_key(mn));
        atomicMax(&keys[1], float_key(mx));
    }
}

// AHR: one CTA per (kernel, chunk of footprint rows).
template <int D>
__global__ void __launch_bounds__(256) k_range_kernels(Geom g, const float *__restrict__ in,
                                                       uint32_t *__restrict__ keys, int chunks) {
    const int64_t k = blockIdx.x / chunks;
    const int chunk = blockIdx.x - int(k * chunks);
    int kk[kMaxDim];
    {
        int64_t r = k;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            kk[j] = int(r % g.d[j].n);
            r /= g.d[j].n;
        }
    }
    int lo[kMaxDim], len[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        Foot f = footprint(g.d[j], kk[j]);
        lo[j] = f.lo;
        len[j] = f.hi - f.lo;
    }
    int R = 1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) R *= len[j];
    const int r0 = int((int64_t(R) * chunk) / chunks);
    const int r1 = int((int64_t(R) * (chunk + 1)) / chunks);
    const int L = len[D - 1];

    float mn = INFINITY, mx = -INFINITY;
    // lanes of a warp walk one row, warps take rows in turn
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    RowIter<D> it;
    it.init(len, r0 + warp, nw);
    for (int r = r0 + warp; r < r1; r += nw) {
        int64_t base = lo[D - 1];
#pragma unroll
        for (int j = 0; j < D - 1; ++j) base += int64_t(lo[j] + it.c[j]) * g.d[j].stride;
        for (int x = lane; x < L; x += 32) {
            float v = in[base + x];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        it.next();
    }
    block_minmax(mn, mx);
    if (threadIdx.x == 0 && r1 > r0) {
        atomicMax(&keys[2 * k], ~float_key(mn));
        atomicMax(&keys[2 * k + 1], float_key(mx));
    }
}

cudaError_t launch_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                         cudaStream_t st) {
    const Geom &g = p.g;
    uint32_t *keys = reinterpret_cast<uint32_t *>(ws + p.ws.keys);
    if (g.mode == MCLAHE_RANGE_GLOBAL) {
        if (g.has_range) return cudaSuccess;
        int64_t nq = (g.N >> 2) + 1;
        int blocks = int(std::min<int64_t>((nq + 255) / 256, 152 * 4));
        k_range_global<<<blocks, 256, 0, st>>>(in, g.N, keys);
        return cudaGetLastError();
    }
    const int chunks = p.t.hist_chunks;
    const unsigned grid = unsigned(g.K * chunks);
    switch (g.D) {
        case 1: k_range_kernels<1><<<grid, 256, 0, st>>>(g, in, keys, chunks); break;
        case 2: k_range_kernels<2><<<grid, 256, 0, st>>>(g, in, keys, chunks); break;
        case 3: k_range_kernels<3><<<grid, 256, 0, st>>>(g, in, keys, chunks); break;
        case 4: k_range_kernels<4><<<grid, 256, 0, st>>>(g, in, keys, chunks); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mclahe
