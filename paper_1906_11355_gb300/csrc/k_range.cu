// k_range.cu -- histogram ranges (Sec. III.D).
//   GHR: min and max of the whole input (the mirror padding of Sec. III.B
//        repeats voxels, so it changes neither).
//   AHR: min and max of every kernel's padded footprint, either inside the
//        histogram pass (a sweep of each footprint before binning it) or, for
//        plans with range_pass set, by k_range_kernels: one streaming sweep
//        over the volume in memory order, before the histogram pass.
// Results are order-preserving uint32 keys combined with atomicMax; the min
// is stored complemented so that every key starts at 0 (one memset).
#include <algorithm>

#include "hist_impl.cuh"

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

// ---------------------------------------------------------------------------
// Per-kernel ranges in one sweep (Sec. III.D with the padding of Sec. III.B):
// kernel k's range is the min and max over the voxels that have a mirror image
// in its padded box, i.e. over the product of its footprint intervals.  The
// volume is read once, row by row in memory order (rows along the last
// dimension, 128-bit loads through L2, where the histogram pass then finds
// them): CTA b takes rows [R b / grid, R (b + 1) / grid), warp w of it every
// nw-th of those rows.  A row's outer coordinates name the kernels of the
// outer dimensions that hold it (one to three per dimension); along the row,
// the lanes of a warp take consecutive quads, the quads of one kernel are
// reduced across the warp (one leader per kernel) and added to the CTA's keys
// in shared memory, and the CTA adds its keys to the global ones at the end.
// Min and max are exact, so the keys equal those of the in-pass sweep.
// Needs a row length that is a multiple of 4, and 2 K keys plus one word per
// quad position of a row in shared memory.
// ---------------------------------------------------------------------------
constexpr int kRangeQuadsPerLane = 4;   // quads in flight per lane (rows of 512 floats at once)

template <int D>
__global__ void __launch_bounds__(256) k_range_kernels(Geom g, const float *__restrict__ in,
                                                       uint32_t *__restrict__ kkeys, int64_t rows) {
    extern __shared__ uint32_t s_k[];   // [2 K]: ~key(min), key(max) of every kernel,
                                        // then [Q]: the kernel of each quad position
    const int K = int(g.K);
    const Dim &dl = g.d[D - 1];
    const int Q = dl.s >> 2;   // quads per row
    int *s_kx = reinterpret_cast<int *>(s_k + 2 * K);
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) s_k[i] = 0u;
    // every row has the same quad positions: the kernel along the row that
    // holds all four voxels of quad q, or -1 where they differ or a voxel has
    // several (a footprint edge, a mirror image)
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        const Targets t0 = last_targets(dl, 4 * q, 0, dl.n);
        const Targets t3 = last_targets(dl, 4 * q + 3, 0, dl.n);
        s_kx[q] = (t0.n == 1 && t3.n == 1 && t0.kg[0] == t3.kg[0]) ? t0.kg[0] : -1;
    }
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = int(threadIdx.x & 31), warp = int(threadIdx.x >> 5), nw = int(blockDim.x >> 5);
    const int64_t r0 = rows * blockIdx.x / gridDim.x, r1 = rows * (blockIdx.x + 1) / gridDim.x;
    int kst[kMaxDim];          // flat kernel index strides
    {
        int st = 1;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            kst[j] = st;
            st *= g.d[j].n;
        }
    }
    auto add = [&](int k, uint32_t kmn, uint32_t kmx) {
        atomicMax(&s_k[2 * k], kmn);
        atomicMax(&s_k[2 * k + 1], kmx);
    };
    for (int64_t r = r0 + warp; r < r1; r += nw) {
        // the kernels along the outer dimensions that hold this row: flat
        // index bases of their combinations (at most 3^(D-1))
        int base[27];
        int nbase = 1;
        base[0] = 0;
        {
            int64_t rest = r;
            int c[kMaxDim];
#pragma unroll
            for (int j = D - 2; j >= 0; --j) {
                c[j] = int(rest % g.d[j].s);
                rest /= g.d[j].s;
            }
#pragma unroll
            for (int j = 0; j < D - 1; ++j) {
                const Targets t = last_targets(g.d[j], c[j], 0, g.d[j].n);
                const int nb0 = nbase;
                for (int i = 1; i < t.n; ++i)
                    for (int b = 0; b < nb0; ++b) base[i * nb0 + b] = base[b] + t.kg[i] * kst[j];
                for (int b = 0; b < nb0; ++b) base[b] += t.kg[0] * kst[j];
                nbase = nb0 * t.n;
            }
        }
        const float *row = in + r * int64_t(dl.s);
        for (int q0 = 0; q0 < Q; q0 += 32 * kRangeQuadsPerLane) {
            float4 v[kRangeQuadsPerLane];
#pragma unroll
            for (int u = 0; u < kRangeQuadsPerLane; ++u) {
                const int q = q0 + u * 32 + lane;
                v[u] = q < Q ? __ldcg(reinterpret_cast<const float4 *>(row) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kRangeQuadsPerLane; ++u) {
                const int q = q0 + u * 32 + lane;
                if (q0 + u * 32 >= Q) break;   // uniform across the warp
                const bool valid = q < Q;
                // the quad's kernel along the row when all four voxels share one
                const int kx = valid ? s_kx[q] : -1;
                if (valid && kx < 0) {
                    // the quad crosses a footprint edge: voxel by voxel
                    const float vals[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (vals[e] != vals[e]) continue;   // NaN: no effect on min/max
                        const Targets te = last_targets(dl, 4 * q + e, 0, dl.n);
                        for (int i = 0; i < te.n; ++i)
                            for (int b = 0; b < nbase; ++b)
                                add(base[b] + te.kg[i], ~float_key(vals[e]), float_key(vals[e]));
                    }
                }
                float mn = fminf(fminf(v[u].x, v[u].y), fminf(v[u].z, v[u].w));
                float mx = fmaxf(fmaxf(v[u].x, v[u].y), fmaxf(v[u].z, v[u].w));
                const bool has = valid && kx >= 0 && mn <= mx;
                const uint32_t kmn = has ? ~float_key(mn) : 0u, kmx = has ? float_key(mx) : 0u;
                unsigned pend = __ballot_sync(full, has);
                while (pend) {
                    const int leader = __ffs(pend) - 1;
                    const int t = __shfl_sync(full, kx, leader);
                    const bool mine = has && kx == t;
                    pend &= ~__ballot_sync(full, mine);
                    const uint32_t a = __reduce_max_sync(full, mine ? kmn : 0u);
                    const uint32_t b = __reduce_max_sync(full, mine ? kmx : 0u);
                    if (lane == leader)
                        for (int i = 0; i < nbase; ++i) add(base[i] + t, a, b);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x)
        if (s_k[i]) atomicMax(&kkeys[i], s_k[i]);
}

static size_t range_kernels_smem(const Geom &g) {
    return size_t(g.K) * 8 + size_t(g.d[g.D - 1].s >> 2) * 4;
}

bool range_pass_fits(const Geom &g) {
    return g.mode == MCLAHE_RANGE_ADAPTIVE && g.D >= 1 && (g.d[g.D - 1].s & 3) == 0 &&
           range_kernels_smem(g) <= 48 * 1024;
}

// the per-kernel keys (ws keys + 2), cleared by the clear pass
cudaError_t launch_range_kernels(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                 cudaStream_t st) {
    const Geom &g = p.g;
    if (!range_pass_fits(g)) return cudaErrorInvalidValue;
    uint32_t *kkeys = reinterpret_cast<uint32_t *>(ws + p.ws.keys) + 2;
    const int64_t rows = g.N / g.d[g.D - 1].s;
    const size_t smem = range_kernels_smem(g);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, int64_t(device_sms()) * 4)));
    switch (g.D) {
#define MCLAHE_RK(DD)                                                                          \
    case DD:                                                                                   \
        k_range_kernels<DD><<<grid, 256, smem, st>>>(g, in, kkeys, rows);                      \
        break;
        MCLAHE_RK(1)
        MCLAHE_RK(2)
        MCLAHE_RK(3)
        MCLAHE_RK(4)
#undef MCLAHE_RK
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
