// metrics.cu -- mclahe_metrics: the contrast metrics the paper compares its
// results with (Sec. II; Tables I-II of Sec. IV): mean, standard deviation and
// Shannon entropy of a volume normalised to [0, 1] by its own min and max,
// and its mean squared error and PSNR against a reference volume normalised
// the same way.  PSNR = 10 log10(peak^2 / MSE) with peak = 2^23 (the peak the
// tables' PSNR and MSE columns imply); the entropy is over a 256-bin histogram
// binned by the fp32 quantiser of the histogram pass.
// Three launches:
//   k_met_range  min and max of both volumes (order-preserving keys);
//   k_met_sums   per CTA: sum x^, sum x^2, sum (x^ - r^)^2 (compensated fp32 per
//                thread, fp64 per CTA in a fixed tree) and the histogram of x
//                (lane copies in shared memory, then 64-bit global atomics);
//   k_met_final  one CTA: the partials in a fixed order, the metrics.
// Deterministic for a given volume size (the grid depends only on it).
#include <algorithm>
#include <cmath>

#include "mclahe_internal.cuh"

namespace mclahe {

constexpr int kMetBins = 256;
constexpr int kMetCopies = 8;

__device__ __forceinline__ void met_minmax(float &mn, float &mx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
}

__global__ void __launch_bounds__(256) k_met_range(const float *__restrict__ x, const float *__restrict__ r,
                                                   int64_t n, uint32_t *__restrict__ keys) {
    float mn = INFINITY, mx = -INFINITY, rn = INFINITY, rx = -INFINITY;
    const int64_t nq = n >> 2, stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nq; i += stride) {
        const float4 v = ldq(x + 4 * i, true);
        mn = fminf(mn, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
        mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
        if (r) {
            const float4 w = ldq(r + 4 * i, true);
            rn = fminf(rn, fminf(fminf(w.x, w.y), fminf(w.z, w.w)));
            rx = fmaxf(rx, fmaxf(fmaxf(w.x, w.y), fmaxf(w.z, w.w)));
        }
    }
    for (int64_t t = (nq << 2) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride) {
        mn = fminf(mn, x[t]);
        mx = fmaxf(mx, x[t]);
        if (r) {
            rn = fminf(rn, r[t]);
            rx = fmaxf(rx, r[t]);
        }
    }
    met_minmax(mn, mx);
    met_minmax(rn, rx);
    if ((threadIdx.x & 31) == 0 && mn <= mx) {
        atomicMax(&keys[0], ~float_key(mn));
        atomicMax(&keys[1], float_key(mx));
        if (r) {
            atomicMax(&keys[2], ~float_key(rn));
            atomicMax(&keys[3], float_key(rx));
        }
    }
}

// normalisation x^ = (x - lo) * inv, inv = 1 / (hi - lo) (0 for a constant volume)
struct MetNorm {
    float lo, inv;
};
__device__ __forceinline__ MetNorm met_norm(uint32_t kmin, uint32_t kmax) {
    float lo, hi;
    keys_to_range(kmin, kmax, lo, hi);
    return MetNorm{lo, hi > lo ? 1.0f / (hi - lo) : 0.0f};
}

// Deterministic block sum in double; valid in thread 0.
__device__ __forceinline__ double met_block_sum(double v, double *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += s_w[w];
    return s;
}

struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float t) {
        const float y = __fsub_rn(t, c);
        const float u = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(u, s), y);
        s = u;
    }
    __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

__global__ void __launch_bounds__(256) k_met_sums(const float *__restrict__ x, const float *__restrict__ r,
                                                  int64_t n, const uint32_t *__restrict__ keys,
                                                  double *__restrict__ partial,
                                                  unsigned long long *__restrict__ hist) {
    __shared__ uint32_t sh[kMetBins * kMetCopies + kMetCopies];   // [bin 0..256][copy]
    __shared__ double s_w[32];
    for (int i = threadIdx.x; i < (kMetBins + 1) * kMetCopies; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const MetNorm nx = met_norm(__ldcg(keys), __ldcg(keys + 1));
    const MetNorm nr = r ? met_norm(__ldcg(keys + 2), __ldcg(keys + 3)) : MetNorm{0.0f, 0.0f};
    // bins: the histogram pass's exact quantiser with 256 bins over [lo, hi]
    float hlo, hhi;
    keys_to_range(__ldcg(keys), __ldcg(keys + 1), hlo, hhi);
    const float sc = range_scale(hlo, hhi, kMetBins);
    constexpr float qkf = float(kMetBins), iqk = 1.0f / float(kMetBins);
    const uint32_t base = uint32_t(__cvta_generic_to_shared(sh)) +
                          4u * uint32_t(threadIdx.x & (kMetCopies - 1)) - kBinBias * 4u * kMetCopies;
    Kahan s1, s2, s3;
    auto one = [&](float v, float w, bool has_r) {
        const float a = __fmul_rn(__fsub_rn(v, nx.lo), nx.inv);
        s1.add(a);
        s2.add(__fmul_rn(a, a));
        if (has_r) {
            const float d = __fsub_rn(a, __fmul_rn(__fsub_rn(w, nr.lo), nr.inv));
            s3.add(__fmul_rn(d, d));
        }
        const uint32_t b = qbits1(v, -hlo, sc, iqk, qkf);
        red_shared_add(b * 4u * kMetCopies + base, 1u);
    };
    const int64_t nq = n >> 2, stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nq; i += stride) {
        const float4 v = ldq(x + 4 * i, true);
        const float4 w = r ? ldq(r + 4 * i, true) : make_float4(0.f, 0.f, 0.f, 0.f);
        one(v.x, w.x, r != nullptr);
        one(v.y, w.y, r != nullptr);
        one(v.z, w.z, r != nullptr);
        one(v.w, w.w, r != nullptr);
    }
    for (int64_t t = (nq << 2) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride)
        one(x[t], r ? r[t] : 0.0f, r != nullptr);
    const double a1 = met_block_sum(s1.value(), s_w);
    const double a2 = met_block_sum(s2.value(), s_w);
    const double a3 = met_block_sum(s3.value(), s_w);
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x] = a1;
        partial[3 * blockIdx.x + 1] = a2;
        partial[3 * blockIdx.x + 2] = a3;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kMetBins; j += blockDim.x) {
        uint32_t c = 0;
        for (int k = 0; k < kMetCopies; ++k) c += sh[j * kMetCopies + k];
        if (j == kMetBins - 1)   // index 256 (x = hi) is the last bin
            for (int k = 0; k < kMetCopies; ++k) c += sh[kMetBins * kMetCopies + k];
        if (c) atomicAdd(&hist[j], static_cast<unsigned long long>(c));
    }
}

__global__ void __launch_bounds__(256) k_met_final(const double *__restrict__ partial, int nblocks,
                                                   const unsigned long long *__restrict__ hist,
                                                   int64_t n, int has_ref, double *__restrict__ out) {
    __shared__ double s_w[32];
    double a1 = 0.0, a2 = 0.0, a3 = 0.0, e = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        a1 += partial[3 * b];
        a2 += partial[3 * b + 1];
        a3 += partial[3 * b + 2];
    }
    const double dn = double(n);
    for (int j = threadIdx.x; j < kMetBins; j += blockDim.x) {
        const double p = double(hist[j]) / dn;
        if (p > 0.0) e -= p * log2(p);
    }
    a1 = met_block_sum(a1, s_w);
    a2 = met_block_sum(a2, s_w);
    a3 = met_block_sum(a3, s_w);
    e = met_block_sum(e, s_w);
    if (threadIdx.x == 0) {
        const double mean = a1 / dn;
        const double var = fmax(a2 / dn - mean * mean, 0.0);
        out[0] = mean;
        out[1] = sqrt(var);
        out[2] = e;
        const double mse = a3 / dn;
        out[3] = has_ref ? mse : nan("");
        const double peak = 8388608.0;   // 2^23
        out[4] = has_ref ? (mse > 0.0 ? 10.0 * log10(peak * peak / mse) : INFINITY) : nan("");
    }
}

static int met_grid(int64_t n) {
    const int64_t nq = (n >> 2) + 1;
    return int(std::max<int64_t>(1, std::min<int64_t>((nq + 255) / 256, int64_t(device_sms()) * 4)));
}

size_t met_ws_bytes(int64_t n) {
    return 256 + sizeof(unsigned long long) * kMetBins + sizeof(double) * 3 * size_t(met_grid(n));
}

}  // namespace mclahe

using namespace mclahe;

extern "C" size_t mclahe_metrics_workspace_bytes(int64_t n) { return n >= 1 ? met_ws_bytes(n) : 0; }

extern "C" mclahe_status mclahe_metrics(const float *d_x, const float *d_ref, int64_t n, void *d_ws,
                                        size_t ws_bytes, double *d_out, mclahe_stream_t stream) {
    if (!d_x || !d_out || n < 1 || d_x == d_ref) return MCLAHE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_x) & 15) || (reinterpret_cast<uintptr_t>(d_ref) & 15) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7))
        return MCLAHE_ERR_INVALID_ARG;
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255) || ws_bytes < met_ws_bytes(n))
        return MCLAHE_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_ws);
    uint32_t *keys = reinterpret_cast<uint32_t *>(ws);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(ws + 256);
    double *partial = reinterpret_cast<double *>(ws + 256 + sizeof(unsigned long long) * kMetBins);
    if (cudaMemsetAsync(ws, 0, 256 + sizeof(unsigned long long) * kMetBins, st) != cudaSuccess)
        return MCLAHE_ERR_CUDA;
    const int grid = met_grid(n);
    k_met_range<<<grid, 256, 0, st>>>(d_x, d_ref, n, keys);
    k_met_sums<<<grid, 256, 0, st>>>(d_x, d_ref, n, keys, partial, hist);
    k_met_final<<<1, 256, 0, st>>>(partial, grid, hist, n, d_ref ? 1 : 0, d_out);
    return cudaGetLastError() == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}
