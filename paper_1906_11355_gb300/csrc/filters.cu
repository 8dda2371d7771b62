// filters.cu -- the pre-filters the paper applies before MCLAHE: a separable
// Gaussian (Sec. IV.A, photoemission data) and a median filter (Sec. IV.B,
// fluorescence data, window (2, 2, 2, 1)).  Readings of what the paper leaves
// open (scipy.ndimage's conventions):
//   boundary  the edge-inclusive mirror of MCLAHE's padding (Sec. III.B),
//             reflected as often as needed;
//   Gaussian  dimension by dimension (0 first), radius r = floor(4 sigma +
//             0.5), weights exp(-k^2 / (2 sigma^2)) normalised in double and
//             rounded to fp32 (mclahe_gaussian_weights); each output is the fp32
//             sum over the taps k = -r..r in that order of fp32(w_k * x), every
//             product and sum rounded to nearest (no contraction), so that the
//             result is one exact function of the input;
//   median    window [x - floor(k/2), x - floor(k/2) + k - 1] per dimension; the
//             value of rank floor(n/2) (0-based) of the window's n values.
#include <algorithm>
#include <cmath>

#include "mclahe_internal.cuh"

namespace mclahe {

constexpr int kGaussMaxRadius = 64;
constexpr int kMedianMaxWindow = 32;

struct GaussTaps {
    float w[2 * kGaussMaxRadius + 1];
    int r;
};

__device__ __forceinline__ int mirror_any(int j, int s) {
    while (j < 0 || j >= s) j = j < 0 ? -1 - j : 2 * s - 1 - j;
    return j;
}

// One Gaussian pass along a dimension of n elements: the volume as
// [outer][n][inner], inner contiguous.
__global__ void __launch_bounds__(256) k_gauss_pass(const float *__restrict__ in, float *__restrict__ out,
                                                    int64_t outer, int n, int64_t inner,
                                                    const GaussTaps taps) {
    const int64_t total = outer * n * inner;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t c = t % inner;
        const int64_t rest = t / inner;
        const int i = int(rest % n);
        const int64_t o = rest / n;
        const float *line = in + o * n * inner + c;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * taps.r; ++k) {
            const int j = mirror_any(i + k - taps.r, n);
            acc = __fadd_rn(acc, __fmul_rn(taps.w[k], __ldg(line + int64_t(j) * inner)));
        }
        out[t] = acc;
    }
}

struct MedianArgs {
    int D;
    int s[kMaxDim];
    int k[kMaxDim];
    int64_t stride[kMaxDim];
};

__global__ void __launch_bounds__(256) k_median(const float *__restrict__ in, float *__restrict__ out,
                                                int64_t total, const MedianArgs a) {
    const int64_t step = int64_t(gridDim.x) * blockDim.x;
    int nwin = 1;
    for (int j = 0; j < a.D; ++j) nwin *= a.k[j];
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += step) {
        int x[kMaxDim];
        int64_t rest = t;
        for (int j = a.D - 1; j >= 0; --j) {
            x[j] = int(rest % a.s[j]);
            rest /= a.s[j];
        }
        float v[kMedianMaxWindow];
        for (int w = 0; w < nwin; ++w) {
            int rw = w;
            int64_t addr = 0;
            for (int j = a.D - 1; j >= 0; --j) {
                const int oj = rw % a.k[j];
                rw /= a.k[j];
                addr += int64_t(mirror_any(x[j] - a.k[j] / 2 + oj, a.s[j])) * a.stride[j];
            }
            v[w] = __ldg(in + addr);
        }
        // the value of rank nwin / 2: v_i with (#smaller) + (#equal before i) == rank
        const int rank = nwin / 2;
        float m = v[0];
        for (int i = 0; i < nwin; ++i) {
            int below = 0;
            for (int j = 0; j < nwin; ++j) below += (v[j] < v[i]) || (v[j] == v[i] && j < i);
            if (below == rank) m = v[i];
        }
        out[t] = m;
    }
}

static int filter_grid(int64_t total) {
    return int(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, int64_t(device_sms()) * 8)));
}

static bool valid_shape(int ndim, const int64_t *shape, int64_t *total) {
    if (ndim < 1 || ndim > kMaxDim || !shape) return false;
    int64_t n = 1;
    for (int j = 0; j < ndim; ++j) {
        if (shape[j] < 1 || shape[j] > (int64_t(1) << 31) - 1) return false;
        n *= shape[j];
    }
    *total = n;
    return true;
}

}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_gaussian_weights(float sigma, float *w, int capacity, int *radius) {
    if (!w || !radius || !(sigma > 0.0f) || !std::isfinite(sigma)) return MCLAHE_ERR_INVALID_ARG;
    const int r = int(4.0 * double(sigma) + 0.5);
    if (r > kGaussMaxRadius) return MCLAHE_ERR_UNSUPPORTED;
    if (capacity < 2 * r + 1) return MCLAHE_ERR_INVALID_ARG;
    double wd[2 * kGaussMaxRadius + 1], sum = 0.0;
    for (int k = -r; k <= r; ++k) {
        wd[k + r] = std::exp(-double(k) * double(k) / (2.0 * double(sigma) * double(sigma)));
        sum += wd[k + r];
    }
    for (int k = 0; k <= 2 * r; ++k) w[k] = float(wd[k] / sum);
    *radius = r;
    return MCLAHE_OK;
}

extern "C" mclahe_status mclahe_filter_gaussian(const float *d_in, float *d_out, float *d_tmp, int ndim,
                                                const int64_t *shape, const float *sigma,
                                                mclahe_stream_t stream) {
    int64_t total = 0;
    if (!d_in || !d_out || d_in == d_out || !sigma || !valid_shape(ndim, shape, &total))
        return MCLAHE_ERR_INVALID_ARG;
    int passes = 0;
    GaussTaps taps[kMaxDim];
    for (int j = 0; j < ndim; ++j) {
        if (!(sigma[j] >= 0.0f) || !std::isfinite(sigma[j])) return MCLAHE_ERR_INVALID_ARG;
        taps[j].r = -1;
        if (sigma[j] > 0.0f) {
            const mclahe_status s = mclahe_gaussian_weights(sigma[j], taps[j].w, 2 * kGaussMaxRadius + 1,
                                                            &taps[j].r);
            if (s != MCLAHE_OK) return s;
            ++passes;
        }
    }
    if (passes >= 2 && (!d_tmp || d_tmp == d_in || d_tmp == d_out)) return MCLAHE_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (passes == 0)
        return cudaMemcpyAsync(d_out, d_in, sizeof(float) * size_t(total), cudaMemcpyDeviceToDevice, st) ==
                       cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
    // ping-pong so that the last pass writes d_out
    const float *src = d_in;
    int done = 0;
    for (int j = 0; j < ndim; ++j) {
        if (taps[j].r < 0) continue;
        ++done;
        float *dst = ((passes - done) % 2 == 0) ? d_out : d_tmp;
        int64_t outer = 1, inner = 1;
        for (int i = 0; i < j; ++i) outer *= shape[i];
        for (int i = j + 1; i < ndim; ++i) inner *= shape[i];
        k_gauss_pass<<<filter_grid(total), 256, 0, st>>>(src, dst, outer, int(shape[j]), inner, taps[j]);
        if (cudaGetLastError() != cudaSuccess) return MCLAHE_ERR_CUDA;
        src = dst;
    }
    return MCLAHE_OK;
}

extern "C" mclahe_status mclahe_filter_median(const float *d_in, float *d_out, int ndim, const int64_t *shape,
                                              const int32_t *size, mclahe_stream_t stream) {
    int64_t total = 0;
    if (!d_in || !d_out || d_in == d_out || !size || !valid_shape(ndim, shape, &total))
        return MCLAHE_ERR_INVALID_ARG;
    MedianArgs a;
    a.D = ndim;
    int nwin = 1;
    int64_t st_ = 1;
    for (int j = ndim - 1; j >= 0; --j) {
        if (size[j] < 1) return MCLAHE_ERR_INVALID_ARG;
        a.s[j] = int(shape[j]);
        a.k[j] = size[j];
        a.stride[j] = st_;
        st_ *= shape[j];
        nwin *= size[j];
        if (nwin > kMedianMaxWindow) return MCLAHE_ERR_UNSUPPORTED;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_median<<<filter_grid(total), 256, 0, st>>>(d_in, d_out, total, a);
    return cudaGetLastError() == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}
