// k_lut.cu -- clip, redistribute, cumulate and normalise every kernel's
// histogram into its mapping table (Algorithm 1, the three steps after the
// histogram), one warp per kernel.
//
// With T = clip * V, E = sum_{h > T} (h - T), N_c = #{h > T}:
//   h'_j = min(h_j, T) + E / nb,   C_j = sum_{i <= j} h'_i,
//   lut_j = (C_j - C_0) / (C_{nb-1} - C_0)   (0 when the CDF is constant).
// Writing S_j = sum of unclipped counts up to j and A_j = clipped bins up to
// j, C_j - C_0 = (S_j - S_0) + T (A_j - A_0) + j E / nb.  The clip decisions
// h > T are taken exactly in integers (h > floor(T)), the prefix sums are
// exact integers, and only the final combination is rounded in fp32.
#include "mclahe_internal.cuh"

namespace mclahe {

// 2^e as a float for -149 <= e <= 0, built from its bits.
__device__ __forceinline__ float pow2f(int e) {
    return e >= -126 ? __uint_as_float(uint32_t(e + 127) << 23)
                     : __uint_as_float(1u << (e + 149));
}

// floor(c * V) and the fractional part c * V - floor(c * V) for a float
// c in [0, 1], exactly, from the float's bits.
__device__ __forceinline__ void clip_threshold(float c, int64_t V, int64_t &t_floor, float &t_frac) {
    const uint32_t u = __float_as_uint(c);
    const int e = int((u >> 23) & 0xff);
    uint64_t mant = u & 0x7fffffu;
    int ex;
    if (e == 0) {
        ex = -126 - 23;          // subnormal
    } else {
        mant |= 0x800000u;
        ex = e - 127 - 23;
    }
    if (mant == 0) {
        t_floor = 0;
        t_frac = 0.0f;
        return;
    }
    const uint64_t prod = mant * uint64_t(V);   // < 2^24 * 2^31
    if (ex >= 0) {                               // c >= 1 (clamped to 1 before)
        t_floor = int64_t(prod << ex);
        t_frac = 0.0f;
        return;
    }
    const int sh = -ex;
    if (sh >= 64) {
        t_floor = 0;
        t_frac = (ex >= -149) ? __fmul_rn(float(prod), pow2f(ex)) : 0.0f;
        return;
    }
    t_floor = int64_t(prod >> sh);
    const uint64_t rem = prod & ((uint64_t(1) << sh) - 1);
    t_frac = __fmul_rn(float(rem), pow2f(ex));   // scaling by a power of two
}

__device__ __forceinline__ float load_clip(const float *d_clip, float plan_clip) {
    float c = d_clip ? *d_clip : plan_clip;
    c = fminf(fmaxf(c, 0.0f), 1.0f);   // NaN -> 0
    return c;
}

__global__ void __launch_bounds__(256) k_lut(Geom g, const uint32_t *__restrict__ hist,
                                             const uint32_t *__restrict__ keys,
                                             const float *__restrict__ d_clip,
                                             float *__restrict__ lut, float *__restrict__ lo_out,
                                             float *__restrict__ scale_out) {
    const int lane = threadIdx.x & 31;
    const int64_t k = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= g.K) return;
    const int nb = g.nb;
    const uint32_t *h = hist + k * nb;
    const int per = (nb + 31) >> 5;
    const int j0 = min(lane * per, nb), j1 = min(j0 + per, nb);

    int64_t tf;
    float tr;
    clip_threshold(load_clip(d_clip, g.clip), g.V, tf, tr);

    // clipped bins and their counts
    int64_t nc = 0, hc = 0, su = 0;
    for (int j = j0; j < j1; ++j) {
        const int64_t v = h[j];
        if (v > tf) {
            nc += 1;
            hc += v;
        } else {
            su += v;
        }
    }
    // lane-exclusive prefixes of (unclipped sum, clipped count)
    int64_t ps = su, pa = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t s2 = __shfl_up_sync(0xffffffffu, ps, o);
        const int64_t a2 = __shfl_up_sync(0xffffffffu, pa, o);
        if (lane >= o) {
            ps += s2;
            pa += a2;
        }
    }
    const int64_t S_tot = __shfl_sync(0xffffffffu, ps, 31);
    const int64_t N_c = __shfl_sync(0xffffffffu, pa, 31);
    int64_t H_c = hc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) H_c += __shfl_xor_sync(0xffffffffu, H_c, o);
    ps -= su;   // exclusive
    pa -= nc;

    // E = (H_c - N_c floor(T)) - N_c frac(T); each bin receives E / nb
    const float E = __fsub_rn(float(H_c - N_c * tf), __fmul_rn(float(N_c), tr));
    const float Eb = __fdiv_rn(E, float(nb));

    const int64_t h0 = h[0];
    const int64_t S0 = (h0 > tf) ? 0 : h0;
    const int64_t A0 = (h0 > tf) ? 1 : 0;
    const bool flat = (N_c == 0) && (S_tot == S0);   // constant CDF

    // C_j - C_0 for the normalisation's denominator (j = nb - 1)
    auto diff = [&](int64_t Sj, int64_t Aj, int j) {
        const int64_t ip = (Sj - S0) + (Aj - A0) * tf;
        return __fadd_rn(__fadd_rn(float(ip), __fmul_rn(float(Aj - A0), tr)),
                         __fmul_rn(float(j), Eb));
    };
    const float den = diff(S_tot, N_c, nb - 1);

    int64_t Sj = ps, Aj = pa;
    float *out = lut + k * nb;
    for (int j = j0; j < j1; ++j) {
        const int64_t v = h[j];
        if (v > tf) Aj += 1; else Sj += v;
        out[j] = flat ? 0.0f : __fdiv_rn(diff(Sj, Aj, j), den);
    }

    if (lane == 0) {
        float lo, hi;
        if (g.mode == MCLAHE_RANGE_ADAPTIVE) {
            keys_to_range(keys[2 * k], keys[2 * k + 1], lo, hi);
        } else if (g.has_range) {
            lo = g.range_lo;
            hi = g.range_hi;
        } else {
            keys_to_range(keys[0], keys[1], lo, hi);
        }
        lo_out[k] = lo;
        scale_out[k] = range_scale(lo, hi, nb);
    }
}

cudaError_t launch_lut(const mclahe_plan_s &p, unsigned char *ws, const float *d_clip,
                       cudaStream_t st) {
    const Geom &g = p.g;
    const int warps = 8;
    const unsigned grid = unsigned((g.K + warps - 1) / warps);
    k_lut<<<grid, warps * 32, 0, st>>>(g, reinterpret_cast<const uint32_t *>(ws + p.ws.hist),
                                       reinterpret_cast<const uint32_t *>(ws + p.ws.keys), d_clip,
                                       reinterpret_cast<float *>(ws + p.ws.lut),
                                       reinterpret_cast<float *>(ws + p.ws.lo),
                                       reinterpret_cast<float *>(ws + p.ws.scale));
    return cudaGetLastError();
}

}  // namespace mclahe
