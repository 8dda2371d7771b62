// k_hist.cu -- per-kernel histograms and mapping tables (Algorithm 1: the
// histogram, clip/redistribute, CDF and normalisation steps), fused into one
// launch with one thread-block cluster per kernel.
//
// The padded volume of Sec. III.B is never built.  Each CTA of a kernel's
// cluster reads a slice of the kernel's footprint in the original volume (the
// original voxels with at least one mirror image inside the padded kernel).
// A voxel counts once per image, its multiplicity being a product of
// per-dimension factors in {1, 2, 3}; this gives exactly the histogram of the
// padded kernel while every voxel is read from HBM once.
//
// Phases of one cluster (kernel k):
//   1. adaptive range only (Sec. III.D): min/max of the CTA's slice, exchanged
//      across the cluster through distributed shared memory;
//   2. histogram of the slice in shared memory: 128-bit loads, several in
//      flight per thread, equal (bin, multiplicity) pairs of a warp merged with
//      __match_any_sync before the shared-memory atomic;
//   3. the slices' bins added into cluster rank 0 (distributed shared memory
//      atomics on integers, so the order does not matter);
//   4. rank 0 stores the histogram, and its first warp turns it into the
//      kernel's mapping table (clip at T = clip * V, excess E spread as E/nb,
//      cumulative sum, min-max normalisation), with exact integer clip
//      decisions and prefix sums.
#include <cooperative_groups.h>

#include "mclahe_internal.cuh"

namespace cg = cooperative_groups;

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
    if (ex >= 0) {                               // not reached for c <= 1
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
    return fminf(fmaxf(c, 0.0f), 1.0f);   // NaN -> 0
}

// One warp turns the histogram h (nb bins, any memory space) into the
// kernel's mapping table.  With S_j = unclipped counts up to j, A_j = clipped
// bins up to j:  C_j - C_0 = (S_j - S_0) + T (A_j - A_0) + j E / nb.
__device__ void warp_lut(const uint32_t *h, int nb, int64_t V, float clip, float *out, int lane) {
    const int per = (nb + 31) >> 5;
    const int j0 = min(lane * per, nb), j1 = min(j0 + per, nb);
    int64_t tf;
    float tr;
    clip_threshold(clip, V, tf, tr);
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
    ps -= su;   // exclusive prefixes
    pa -= nc;
    // E = (H_c - N_c floor(T)) - N_c frac(T); each bin receives E / nb
    const float E = __fsub_rn(float(H_c - N_c * tf), __fmul_rn(float(N_c), tr));
    const float Eb = __fdiv_rn(E, float(nb));
    const int64_t h0 = h[0];
    const int64_t S0 = (h0 > tf) ? 0 : h0;
    const int64_t A0 = (h0 > tf) ? 1 : 0;
    const bool flat = (N_c == 0) && (S_tot == S0);   // constant CDF
    auto diff = [&](int64_t Sj, int64_t Aj, int j) {
        const int64_t ip = (Sj - S0) + (Aj - A0) * tf;
        return __fadd_rn(__fadd_rn(float(ip), __fmul_rn(float(Aj - A0), tr)),
                         __fmul_rn(float(j), Eb));
    };
    const float den = diff(S_tot, N_c, nb - 1);
    int64_t Sj = ps, Aj = pa;
    for (int j = j0; j < j1; ++j) {
        const int64_t v = h[j];
        if (v > tf) Aj += 1; else Sj += v;
        out[j] = flat ? 0.0f : __fdiv_rn(diff(Sj, Aj, j), den);
    }
}

template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(256) k_hist(Geom g, const float *__restrict__ in,
                                              const uint32_t *__restrict__ keys,
                                              const float *__restrict__ d_clip,
                                              uint32_t *__restrict__ hist, float *__restrict__ lut,
                                              float *__restrict__ lo_out,
                                              float *__restrict__ scale_out) {
    extern __shared__ uint32_t sh[];           // nb bins
    __shared__ float s_red[2][32];
    __shared__ float s_mm[2];
    cg::cluster_group cluster = cg::this_cluster();
    const int chunks = int(cluster.num_blocks());
    const int chunk = int(cluster.block_rank());
    const int64_t k = blockIdx.x / chunks;
    const int nb = g.nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    int kk[kMaxDim];
    {
        int64_t r = k;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            kk[j] = int(r % g.d[j].n);
            r /= g.d[j].n;
        }
    }
    Foot f[kMaxDim];
    int len[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        f[j] = footprint(g.d[j], kk[j]);
        len[j] = f[j].hi - f[j].lo;
    }
    int R = 1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) R *= len[j];
    const int r0 = int((int64_t(R) * chunk) / chunks);
    const int r1 = int((int64_t(R) * (chunk + 1)) / chunks);

    const int L = len[D - 1];
    const int xl = f[D - 1].lo;
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);
    const WalkShape ws = walk_shape(L, xl, same_align, blockDim.x);
    const Foot fl = f[D - 1];
    const bool last_mirror = (fl.lh > fl.ll) || (fl.rh > fl.rl);
    int box_lo[kMaxDim];
    int64_t stride[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        box_lo[j] = f[j].lo;
        stride[j] = g.d[j].stride;
    }

    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;

    float lo, hi;
    if (ADAPTIVE) {
        // phase 1: min/max of this CTA's slice
        float mn = INFINITY, mx = -INFINITY;
        struct NoRow {};
        auto row_none = [](const int *, int64_t, NoRow &) {};
        auto mm_quad = [&](NoRow &, const QuadRef &q) {
            const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int el = q.e0 + e;
                if (q.has && el >= 0 && el < L) {
                    mn = fminf(mn, vals[e]);
                    mx = fmaxf(mx, vals[e]);
                }
            }
        };
        if (ws.ru == 1)
            walk_rows<D, 1, NoRow>(in, g.N, stride, box_lo, len, r0, r1, ws, false, row_none, mm_quad);
        else if (ws.ru == 2)
            walk_rows<D, 2, NoRow>(in, g.N, stride, box_lo, len, r0, r1, ws, false, row_none, mm_quad);
        else
            walk_rows<D, 4, NoRow>(in, g.N, stride, box_lo, len, r0, r1, ws, false, row_none, mm_quad);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            s_red[0][warp] = mn;
            s_red[1][warp] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < int(blockDim.x >> 5); ++w) {
                mn = fminf(mn, s_red[0][w]);
                mx = fmaxf(mx, s_red[1][w]);
            }
            s_mm[0] = mn;
            s_mm[1] = mx;
        }
        cluster.sync();   // every slice's min/max is visible
        lo = INFINITY;
        hi = -INFINITY;
        for (int c = 0; c < chunks; ++c) {
            const float *rm = cluster.map_shared_rank(s_mm, c);
            lo = fminf(lo, rm[0]);
            hi = fmaxf(hi, rm[1]);
        }
    } else if (g.has_range) {
        lo = g.range_lo;
        hi = g.range_hi;
        cluster.sync();   // the histogram below is zeroed in every CTA
    } else {
        keys_to_range(keys[0], keys[1], lo, hi);
        cluster.sync();
    }
    const float scale = range_scale(lo, hi, nb);
    const float top = float(nb - 1);

    // phase 2: histogram of this CTA's slice.  Key = bin | multiplicity << 16;
    // the lowest lane of each group of equal keys adds count * multiplicity.
    {
        uint32_t lt_mask;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt_mask));
        struct HRow {
            uint32_t wo;   // multiplicity over dims 0..D-2
        };
        auto hist_row = [&](const int *coords, int64_t, HRow &st) {
            int w = 1;
#pragma unroll
            for (int j = 0; j < D - 1; ++j) w *= f[j].mult(coords[j]);
            st.wo = uint32_t(w);
        };
        auto hist_quad = [&](HRow &st, const QuadRef &q) {
            const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int el = q.e0 + e;
                const bool ok = q.has && el >= 0 && el < L;
                uint32_t w = st.wo;
                if (last_mirror) w *= uint32_t(fl.mult(xl + el));
                const uint32_t bits = quantise_bits(vals[e], lo, scale, top);
                const uint32_t key = ok ? ((bits & 0xffffu) | (w << 16)) : 0xffffffffu;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                if (ok && (peers & lt_mask) == 0)
                    atomicAdd(&sh[key & 0xffffu], uint32_t(__popc(peers)) * (key >> 16));
            }
        };
        if (ws.ru == 1)
            walk_rows<D, 1, HRow>(in, g.N, stride, box_lo, len, r0, r1, ws, false, hist_row, hist_quad);
        else if (ws.ru == 2)
            walk_rows<D, 2, HRow>(in, g.N, stride, box_lo, len, r0, r1, ws, false, hist_row, hist_quad);
        else
            walk_rows<D, 4, HRow>(in, g.N, stride, box_lo, len, r0, r1, ws, false, hist_row, hist_quad);
    }
    __syncthreads();

    // phase 3: add the slices into rank 0
    if (chunks > 1) {
        if (chunk != 0) {
            uint32_t *dst = cluster.map_shared_rank(sh, 0);
            for (int i = threadIdx.x; i < nb; i += blockDim.x) {
                const uint32_t c = sh[i];
                if (c) atomicAdd(&dst[i], c);
            }
        }
        cluster.sync();
    }

    // phase 4: rank 0 stores the histogram and builds the mapping table
    if (chunk == 0) {
        uint32_t *gh = hist + k * nb;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) gh[i] = sh[i];
        if (warp == 0) {
            warp_lut(sh, nb, g.V, load_clip(d_clip, g.clip), lut + k * nb, lane);
            if (lane == 0) {
                lo_out[k] = lo;
                scale_out[k] = scale;
            }
        }
    }
}

template <int D, bool ADAPTIVE>
static cudaError_t launch_hist_dm(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                  const float *d_clip, cudaStream_t st) {
    const Geom &g = p.g;
    const int chunks = p.t.hist_chunks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(g.K * chunks));
    cfg.blockDim = dim3(p.t.hist_threads);
    cfg.dynamicSmemBytes = size_t(g.nb) * sizeof(uint32_t);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = chunks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_hist<D, ADAPTIVE>, g, in,
                              reinterpret_cast<const uint32_t *>(ws + p.ws.keys), d_clip,
                              reinterpret_cast<uint32_t *>(ws + p.ws.hist),
                              reinterpret_cast<float *>(ws + p.ws.lut),
                              reinterpret_cast<float *>(ws + p.ws.lo),
                              reinterpret_cast<float *>(ws + p.ws.scale));
}

template <int D>
static cudaError_t launch_hist_d(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                 const float *d_clip, cudaStream_t st) {
    if (p.g.mode == MCLAHE_RANGE_ADAPTIVE) return launch_hist_dm<D, true>(p, in, ws, d_clip, st);
    return launch_hist_dm<D, false>(p, in, ws, d_clip, st);
}

cudaError_t launch_hist(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                        const float *d_clip, cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_hist_d<1>(p, in, ws, d_clip, st);
        case 2: return launch_hist_d<2>(p, in, ws, d_clip, st);
        case 3: return launch_hist_d<3>(p, in, ws, d_clip, st);
        case 4: return launch_hist_d<4>(p, in, ws, d_clip, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
