// hist_impl.cuh -- per-kernel histogram and mapping table of one kernel
// (Algorithm 1: histogram, clip, redistribute, CDF, normalisation), run by one
// thread-block cluster.  Included by the per-volume launcher (k_hist.cu) and
// by the batched launcher (batch.cu).
//
// The padded volume of Sec. III.B is never built.  Along each dimension the
// kernel's footprint in the original volume splits into at most a few
// intervals of constant mirror multiplicity m in {1, 2, 3} (the number of
// images of a voxel inside the padded kernel), so the footprint is a union of
// boxes of constant weight prod(m).  Every voxel is read from memory once per
// sweep and added to its bin with that weight, which gives exactly the
// histogram of the padded kernel.
//
// Phases of one cluster (kernel k); the cluster's CTAs split every box's rows:
//   1. adaptive range only (Sec. III.D): min/max of the CTA's rows, exchanged
//      across the cluster through distributed shared memory;
//   2. histogram sweep: 128-bit loads, the exact bin quantiser on packed f32x2
//      pairs, and one shared-memory reduction per voxel into a histogram with
//      R lane copies (lane l adds to copy l mod R; with R = 32 the 32 lanes of
//      a warp always hit 32 different banks, whatever the data's skew);
//   3. the copies are summed per bin (in staggered order, conflict-free), the
//      padded indices >= n_bins - 1 folded into the last bin, and the CTAs'
//      counts summed by cluster rank 0 through distributed shared memory in
//      rank order (integers: exact and deterministic);
//   4. rank 0 stores the histogram and turns it into the mapping table with
//      the whole block (clip at T = clip * V, excess E spread as E / nb,
//      cumulative sum, min-max normalisation), the clip decisions and prefix
//      sums exact in integers.
#pragma once

#include <cooperative_groups.h>

#include "mclahe_internal.cuh"

namespace mclahe {

namespace cg = cooperative_groups;

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
    float c = d_clip ? __ldcg(d_clip) : plan_clip;
    return fminf(fmaxf(c, 0.0f), 1.0f);   // NaN -> 0
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Block-wide exclusive scan of two uint32 sequences (one value per thread);
// returns the exclusive prefixes and the totals.  All threads must call it.
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t &ea, uint32_t &eb,
                                            uint32_t &ta, uint32_t &tb) {
    __shared__ uint32_t s_wa[32], s_wb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t xa = __shfl_up_sync(0xffffffffu, ia, o);
        const uint32_t xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += xa;
            ib += xb;
        }
    }
    if (lane == 31) {
        s_wa[warp] = ia;
        s_wb[warp] = ib;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t va = lane < nw ? s_wa[lane] : 0u, vb = lane < nw ? s_wb[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t xa = __shfl_up_sync(0xffffffffu, va, o);
            const uint32_t xb = __shfl_up_sync(0xffffffffu, vb, o);
            if (lane >= o) {
                va += xa;
                vb += xb;
            }
        }
        s_wa[lane] = va;   // inclusive over warps
        s_wb[lane] = vb;
    }
    __syncthreads();
    const uint32_t offa = warp ? s_wa[warp - 1] : 0u, offb = warp ? s_wb[warp - 1] : 0u;
    ea = offa + ia - a;
    eb = offb + ib - b;
    ta = s_wa[nw - 1];
    tb = s_wb[nw - 1];
    __syncthreads();   // s_wa / s_wb may be reused by the next call
}

// Clip statistics of one kernel's histogram h[0..nb) (Algorithm 1, clip and
// redistribute), computed by the whole block; all threads must call it.  With
// T = clip * V, S_j = unclipped counts up to j and A_j = clipped bins up to j
// (h_j > T, decided exactly in integers as h_j > floor(T)):
//   C_j - C_0 = (S_j - S_0) + T (A_j - A_0) + j E / nb,  E = H_c - N_c T.
// Each thread owns the bins [j0, j1); ps / pa are the exclusive prefixes of
// S and A at j0.
struct LutStats {
    int64_t tf;          // floor(T)
    float tr;            // T - floor(T)
    int64_t S0, A0;      // S_0, A_0
    int64_t S_tot, N_c;  // S_{nb-1}, A_{nb-1}
    float Eb;            // E / nb
    float den;           // C_{nb-1} - C_0
    bool flat;           // constant CDF (den = 0)
    int j0, j1;
    int64_t ps, pa;
    __device__ __forceinline__ float diff(int64_t Sj, int64_t Aj, int j) const {
        const int64_t ip = (Sj - S0) + (Aj - A0) * tf;
        return __fadd_rn(__fadd_rn(float(ip), __fmul_rn(float(Aj - A0), tr)),
                         __fmul_rn(float(j), Eb));
    }
};

__device__ __forceinline__ LutStats lut_stats(const uint32_t *h, int nb, int64_t V, float clip) {
    __shared__ uint32_t s_first[2];
    LutStats st;
    const int nt = blockDim.x;
    const int per = (nb + nt - 1) / nt;
    st.j0 = min(int(threadIdx.x) * per, nb);
    st.j1 = min(st.j0 + per, nb);
    clip_threshold(clip, V, st.tf, st.tr);
    uint32_t nc = 0, su = 0;
    for (int j = st.j0; j < st.j1; ++j) {
        const uint32_t v = h[j];
        if (int64_t(v) > st.tf) nc += 1; else su += v;
    }
    if (threadIdx.x == 0) {
        const uint32_t v0 = h[0];
        s_first[0] = (int64_t(v0) > st.tf) ? 0u : v0;   // S_0
        s_first[1] = (int64_t(v0) > st.tf) ? 1u : 0u;   // A_0
    }
    uint32_t ps, pa, S_tot, N_c;
    block_scan2(su, nc, ps, pa, S_tot, N_c);   // its barriers publish s_first
    st.ps = ps;
    st.pa = pa;
    st.S_tot = S_tot;
    st.N_c = N_c;
    st.S0 = s_first[0];
    st.A0 = s_first[1];
    // H_c = V - S_tot: every voxel of the padded kernel is counted once
    const int64_t H_c = V - st.S_tot;
    const float E = __fsub_rn(float(H_c - st.N_c * st.tf), __fmul_rn(float(st.N_c), st.tr));
    st.Eb = __fdiv_rn(E, float(nb));
    st.flat = (st.N_c == 0) && (st.S_tot == st.S0);
    st.den = st.diff(st.S_tot, st.N_c, nb - 1);
    __syncthreads();   // s_first may be reused by the next call
    return st;
}

// The mapping table of one kernel from its histogram h[0..nb) (shared memory),
// written to out[0..LS) (entries nb..LS-1 repeat entry nb-1):
// lut_j = (C_j - C_0) / (C_{nb-1} - C_0), 0 for a constant CDF.  All threads
// of the block call it.
__device__ __forceinline__ void block_lut(const uint32_t *h, int nb, int LS, int64_t V, float clip,
                          float *__restrict__ out) {
    const LutStats st = lut_stats(h, nb, V, clip);
    int64_t Sj = st.ps, Aj = st.pa;
    for (int j = st.j0; j < st.j1; ++j) {
        const uint32_t v = h[j];
        if (int64_t(v) > st.tf) Aj += 1; else Sj += v;
        out[j] = st.flat ? 0.0f : __fdiv_rn(st.diff(Sj, Aj, j), st.den);
    }
    // the last entry is den / den = 1 (0 for a constant CDF)
    for (int j = nb + int(threadIdx.x); j < LS; j += blockDim.x) out[j] = st.flat ? 0.0f : 1.0f;
}

// Shared memory of one histogram CTA: R copies of P bins plus P counts.
__host__ __device__ inline size_t hist_smem_words(int P, int R) { return size_t(P) * R + P; }

template <int D, bool ADAPTIVE>
__device__ __forceinline__ void hist_kernel(const Geom &g, const float *__restrict__ in,
                                            const uint32_t *__restrict__ keys,
                                            const float *__restrict__ d_clip,
                                            uint32_t *__restrict__ hist, float *__restrict__ lut,
                                            float *__restrict__ lo_out,
                                            float *__restrict__ scale_out, int64_t k, int R,
                                            uint32_t *sh) {
    __shared__ float s_red[2][32];
    __shared__ float s_mm[2];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int nb = g.nb, P = g.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *cnt = sh + size_t(P) * R;

    // kernel coordinates and the constant-multiplicity pieces of its footprint
    Pieces pc[D];
    int nsub = 1;
    {
        int64_t r = k;
        int kk[kMaxDim];
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            kk[j] = int(r % g.d[j].n);
            r /= g.d[j].n;
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            pc[j] = footprint_pieces(g.d[j], kk[j]);
            nsub *= pc[j].n;
        }
    }
    int64_t stride[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) stride[j] = g.d[j].stride;
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);

    // visits every box of the footprint: fn(box_lo, box_len, weight, r0, r1)
    auto for_boxes = [&](auto &&fn) {
        for (int sb = 0; sb < nsub; ++sb) {
            int box_lo[kMaxDim], len[kMaxDim];
            int w = 1, rest = sb, rows = 1;
#pragma unroll
            for (int j = D - 1; j >= 0; --j) {
                const int i = rest % pc[j].n;
                rest /= pc[j].n;
                box_lo[j] = pc[j].a[i];
                len[j] = pc[j].e[i] - pc[j].a[i];
                w *= pc[j].m[i];
                if (j < D - 1) rows *= len[j];
            }
            const int r0 = int((int64_t(rows) * rank) / C);
            const int r1 = int((int64_t(rows) * (rank + 1)) / C);
            if (r1 > r0) fn(box_lo, len, w, r0, r1);
        }
    };

    {   // zero the copies and the counts
        uint4 *z = reinterpret_cast<uint4 *>(sh);
        const int n4 = int(hist_smem_words(P, R) / 4);
        for (int i = threadIdx.x; i < n4; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
        for (int i = n4 * 4 + threadIdx.x; i < int(hist_smem_words(P, R)); i += blockDim.x) sh[i] = 0;
    }

    struct NoRow {};
    auto no_row = [](const int *, int64_t, NoRow &) {};

    float lo, hi;
    if (ADAPTIVE) {
        // phase 1: min/max of this CTA's rows of the footprint
        float mn = INFINITY, mx = -INFINITY;
        for_boxes([&](const int *box_lo, const int *len, int, int r0, int r1) {
            const int L = len[D - 1];
            auto mm_quad = [&](NoRow &, const QuadRef &q) {
                if (!q.has) return;
                if (q.e0 >= 0 && q.e0 + 4 <= L) {
                    mn = min3f(mn, q.v.x, q.v.y);
                    mn = min3f(mn, q.v.z, q.v.w);
                    mx = max3f(mx, q.v.x, q.v.y);
                    mx = max3f(mx, q.v.z, q.v.w);
                } else {
                    const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int el = q.e0 + e;
                        if (el >= 0 && el < L) {
                            mn = fminf(mn, vals[e]);
                            mx = fmaxf(mx, vals[e]);
                        }
                    }
                }
            };
            walk_box<D, 4, NoRow>(in, nullptr, g.N, stride, box_lo, len, r0, r1, same_align, false, no_row,
                               mm_quad);
        });
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
        cluster.sync();   // every CTA's min/max (and zeroed bins) are visible
        lo = INFINITY;
        hi = -INFINITY;
        for (int c = 0; c < C; ++c) {
            const float *rm = cluster.map_shared_rank(s_mm, c);
            lo = fminf(lo, rm[0]);
            hi = fmaxf(hi, rm[1]);
        }
    } else {
        if (g.has_range) {
            lo = g.range_lo;
            hi = g.range_hi;
        } else {
            keys_to_range(__ldcg(keys), __ldcg(keys + 1), lo, hi);   // L2: may be this launch's
        }
        __syncthreads();   // bins zeroed
    }
    const float scale = range_scale(lo, hi, nb);

    // phase 2: histogram sweep, weight w per box
    {
        const uint32_t sh_base = uint32_t(__cvta_generic_to_shared(sh));
        const uint32_t r4 = uint32_t(4 * R);
        const uint32_t base_l = sh_base + 4u * uint32_t(lane & (R - 1)) - kBinBias * r4;
        const float2 nlo2 = make_float2(-lo, -lo), sc2 = make_float2(scale, scale);
        const float iqk = g.iqk, qkf = g.qkf;
        for_boxes([&](const int *box_lo, const int *len, int w, int r0, int r1) {
            const int L = len[D - 1];
            const uint32_t wu = uint32_t(w);
            auto hist_quad = [&](NoRow &, const QuadRef &q) {
                if (!q.has) return;
                const uint2 b01 = qbits2(make_float2(q.v.x, q.v.y), nlo2, sc2, iqk, qkf);
                const uint2 b23 = qbits2(make_float2(q.v.z, q.v.w), nlo2, sc2, iqk, qkf);
                const uint32_t bits[4] = {b01.x, b01.y, b23.x, b23.y};
                if (q.e0 >= 0 && q.e0 + 4 <= L) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) red_shared_add(bits[e] * r4 + base_l, wu);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int el = q.e0 + e;
                        if (el >= 0 && el < L) red_shared_add(bits[e] * r4 + base_l, wu);
                    }
                }
            };
            walk_box<D, 4, NoRow>(in, nullptr, g.N, stride, box_lo, len, r0, r1, same_align, false, no_row,
                               hist_quad);
        });
    }
    __syncthreads();

    // phase 3: sum the copies (copy (c + j) mod R of bin j at step c: the
    // threads of a warp read different banks), fold the padded indices
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        const uint32_t *row = sh + size_t(j) * R;
        uint32_t s = 0;
        for (int c = 0; c < R; ++c) s += row[(c + j) & (R - 1)];
        cnt[j] = s;
    }
    __syncthreads();
    for (int j = nb + int(threadIdx.x); j < P; j += blockDim.x) atomicAdd(&cnt[nb - 1], cnt[j]);
    if (C > 1) {
        cluster.sync();   // every CTA's counts are complete
        if (rank == 0) {
            for (int j = threadIdx.x; j < nb; j += blockDim.x) {
                uint32_t s = cnt[j];
                for (int c = 1; c < C; ++c) s += cluster.map_shared_rank(cnt, c)[j];
                cnt[j] = s;
            }
        }
        cluster.sync();   // rank 0 has read the other CTAs' shared memory
    } else {
        __syncthreads();
    }

    // phase 4: rank 0 stores the histogram and builds the mapping table
    if (rank == 0) {
        uint32_t *gh = hist + k * nb;
        for (int j = threadIdx.x; j < nb; j += blockDim.x) gh[j] = cnt[j];
        block_lut(cnt, nb, g.LS, g.V, load_clip(d_clip, g.clip), lut + k * g.LS);
        if (threadIdx.x == 0) {
            lo_out[k] = lo;
            scale_out[k] = scale;
        }
    }
}

}  // namespace mclahe
