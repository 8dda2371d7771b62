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
// A work item is a group of G consecutive kernels along the last dimension
// (see hist_group); its CTAs split every footprint box's rows.  Phases:
//   1. adaptive range only (Sec. III.D): min/max of every kernel of the group
//      over the CTA's rows, exchanged across the cluster through distributed
//      shared memory;
//   2. histogram sweep: 128-bit loads, the exact bin quantiser on packed f32x2
//      pairs, and one shared-memory reduction per voxel into its kernel's
//      histogram, kept in R lane copies (lane l adds to copy l mod R; with
//      R = 32 the lanes of a warp always hit different banks, whatever the
//      data's skew).  Each thread owns fixed quad slots of every row (tile
//      walker), so the kernel and weight of a slot are found once per box;
//      quads that straddle kernels or mirror boundaries take a per-voxel path;
//   3. the copies are summed per bin (in staggered order, conflict-free) and
//      the padded indices >= n_bins - 1 folded into the last bin;
//   4. cluster rank r owns kernels r, r + C, ... of the group: it sums the
//      CTAs' counts in rank order through distributed shared memory (integers:
//      exact and deterministic), stores the histogram and turns it into the
//      mapping table with the whole block (clip at T = clip * V, excess E
//      spread as E / nb, cumulative sum, min-max normalisation), the clip
//      decisions and prefix sums exact in integers.
#pragma once

#include <cooperative_groups.h>

#include "mclahe_internal.cuh"
#include "tma.cuh"

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

// The same table built by one warp, so the warps of a block build several
// kernels' tables at once.  Lane l owns the contiguous bins [l c, l c + c),
// c = ceil(nb / 32): one pass over its bins for the unclipped sum and clipped
// count, one warp scan for the prefixes at its first bin, then its bins in
// order.  The statistics are the same integers and every entry the same float
// operations as block_lut's: the tables are identical.
__device__ __forceinline__ void warp_lut(const uint32_t *h, int nb, int LS, int64_t V, float clip,
                                         float *__restrict__ out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    LutStats st;
    clip_threshold(clip, V, st.tf, st.tr);
    const int per = (nb + 31) >> 5;
    const int j0 = min(lane * per, nb), j1 = min(j0 + per, nb);
    uint32_t nc = 0, su = 0;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const uint32_t v = h[j];
        if (int64_t(v) > st.tf) nc += 1; else su += v;
    }
    // inclusive warp scans of the per-lane sums
    uint32_t is = su, ia = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t xs = __shfl_up_sync(full, is, o);
        const uint32_t xa = __shfl_up_sync(full, ia, o);
        if (lane >= o) {
            is += xs;
            ia += xa;
        }
    }
    st.S_tot = __shfl_sync(full, is, 31);
    st.N_c = __shfl_sync(full, ia, 31);
    const uint32_t v0 = h[0];
    st.S0 = (int64_t(v0) > st.tf) ? 0 : v0;
    st.A0 = (int64_t(v0) > st.tf) ? 1 : 0;
    const int64_t H_c = V - st.S_tot;
    const float E = __fsub_rn(float(H_c - st.N_c * st.tf), __fmul_rn(float(st.N_c), st.tr));
    st.Eb = __fdiv_rn(E, float(nb));
    st.flat = (st.N_c == 0) && (st.S_tot == st.S0);
    st.den = st.diff(st.S_tot, st.N_c, nb - 1);
    int64_t Sj = is - su, Aj = ia - nc;   // exclusive prefixes at j0
    // unrolled: the bins' divisions are independent and overlap
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const uint32_t v = h[j];
        if (int64_t(v) > st.tf) Aj += 1; else Sj += v;
        out[j] = st.flat ? 0.0f : __fdiv_rn(st.diff(Sj, Aj, j), st.den);
    }
    for (int j = nb + lane; j < LS; j += 32) out[j] = st.flat ? 0.0f : 1.0f;
}

// The tables of n kernels at once, g = nw / n >= 2 warps per kernel: kernel
// i's histogram h0 + i P is built by warps [i g, (i + 1) g), lane li of the
// group owning the contiguous bins [li c, li c + c), c = ceil(nb / 32 g).
// The statistics are the same integers (the group's scan gives every lane the
// same exclusive prefixes as a warp or block scan) and every entry the same
// float operations as warp_lut's: the tables are identical.  All threads of
// the block call it (two block barriers).
__device__ __forceinline__ void group_luts(const uint32_t *h0, int P, int n, int nb, int LS, int64_t V,
                                           float clip, float *__restrict__ lut, int64_t k0,
                                           int64_t kstep) {
    __shared__ uint32_t s_su[32], s_nc[32];
    const unsigned full = 0xffffffffu;
    const int nw = int(blockDim.x >> 5), warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const int g = nw / n, i = warp / g, wg = warp - i * g;
    const bool active = i < n;   // the last nw - n g warps idle
    const uint32_t *h = h0 + size_t(active ? i : 0) * P;
    LutStats st;
    clip_threshold(clip, V, st.tf, st.tr);
    const int L = 32 * g, li = wg * 32 + lane;
    const int per = (nb + L - 1) / L;
    const int j0 = active ? min(li * per, nb) : nb, j1 = active ? min(j0 + per, nb) : nb;
    uint32_t nc = 0, su = 0;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const uint32_t v = h[j];
        if (int64_t(v) > st.tf) nc += 1; else su += v;
    }
    uint32_t is = su, ia = nc;   // inclusive scans within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t xs = __shfl_up_sync(full, is, o);
        const uint32_t xa = __shfl_up_sync(full, ia, o);
        if (lane >= o) {
            is += xs;
            ia += xa;
        }
    }
    if (lane == 31) {
        s_su[warp] = is;
        s_nc[warp] = ia;
    }
    __syncthreads();
    uint32_t os = 0, oa = 0, ts = 0, ta = 0;   // earlier warps of the group; the group's totals
    if (active)
        for (int w = 0; w < g; ++w) {
            const uint32_t a = s_su[i * g + w], b = s_nc[i * g + w];
            if (w < wg) {
                os += a;
                oa += b;
            }
            ts += a;
            ta += b;
        }
    __syncthreads();   // s_su / s_nc may be reused by the next call
    if (!active) return;
    st.S_tot = ts;
    st.N_c = ta;
    const uint32_t v0 = h[0];
    st.S0 = (int64_t(v0) > st.tf) ? 0 : v0;
    st.A0 = (int64_t(v0) > st.tf) ? 1 : 0;
    const int64_t H_c = V - st.S_tot;
    const float E = __fsub_rn(float(H_c - st.N_c * st.tf), __fmul_rn(float(st.N_c), st.tr));
    st.Eb = __fdiv_rn(E, float(nb));
    st.flat = (st.N_c == 0) && (st.S_tot == st.S0);
    st.den = st.diff(st.S_tot, st.N_c, nb - 1);
    float *out = lut + (k0 + i * kstep) * LS;
    int64_t Sj = int64_t(os) + (is - su), Aj = int64_t(oa) + (ia - nc);   // exclusive prefixes at j0
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const uint32_t v = h[j];
        if (int64_t(v) > st.tf) Aj += 1; else Sj += v;
        out[j] = st.flat ? 0.0f : __fdiv_rn(st.diff(Sj, Aj, j), st.den);
    }
    for (int j = nb + li; j < LS; j += L) out[j] = st.flat ? 0.0f : 1.0f;
}

// Tables of n kernels whose histograms lie in shared memory at h + i * P:
// one block-wide build for a single kernel, a group of warps per kernel while
// every kernel gets at least two warps, else one warp per kernel (block builds
// one kernel after another measured slower on the 4-D workload: 3 kernels per
// 512-thread CTA).
__device__ __forceinline__ void build_luts(const uint32_t *h, int P, int n, int nb, int LS, int64_t V,
                                           float clip, float *__restrict__ lut, int64_t k0,
                                           int64_t kstep) {
    if (n == 1) {
        block_lut(h, nb, LS, V, clip, lut + k0 * LS);
        return;
    }
    const int nw = int(blockDim.x >> 5), warp = int(threadIdx.x >> 5);
    if (2 * n <= nw && nw <= 32) {
        group_luts(h, P, n, nb, LS, V, clip, lut, k0, kstep);
        return;
    }
    for (int i = warp; i < n; i += nw)
        warp_lut(h + size_t(i) * P, nb, LS, V, clip, lut + (k0 + i * kstep) * LS);
}

// ---------------------------------------------------------------------------
// Work item of the histogram pass: a group of G consecutive kernels along the
// last (contiguous) dimension, at fixed kernel coordinates along the others.
// Its footprint rows are contiguous runs of memory covering all G kernels, so
// neighbouring kernels' voxels are read once, in whole sectors, by one item.
// Shared memory of one CTA (32-bit words): R lane copies of the P padded bins
// of every kernel of the group, the P counts of every kernel, and per kernel
// its range keys and quantiser constants.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t hist_smem_words(int P, int R, int G) {
    return size_t(G) * P * R + size_t(G) * P + 5 * size_t(G);
}
// How a CTA streams the rows of a box (the shared memory behind these words):
//   kHistLsu   walk_tile, 128-bit loads into registers (batched launch);
//   kHistRing  walk_tile_async: a cp.async ring of kHistStages row stages of
//              kHistQmax quads per thread, two rows per thread in flight;
//   kHistTma   walk_tile_tma: box tiles of up to kHistTileFloats floats
//              loaded by TMA into kHistTmaStages stages (boxes wider than the
//              tile fall back to the ring).
constexpr int kHistLsu = 0, kHistRing = 1, kHistTma = 2;
// Boxes along the last dim are cut into segments of at most kHistSeg elements.
constexpr int kHistSeg = 4 * 32 * 4 - 4;
constexpr int kHistQmax = 4;     // quad slots per thread and row in the histogram pass
constexpr int kHistStages = 3;
constexpr int kHistTmaStages = 4;
constexpr int kHistTileFloats = 2048;   // 2 quads per thread of 256
constexpr uint32_t kHistTmaStage = kHistTileFloats * 4;

// Tensor map of the volume with its tile box (Bx elements along the last dim,
// By rows along dim D-2), for kHistTma.
struct HistTma {
    const CUtensorMap *map;
    int bx, by;
};
__host__ __device__ inline size_t hist_ring_offset_words(size_t words) { return (words + 3) & ~size_t(3); }
__host__ __device__ inline size_t hist_ring_bytes(int nthreads) {
    return size_t(kHistStages) * kHistQmax * size_t(nthreads) * 16;
}

// Kernels (relative to kl0, among [kl0, kl1)) that hold an image of the
// original index x along one dimension, with multiplicities (Sec. III.B: x
// has its main image at x + p0 and mirror images at p0 - 1 - x for x < p0 and
// at 2s - 1 - x + p0 for x >= s - p1).
struct Targets {
    int n;               // distinct kernels
    int kg[3], m[3];     // group-relative kernel and multiplicity (static indices only)
};

__device__ __forceinline__ Targets last_targets(const Dim &d, int x, int kl0, int kl1) {
    int kc[3];
    kc[0] = (x + d.p0) / d.b;
    kc[1] = (x < d.p0) ? (d.p0 - 1 - x) / d.b : -1;
    kc[2] = (x >= d.s - d.p1) ? (2 * d.s - 1 - x + d.p0) / d.b : -1;
    Targets t;
    t.n = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        t.kg[i] = 0;
        t.m[i] = 0;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int k = kc[i];
        if (k < kl0 || k >= kl1) continue;
        bool merged = false;
#pragma unroll
        for (int j = 0; j < i; ++j)
            if (j < t.n && t.kg[j] == k - kl0) {
                t.m[j] += 1;
                merged = true;
            }
        if (!merged) {
            // append at position t.n (0..2) with static stores
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j == t.n) {
                    t.kg[j] = k - kl0;
                    t.m[j] = 1;
                }
            t.n += 1;
        }
    }
    return t;
}

// Phase 4 of the cluster form: cluster rank r owns kernels r, r + C, ... of
// the GK kernels of the item: it sums the CTAs' counts (cnt, [GK][P] in every
// CTA's shared memory) in rank order into its own copy area (sh, free now),
// stores the histograms and ranges and builds the mapping tables.  Every CTA
// of the cluster calls it after a cluster barrier that follows the counts.
__device__ __forceinline__ void merge_and_build(const Geom &g, uint32_t *sh, uint32_t *cnt,
                                                const float *s_lo, const float *s_sc, int GK, int C,
                                                int rank, uint32_t *__restrict__ hist,
                                                float *__restrict__ lut, float *__restrict__ lo_out,
                                                float *__restrict__ scale_out, int64_t kfirst,
                                                const float *__restrict__ d_clip) {
    cg::cluster_group cluster = cg::this_cluster();
    const int nb = g.nb, P = g.P;
    const int n_own = GK > rank ? (GK - rank + C - 1) / C : 0;
    uint32_t *own = sh;   // [n_own][P]
    for (int t = threadIdx.x; t < n_own * nb; t += blockDim.x) {
        const int i = t / nb, j = t - i * nb;
        const int kg = rank + i * C;
        uint32_t s = 0;
        if (C > 1) {
            for (int c = 0; c < C; ++c) s += cluster.map_shared_rank(cnt, c)[size_t(kg) * P + j];
        } else {
            s = cnt[size_t(kg) * P + j];
        }
        own[size_t(i) * P + j] = s;
        hist[(kfirst + kg) * nb + j] = s;
    }
    for (int i = threadIdx.x; i < n_own; i += blockDim.x) {
        const int kg = rank + i * C;
        lo_out[kfirst + kg] = s_lo[kg];
        scale_out[kfirst + kg] = s_sc[kg];
    }
    __syncthreads();
    if (n_own > 0)
        build_luts(own, P, n_own, nb, g.LS, g.V, load_clip(d_clip, g.clip), lut, kfirst + rank, C);
    if (C > 1) cluster.sync(); else __syncthreads();   // the other CTAs' shared memory is no longer read
}

// Phase 3: sum the R lane copies of every bin of GK kernels into cnt[GK][P]
// and fold the padded indices >= n_bins - 1 into the last bin.  Thread t sums
// bin row t (words t R .. t R + R - 1); at step c lane l reads copy
// (c + l R / 32) mod R, so the R lanes whose rows start in the same bank
// (l mod 32/R equal, R <= 32) read R different banks: no conflicts.  All
// threads of the block call it after the sweep's barrier.
__device__ __forceinline__ void sum_copies(const uint32_t *sh, uint32_t *cnt, int GK, int P, int R,
                                           int nb) {
    const int rot = (int(threadIdx.x & 31) * R) >> 5;
    for (int t = threadIdx.x; t < GK * P; t += blockDim.x) {
        const uint32_t *row = sh + size_t(t) * R;
        uint32_t s = 0;
        for (int c = 0; c < R; ++c) s += row[(c + rot) & (R - 1)];
        cnt[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < GK * (P - nb); t += blockDim.x) {
        const int kg = t / (P - nb), j = nb + t % (P - nb);
        atomicAdd(&cnt[kg * P + nb - 1], cnt[kg * P + j]);
    }
}

// Modes of hist_group:
//   kHistCluster   one thread-block cluster per item (phases 1-4 below; the
//                  ranks split the rows, merge through DSMEM, build the tables);
//   kHistFlat      shares [c0, c1) of `nchunks` of an item (the same fraction
//                  of the rows of every box) in the flat persistent pass: the
//                  CTA adds its counts to the global histograms with integer
//                  atomics and bumps the item's ticket by c1 - c0; the CTA that
//                  completes the ticket builds the item's tables from the
//                  global histograms.  Adaptive ranges come from the per-kernel
//                  keys the range pass left;
//   kHistMinMax    that range pass: min/max of the same shares, added to the
//                  per-kernel keys with atomic max.
constexpr int kHistCluster = 0, kHistFlat = 1, kHistMinMax = 2;

template <int D, bool ADAPTIVE, int MODE = kHistCluster, int HW = kHistLsu, typename T = float>
__device__ __forceinline__ void hist_group(const Geom &g, const T *__restrict__ in,
                                           const uint32_t *__restrict__ keys,
                                           const float *__restrict__ d_clip,
                                           uint32_t *__restrict__ hist, float *__restrict__ lut,
                                           float *__restrict__ lo_out,
                                           float *__restrict__ scale_out, int64_t item, int G,
                                           int R, uint32_t *sh, int c0 = 0, int c1 = 1,
                                           int nchunks = 1,
                                           uint32_t *__restrict__ tickets = nullptr,
                                           uint32_t *__restrict__ kkeys = nullptr,
                                           const HistTma *htma = nullptr,
                                           TmaRing<kHistTmaStages> *tring = nullptr) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = MODE == kHistCluster ? int(cluster.num_blocks()) : 1;
    const int rank = MODE == kHistCluster ? int(cluster.block_rank()) : 0;
    // this CTA's shares of the rows of every box
    const int sh0 = MODE == kHistCluster ? rank : c0;
    const int sh1 = MODE == kHistCluster ? rank + 1 : c1;
    const int nsh = MODE == kHistCluster ? C : nchunks;
    const int nb = g.nb, P = g.P;
    const int lane = threadIdx.x & 31;
    const Dim &dl = g.d[D - 1];
    // a one-CTA cluster needs only block barriers
    auto csync = [&]() {
        if (MODE == kHistCluster && C > 1) cluster.sync(); else __syncthreads();
    };
    const int n_groups = (dl.n + G - 1) / G;

    // item -> outer kernel coordinates and the group along the last dim
    int kk[kMaxDim];
    int64_t outer = item / n_groups;
    const int grp = int(item - outer * n_groups);
    {
        int64_t r = outer;
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            kk[j] = int(r % g.d[j].n);
            r /= g.d[j].n;
        }
    }
    const int kl0 = grp * G, kl1 = min(kl0 + G, dl.n), GK = kl1 - kl0;
    const int64_t kfirst = outer * dl.n + kl0;   // flat index of the group's first kernel

    // smem: copies [G][P][R], counts [G][P], keys [2G], -lo [G], scale [G], lo [G]
    // (the range pass keeps only the keys and the ranges)
    constexpr bool kKeysOnly = MODE == kHistMinMax;
    uint32_t *cnt = sh + (kKeysOnly ? 0 : size_t(G) * P * R);
    uint32_t *s_keys = cnt + (kKeysOnly ? 0 : size_t(G) * P);
    float *s_nlo = reinterpret_cast<float *>(s_keys + 2 * G);
    float *s_sc = s_nlo + G;
    float *s_lo = s_sc + G;
    {
        uint4 *z = reinterpret_cast<uint4 *>(sh);
        const int nw = kKeysOnly ? 5 * G : int(hist_smem_words(P, R, G));
        for (int i = threadIdx.x; i < nw / 4; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
        for (int i = (nw / 4) * 4 + threadIdx.x; i < nw; i += blockDim.x) sh[i] = 0;
    }

    // outer pieces (dims 0..D-2) and the last-dim extent of the group, in
    // shared memory (the same for every thread)
    __shared__ Pieces pc[kMaxDim + 1];
    if (threadIdx.x < D - 1) pc[threadIdx.x] = footprint_pieces(g.d[threadIdx.x], kk[threadIdx.x]);
    if (threadIdx.x == kMaxDim) pc[kMaxDim] = footprint_pieces(dl, kl0);   // one-kernel groups
    __syncthreads();
    int nsub = 1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) nsub *= pc[j].n;
    int xlo = dl.s, xhi = 0;
    for (int k = kl0; k < kl1; ++k) {
        const Foot f = footprint(dl, k);
        xlo = min(xlo, f.lo);
        xhi = max(xhi, f.hi);
    }
    int64_t stride[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) stride[j] = g.d[j].stride;
    const bool tiled = (dl.s & 3) == 0;   // every row starts at the same alignment
    // Visits every box: fn(box_lo, box_len, weight, r0, r1, kgfix).  With one
    // kernel in the group the last dimension is cut into its constant-
    // multiplicity pieces too, so every voxel of a box adds `weight` to
    // kernel kgfix = 0; otherwise kgfix = -1 and the boxes are segments of
    // the group's extent whose voxels are assigned to kernels quad by quad.
    const bool single = GK == 1;
    const Pieces &pl = pc[kMaxDim];
    auto for_boxes = [&](auto &&fn) {
        for (int sb = 0; sb < nsub; ++sb) {
            int box_lo[kMaxDim], len[kMaxDim];
            int w = 1, rest = sb, rows = 1;
#pragma unroll
            for (int j = D - 2; j >= 0; --j) {
                const int i = rest % pc[j].n;
                rest /= pc[j].n;
                box_lo[j] = pc[j].a[i];
                len[j] = pc[j].e[i] - pc[j].a[i];
                w *= pc[j].m[i];
                rows *= len[j];
            }
            const int r0 = int((int64_t(rows) * sh0) / nsh);
            const int r1 = int((int64_t(rows) * sh1) / nsh);
            if (r1 <= r0) continue;
            // [a, e) along the last dim in ceil((e - a) / kHistSeg) segments of
            // about equal length, inner boundaries on 16-byte boundaries
            // (every segment fits a walk's 512-element row: head + length)
            auto segments = [&](int a, int e, int wt, int kgfix) {
                const int n = (e - a + kHistSeg - 1) / kHistSeg;
                int x0 = a;
                for (int i = 1; i <= n; ++i) {
                    const int x1 = i == n ? e : ((a + int((int64_t(e - a) * i) / n)) & ~3);
                    if (x1 > x0) {
                        box_lo[D - 1] = x0;
                        len[D - 1] = x1 - x0;
                        fn(box_lo, len, wt, r0, r1, kgfix);
                    }
                    x0 = x1;
                }
            };
            if (single) {
                for (int i = 0; i < pl.n; ++i) segments(pl.a[i], pl.e[i], w * pl.m[i], 0);
            } else {
                segments(xlo, xhi, w, -1);
            }
        }
    };
    struct NoRow {};
    auto no_row = [](const int *, NoRow &) {};
    // every voxel of rows [r0, r1) of a box, one per thread at a time:
    // fn(x along the last dim, value)
    auto for_voxels = [&](const int *box_lo, const int *len, int r0, int r1, auto &&fn) {
        const int L = len[D - 1];
        const int64_t total = int64_t(r1 - r0) * L;
        for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
            const int r = r0 + int(t / L), e = int(t % L);
            int rest = r;
            int64_t a = box_lo[D - 1] + e;
#pragma unroll
            for (int j = D - 2; j >= 0; --j) {
                int rr;
                rest = small_div(rest, len[j], rr);
                a += int64_t(box_lo[j] + rr) * stride[j];
            }
            fn(box_lo[D - 1] + e, ld1(in + a));
        }
    };

    // rows [r0, r1) of a box in fixed quad slots: walk_tile, the cp.async
    // ring, or TMA tiles (boxes that fit the tile's width)
    float4 *ring = reinterpret_cast<float4 *>(
        sh + hist_ring_offset_words(kKeysOnly ? 5 * size_t(G) : hist_smem_words(P, R, G)));
    // whole-quad boxes: every slot of every row is a full quad (head 0 and
    // L = 4 * LPR * QL with QL = kHistQmax), walked without per-slot tests
    // and counted by quad_full
    auto whole_quads = [&](const int *len, const TileShape &ts) {
        return ts.head == 0 && ts.QL == kHistQmax && len[D - 1] == 4 * ts.LPR * kHistQmax;
    };
    auto walk_full = [&](auto sd_tag, const int *box_lo, const int *len, int r0, int r1,
                         const TileShape &ts, auto &&slot, auto &&quad_full) {
        using SD = typename decltype(sd_tag)::type;
        if constexpr (HW == kHistRing) {
            walk_tile_async<D, kHistQmax, kHistStages, NoRow, SD, true>(in, stride, box_lo, len, r0, r1,
                                                                        ts, ring, slot, no_row, quad_full);
        } else {
            walk_tile<D, kHistQmax, 4, NoRow, SD, false, false, true>(in, nullptr, stride, box_lo, len, r0,
                                                                      r1, ts, false, slot, no_row,
                                                                      quad_full);
        }
    };
    auto walk = [&](auto sd_tag, const int *box_lo, const int *len, int r0, int r1,
                    const TileShape &ts, auto &&slot, auto &&quad) {
        using SD = typename decltype(sd_tag)::type;
        if constexpr (HW == kHistTma) {
            if ((box_lo[D - 1] & 3) + len[D - 1] <= htma->bx) {
                walk_tile_tma<D, kHistTmaStages, kHistTileFloats / 1024, kHistTmaStage, SD>(
                    htma->map, box_lo, len, r0, r1, htma->bx, htma->by, *tring, slot,
                    [&](const SD &sd, int i, const float4 &v) {
                        NoRow nr;
                        quad(nr, sd, i, v, v, int64_t(0));
                    });
                return;
            }
        }
        if constexpr (HW == kHistRing) {
            walk_tile_async<D, kHistQmax, kHistStages, NoRow, SD>(in, stride, box_lo, len, r0, r1, ts,
                                                                  ring, slot, no_row, quad);
        } else {
            walk_tile<D, kHistQmax, 4, NoRow, SD, false>(in, nullptr, stride, box_lo, len, r0, r1, ts,
                                                         false, slot, no_row, quad);
        }
    };

    // ---- phase 1 (adaptive range only): min/max of every kernel of the group
    if (ADAPTIVE && MODE != kHistFlat && (MODE == kHistMinMax || kkeys == nullptr)) {
        auto key_min = [&](int kg, float v) { atomicMax(&s_keys[2 * kg], ~float_key(v)); };
        auto key_max = [&](int kg, float v) { atomicMax(&s_keys[2 * kg + 1], float_key(v)); };
        auto slow_elem = [&](int x, float v) {
            const Targets tg = last_targets(dl, x, kl0, kl1);
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (t < tg.n) {
                    key_min(tg.kg[t], v);
                    key_max(tg.kg[t], v);
                }
        };
        for_boxes([&](const int *box_lo, const int *len, int, int r0, int r1, int kgfix) {
            const int L = len[D - 1], xs = box_lo[D - 1];
            if (tiled) {
                const TileShape ts = tile_shape(L, xs & 3, blockDim.x, kHistQmax);
                struct MSlot {
                    int kg;          // kernel of the group, -1: per-voxel path
                    int q0;          // element offset of the slot in the row
                    bool full;       // all four voxels inside the box
                };
                float mn[kHistQmax], mx[kHistQmax];
                int tk[kHistQmax];
#pragma unroll
                for (int i = 0; i < kHistQmax; ++i) {
                    mn[i] = INFINITY;
                    mx[i] = -INFINITY;
                    tk[i] = -1;
                }
                auto slot = [&](int i, int e0) {
                    MSlot sd{-1, e0, e0 >= 0 && e0 + 4 <= L};
                    if (kgfix >= 0) {
                        sd.kg = kgfix;
                    } else if (sd.full) {
                        // the targets change monotonically along x, so equal
                        // single targets at both ends hold for the whole quad
                        const Targets t0 = last_targets(dl, xs + e0, kl0, kl1);
                        const Targets t1 = last_targets(dl, xs + e0 + 3, kl0, kl1);
                        if (t0.n == 1 && t1.n == 1 && t1.kg[0] == t0.kg[0]) sd.kg = t0.kg[0];
                    }
                    tk[i] = sd.full ? sd.kg : -1;
                    return sd;
                };
                auto quad = [&](NoRow &, const MSlot &sd, int i, const float4 &v, const float4 &, int64_t) {
                    if (sd.full && sd.kg >= 0) {
                        mn[i] = min3f(mn[i], v.x, v.y);
                        mn[i] = min3f(mn[i], v.z, v.w);
                        mx[i] = max3f(mx[i], v.x, v.y);
                        mx[i] = max3f(mx[i], v.z, v.w);
                    } else {
                        const float vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (sd.q0 + e < 0 || sd.q0 + e >= L) continue;
                            if (sd.kg >= 0) {
                                key_min(sd.kg, vals[e]);
                                key_max(sd.kg, vals[e]);
                            } else {
                                slow_elem(xs + sd.q0 + e, vals[e]);
                            }
                        }
                    }
                };
                if (HW != kHistTma && kgfix >= 0 && whole_quads(len, ts)) {
                    auto quad_full = [&](NoRow &, const MSlot &, int i, const float4 &v, const float4 &,
                                         int64_t) {
                        mn[i] = min3f(mn[i], v.x, v.y);
                        mn[i] = min3f(mn[i], v.z, v.w);
                        mx[i] = max3f(mx[i], v.x, v.y);
                        mx[i] = max3f(mx[i], v.z, v.w);
                    };
                    walk_full(Tag<MSlot>{}, box_lo, len, r0, r1, ts, slot, quad_full);
                } else {
                    walk(Tag<MSlot>{}, box_lo, len, r0, r1, ts, slot, quad);
                }
                // warp-aggregated: one pair of shared atomics per warp and
                // target kernel (256 threads' atomics on one key serialise)
#pragma unroll
                for (int i = 0; i < kHistQmax; ++i) {
                    const bool has = tk[i] >= 0 && mn[i] <= mx[i];
                    const uint32_t kmn = has ? ~float_key(mn[i]) : 0u;
                    const uint32_t kmx = has ? float_key(mx[i]) : 0u;
                    unsigned pend = __ballot_sync(0xffffffffu, has);
                    while (pend) {
                        const int leader = __ffs(pend) - 1;
                        const int t = __shfl_sync(0xffffffffu, tk[i], leader);
                        const bool mine = has && tk[i] == t;
                        pend &= ~__ballot_sync(0xffffffffu, mine);
                        const uint32_t a = __reduce_max_sync(0xffffffffu, mine ? kmn : 0u);
                        const uint32_t b = __reduce_max_sync(0xffffffffu, mine ? kmx : 0u);
                        if (lane == leader) {
                            atomicMax(&s_keys[2 * t], a);
                            atomicMax(&s_keys[2 * t + 1], b);
                        }
                    }
                }
            } else {
                // rows at varying alignments: voxel by voxel
                for_voxels(box_lo, len, r0, r1, [&](int x, float v) {
                    if (kgfix >= 0) {
                        key_min(kgfix, v);
                        key_max(kgfix, v);
                    } else {
                        slow_elem(x, v);
                    }
                });
            }
        });
        if (MODE == kHistMinMax) {
            __syncthreads();
            for (int kg = threadIdx.x; kg < GK; kg += blockDim.x) {
                atomicMax(&kkeys[2 * (kfirst + kg)], s_keys[2 * kg]);
                atomicMax(&kkeys[2 * (kfirst + kg) + 1], s_keys[2 * kg + 1]);
            }
            return;
        }
        csync();   // every CTA's keys are complete
        for (int kg = threadIdx.x; kg < GK; kg += blockDim.x) {
            uint32_t a = 0, b = 0;
            for (int c = 0; c < C; ++c) {
                const uint32_t *rk = C > 1 ? cluster.map_shared_rank(s_keys, c) : s_keys;
                a = max(a, rk[2 * kg]);
                b = max(b, rk[2 * kg + 1]);
            }
            float lo, hi;
            keys_to_range(a, b, lo, hi);
            s_lo[kg] = lo;
            s_nlo[kg] = -lo;
            s_sc[kg] = range_scale(lo, hi, nb);
        }
    } else if (ADAPTIVE) {   // a range pass (flat, or k_range_kernels) left the per-kernel keys
        for (int kg = threadIdx.x; kg < GK; kg += blockDim.x) {
            float lo, hi;
            keys_to_range(__ldcg(kkeys + 2 * (kfirst + kg)), __ldcg(kkeys + 2 * (kfirst + kg) + 1), lo, hi);
            s_lo[kg] = lo;
            s_nlo[kg] = -lo;
            s_sc[kg] = range_scale(lo, hi, nb);
        }
    } else {
        float lo, hi;
        if (g.has_range) {
            lo = g.range_lo;
            hi = g.range_hi;
        } else {
            keys_to_range(__ldcg(keys), __ldcg(keys + 1), lo, hi);   // L2: may be this launch's
        }
        for (int kg = threadIdx.x; kg < GK; kg += blockDim.x) {
            s_lo[kg] = lo;
            s_nlo[kg] = -lo;
            s_sc[kg] = range_scale(lo, hi, nb);
        }
    }
    __syncthreads();

    // ---- phase 2: histogram sweep.  Copies: the lanes of a warp that read the
    // same quad position of different rows (and so may add to the same kernel)
    // take different copies: with LPR lanes per row, lane = r * LPR + gl adds
    // to copy (r + gl * 32 / LPR) mod R.  With ZC the voxels in bin 0 are
    // counted in a register per quad slot and added once per box (measured
    // slower on count data than one reduction per voxel: off).
    {
        constexpr bool ZC = false;
        const uint32_t sh_base = uint32_t(__cvta_generic_to_shared(sh));
        const uint32_t r4 = uint32_t(4 * R);
        const uint32_t lane_off = 4u * uint32_t(lane & (R - 1));
        const uint32_t kstride = uint32_t(P) * r4;   // bytes per kernel's copies
        const float iqk = g.iqk, qkf = g.qkf;
        // copy offset of this lane when LPR lanes share a row (LPR a power of
        // two <= 32; 0: lane order)
        auto copy_off = [&](int lpr) {
            if (lpr <= 1 || lpr > 32 || (lpr & (lpr - 1))) return lane_off;
            return 4u * uint32_t(((lane / lpr) + (lane % lpr) * (32 / lpr)) & (R - 1));
        };
        // lanes per row of the walk a box takes
        auto box_lpr = [&](const int *box_lo, const int *len, const TileShape &ts) {
            if constexpr (HW == kHistTma) {
                if ((box_lo[D - 1] & 3) + len[D - 1] <= htma->bx) return htma->bx / 4;
            }
            return ts.LPR;
        };
        auto add_elem = [&](int x, float v, uint32_t w) {
            const Targets tg = last_targets(dl, x, kl0, kl1);
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (t < tg.n) {
                    const int kg = tg.kg[t];
                    const uint32_t b = qbits1(v, s_nlo[kg], s_sc[kg], iqk, qkf);
                    red_shared_add(sh_base + uint32_t(kg) * kstride + lane_off + (b - kBinBias) * r4,
                                   w * uint32_t(tg.m[t]));
                }
        };
        // one voxel of a whole quad: bin 0 counted in z (ZC), else reduced
        auto add_bits = [&](uint32_t bits, uint32_t base, uint32_t w, uint32_t &z) {
            if (ZC) {
                if (bits == kBinBias) {
                    z += 1u;
                    return;
                }
            }
            red_shared_add(bits * r4 + base, w);
        };
        for_boxes([&](const int *box_lo, const int *len, int w, int r0, int r1, int kgfix) {
            const int L = len[D - 1], xs = box_lo[D - 1];
            const uint32_t wu = uint32_t(w);
            if (tiled && kgfix >= 0) {
                // every voxel of the box goes to kernel kgfix with weight w
                const TileShape ts = tile_shape(L, xs & 3, blockDim.x, kHistQmax);
                struct FSlot {
                    int q0;          // element offset of the slot in the row
                    bool full;       // all four voxels inside the box
                };
                const uint32_t base = sh_base + uint32_t(kgfix) * kstride +
                                      copy_off(box_lpr(box_lo, len, ts)) - kBinBias * r4;
                const float2 n2 = make_float2(s_nlo[kgfix], s_nlo[kgfix]);
                const float2 s2 = make_float2(s_sc[kgfix], s_sc[kgfix]);
                uint32_t z = 0;
                auto slot = [&](int, int e0) { return FSlot{e0, e0 >= 0 && e0 + 4 <= L}; };
                auto quad = [&](NoRow &, const FSlot &sd, int, const float4 &v, const float4 &, int64_t) {
                    const uint2 b01 = qbits2(make_float2(v.x, v.y), n2, s2, iqk, qkf);
                    const uint2 b23 = qbits2(make_float2(v.z, v.w), n2, s2, iqk, qkf);
                    if (sd.full) {
                        add_bits(b01.x, base, wu, z);
                        add_bits(b01.y, base, wu, z);
                        add_bits(b23.x, base, wu, z);
                        add_bits(b23.y, base, wu, z);
                    } else {
                        const uint32_t bits[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (sd.q0 + e >= 0 && sd.q0 + e < L) red_shared_add(bits[e] * r4 + base, wu);
                    }
                };
                if (HW != kHistTma && whole_quads(len, ts)) {
                    auto quad_full = [&](NoRow &, const FSlot &, int, const float4 &v, const float4 &,
                                         int64_t) {
                        const uint2 b01 = qbits2(make_float2(v.x, v.y), n2, s2, iqk, qkf);
                        const uint2 b23 = qbits2(make_float2(v.z, v.w), n2, s2, iqk, qkf);
                        add_bits(b01.x, base, wu, z);
                        add_bits(b01.y, base, wu, z);
                        add_bits(b23.x, base, wu, z);
                        add_bits(b23.y, base, wu, z);
                    };
                    walk_full(Tag<FSlot>{}, box_lo, len, r0, r1, ts, slot, quad_full);
                } else {
                    walk(Tag<FSlot>{}, box_lo, len, r0, r1, ts, slot, quad);
                }
                if (ZC && z) red_shared_add(kBinBias * r4 + base, z * wu);
            } else if (tiled) {
                // groups of kernels: a slot's quad goes to one kernel (with
                // one multiplicity) when its first and last voxel do -- the
                // targets change monotonically along x -- else voxel by voxel
                const TileShape ts = tile_shape(L, xs & 3, blockDim.x, kHistQmax);
                const uint32_t coff = copy_off(box_lpr(box_lo, len, ts));
                struct HSlot {
                    uint32_t base;   // copy address of bin 0 minus the bias; ~0: per-voxel path
                    uint32_t w;      // weight of the slot's voxels
                    int q0;          // element offset of the slot in the row
                    int kg;          // the slot's kernel (adaptive range constants)
                };
                // bin-0 counts per slot (ZC), with the slot's address and weight
                uint32_t zc[kHistQmax], zbase[kHistQmax], zw[kHistQmax];
#pragma unroll
                for (int i = 0; i < kHistQmax; ++i) {
                    zc[i] = 0;
                    zbase[i] = 0xffffffffu;
                    zw[i] = 0;
                }
                auto slot = [&](int i, int e0) {
                    HSlot sd{0xffffffffu, 0u, e0, 0};
                    if (e0 < 0 || e0 + 4 > L) return sd;
                    const Targets t0 = last_targets(dl, xs + e0, kl0, kl1);
                    const Targets t1 = last_targets(dl, xs + e0 + 3, kl0, kl1);
                    if (t0.n != 1 || t1.n != 1 || t1.kg[0] != t0.kg[0] || t1.m[0] != t0.m[0]) return sd;
                    sd.base = sh_base + uint32_t(t0.kg[0]) * kstride + coff - kBinBias * r4;
                    sd.w = wu * uint32_t(t0.m[0]);
                    sd.kg = t0.kg[0];
#pragma unroll
                    for (int j = 0; j < kHistQmax; ++j)
                        if (j == i) {
                            zbase[j] = sd.base;
                            zw[j] = sd.w;
                        }
                    return sd;
                };
                const float2 gnl = make_float2(s_nlo[0], s_nlo[0]), gsc = make_float2(s_sc[0], s_sc[0]);
                auto quad = [&](NoRow &, const HSlot &sd, int i, const float4 &v, const float4 &, int64_t) {
                    if (sd.base != 0xffffffffu) {
                        float2 n2 = gnl, s2 = gsc;
                        if (ADAPTIVE) {
                            n2 = make_float2(s_nlo[sd.kg], s_nlo[sd.kg]);
                            s2 = make_float2(s_sc[sd.kg], s_sc[sd.kg]);
                        }
                        const uint2 b01 = qbits2(make_float2(v.x, v.y), n2, s2, iqk, qkf);
                        const uint2 b23 = qbits2(make_float2(v.z, v.w), n2, s2, iqk, qkf);
                        uint32_t z = 0;
                        add_bits(b01.x, sd.base, sd.w, z);
                        add_bits(b01.y, sd.base, sd.w, z);
                        add_bits(b23.x, sd.base, sd.w, z);
                        add_bits(b23.y, sd.base, sd.w, z);
                        if (ZC) {
#pragma unroll
                            for (int j = 0; j < kHistQmax; ++j)
                                if (j == i) zc[j] += z;
                        }
                    } else {
                        const float vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (sd.q0 + e >= 0 && sd.q0 + e < L) add_elem(xs + sd.q0 + e, vals[e], wu);
                    }
                };
                walk(Tag<HSlot>{}, box_lo, len, r0, r1, ts, slot, quad);
                if (ZC) {
#pragma unroll
                    for (int i = 0; i < kHistQmax; ++i)
                        if (zc[i]) red_shared_add(kBinBias * r4 + zbase[i], zc[i] * zw[i]);
                }
            } else {
                // rows at varying alignments: voxel by voxel
                for_voxels(box_lo, len, r0, r1, [&](int x, float v) {
                    if (kgfix >= 0) {
                        const uint32_t b = qbits1(v, s_nlo[kgfix], s_sc[kgfix], iqk, qkf);
                        red_shared_add(sh_base + uint32_t(kgfix) * kstride + lane_off + (b - kBinBias) * r4, wu);
                    } else {
                        add_elem(x, v, wu);
                    }
                });
            }
        });
    }
    __syncthreads();

    // ---- phase 3: sum the copies, fold the padded indices
    sum_copies(sh, cnt, GK, P, R, nb);
    if (MODE == kHistFlat) {
        __syncthreads();
        // add this CTA's counts to the item's global histograms
        for (int t = threadIdx.x; t < GK * nb; t += blockDim.x) {
            const int kg = t / nb, j = t - kg * nb;
            const uint32_t c = cnt[size_t(kg) * P + j];
            if (c) atomicAdd(&hist[(kfirst + kg) * nb + j], c);
        }
        __threadfence();   // every thread's counts before the ticket
        __syncthreads();
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            const uint32_t done = uint32_t(c1 - c0);   // shares of this item done here
            s_last = (atomicAdd(&tickets[item], done) + done == uint32_t(nchunks));
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        // the last contributor: every share's counts are in the global histograms
        for (int t = threadIdx.x; t < GK * nb; t += blockDim.x) {
            const int kg = t / nb, j = t - kg * nb;
            cnt[size_t(kg) * P + j] = __ldcg(hist + (kfirst + kg) * nb + j);
        }
        for (int kg = threadIdx.x; kg < GK; kg += blockDim.x) {
            lo_out[kfirst + kg] = s_lo[kg];
            scale_out[kfirst + kg] = s_sc[kg];
        }
        __syncthreads();
        build_luts(cnt, P, GK, nb, g.LS, g.V, load_clip(d_clip, g.clip), lut, kfirst, 1);
        return;
    }
    csync();   // every CTA's counts are complete
    merge_and_build(g, sh, cnt, s_lo, s_sc, GK, C, rank, hist, lut, lo_out, scale_out, kfirst, d_clip);
}

}  // namespace mclahe
