// map_impl.cuh -- intensity mapping of one inter-kernel cell by multilinear
// interpolation (Sec. III.C, Eq. (12)-(13); Algorithm 1, the interpolation
// loop).  Included by the per-volume launcher (k_map.cu) and the batched
// launcher (batch.cu).
//
// Tables and ranges are read through L2 (ld.global.cg), so a batched launch
// may map a volume whose tables were written earlier in the same launch.
//
// Voxels that share the same 2^D nearest kernels form an inter-kernel cell
// (the dotted regions of Fig. 2).  A CTA takes one cell (or a chunk of its
// rows), stages the 2^D neighbouring mapping tables in shared memory, then
// streams its voxels with 128-bit loads and stores, four quads in flight per
// thread.  Each voxel takes its bin under every neighbour's range (one bin for
// a global range), reads the tables at those bins and blends them with the
// Lagrange coefficients
//   out = sum_i prod_j w_{i_j, j} * lut[k0 + i][bin_{k0+i}(x)],
//   w_{1,j} = d_{j0} / b_j,  w_{0,j} = 1 - w_{1,j},
// where d_{j0} = (x_j + p_j0) - (k0_j b_j + (b_j - 1) / 2) is the distance to
// the lower kernel's centre: w_{1,j} = m / (2 b_j) with the integer
// m = 2 (x_j + p_j0) - (b_j - 1) - 2 b_j k0_j in [0, 2 b_j).  The sums over
// the corners run on packed f32x2 pairs.
//
// Shared-memory layout (bank-conflict-free gathers).  The bins of the voxels
// of a warp are unrelated, so 32 lanes reading the same corner of 32 random
// bins would hit random banks.  Each table index therefore owns one 128-byte
// row of 32 slots, slot s holding corner s mod 2^D (32 / 2^D copies of the
// 2^D corner values), and lane l reads, at step t, the corner (t + l) mod 2^D
// from copy l / 2^D: at every step the 32 lanes touch 32 different banks
// whatever their bins.  With a global range the reads are 16-byte corner
// quads and the rule applies per 8-lane phase.  The lane-dependent corner
// order is undone by per-lane rotated copies of the corner ranges and
// weights, built once per CTA and per row.  Tables too large for this layout
// (more than 1280 entries) use one row of 2^D values per index.
//
// Every table has lut[.][0] = 0 (the normalisation subtracts the first CDF
// value), so with a global range a voxel in bin 0 maps to exactly 0 and its
// gathers are skipped (count data are mostly zeros).
#pragma once

#include "mclahe_internal.cuh"
#include "tma.cuh"

namespace mclahe {

// How a CTA streams its cell's voxels:
//   kWalkLsu   fixed quad slots with 128-bit loads (walk_tile);
//   kWalkRing  the same slots through a cp.async row ring (walk_tile_async);
//   kWalkTma   box tiles of the cell through TMA: a ring of kTmaStages tiles
//              in shared memory, loaded by one thread with cp.async.bulk.tensor
//              and completed on mbarriers; each thread maps its quads of a
//              tile in place and one thread stores the tile back with a TMA
//              store.  Cells whose rows are short (a few sectors of a 128-byte
//              line) cost the load/store unit a wavefront per line per request
//              in the other walks; TMA moves whole boxes instead.
constexpr int kWalkLsu = 0, kWalkRing = 1, kWalkTma = 2;
constexpr int kTmaStages = 4;
constexpr int kTmaTileFloats = 2048;   // at most; 2 quads per consumer thread
constexpr int kTmaConsumers = 256;     // mapping threads; one more warp moves the tiles
constexpr uint32_t kTmaWaitLimit = 1u << 22;

// The tile box and tensor maps of a TMA mapping launch.  The box spans the
// whole cell row (bx = b of the last dim), by voxels along dim D-2, bz along
// dim D-3 (4-D only) and one slice along dim 0; tiles step along dim 0 first.
struct MapTma {
    const CUtensorMap *in, *out;
    int bx, by, bz;
    uint32_t *status;   // workspace status word (a wait that gave up)
};

// Rotate an array of N values left by r (0 <= r < N, N a power of two) with
// log2(N) levels of selects, keeping every index static.
template <int N, typename T>
__device__ __forceinline__ void rotate_left(T (&a)[N], int r) {
#pragma unroll
    for (int sh = 1; sh < N; sh <<= 1) {
        const bool on = (r & sh) != 0;
        T t[N];
#pragma unroll
        for (int i = 0; i < N; ++i) t[i] = on ? a[(i + sh) & (N - 1)] : a[i];
#pragma unroll
        for (int i = 0; i < N; ++i) a[i] = t[i];
    }
}

// The replicated layout needs 128 bytes per table index.
__host__ __device__ inline bool map_repl_fits(int P) { return size_t(P) * 128 <= 160 * 1024; }
__host__ __device__ inline size_t map_table_bytes(int D, int P) {
    return map_repl_fits(P) ? size_t(P) * 128 : (size_t(1) << D) * size_t(P) * sizeof(float);
}
// Rows of 3- and 4-D cells stream through a cp.async ring (walk_tile_async):
// kMapStages row stages of up to 4 quads per thread of a 256-thread CTA.
constexpr int kMapStages = 3;
__host__ __device__ inline size_t map_ring_bytes(int D) {
    return D >= 3 ? size_t(kMapStages) * 4 * 256 * 16 : 0;
}
__host__ __device__ inline size_t map_smem_for(int D, int P, bool ring = true) {
    return ((map_table_bytes(D, P) + 15) & ~size_t(15)) + (ring ? map_ring_bytes(D) : 0);
}
// The DOT form of 3- and 4-D cells streams the volume and the upstream
// gradient through two rings of kDotStages row stages each.
constexpr int kDotStages = 2;
__host__ __device__ inline size_t dot_smem_for(int D, int P) {
    return ((map_table_bytes(D, P) + 15) & ~size_t(15)) +
           (D >= 3 ? 2 * size_t(kDotStages) * 4 * 256 * 16 : 0);
}

__device__ __forceinline__ void sts128(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// DOT: instead of storing the mapped voxels, the CTA's threads accumulate
// sum_v gout[v] * mapped(v) over their voxels (x and gout read together with
// per-thread loads) into *dot as a compensated (Kahan) float pair (sum,
// correction); the tables `lut` are then whatever per-kernel tables the caller
// interpolates (the clip-limit gradient uses d lut / dT).
template <int D, bool ADAPTIVE, bool REPL, int WALK = kWalkRing, bool DOT = false,
          typename T = float>
__device__ __forceinline__ void map_cell(const Geom &g, const T *__restrict__ in,
                                         float *__restrict__ out, const float *__restrict__ lut,
                                         const float *__restrict__ lo_k,
                                         const float *__restrict__ scale_k, int64_t cell, int chunk,
                                         int chunks, float *tab, const MapTma *tma = nullptr,
                                         int chunk_end = -1, const float *__restrict__ gout = nullptr,
                                         float2 *dot = nullptr) {
    // rows [R * chunk / chunks, R * chunk_end / chunks) of the cell (chunk_end
    // defaults to chunk + 1)
    if (chunk_end < 0) chunk_end = chunk + 1;
    constexpr bool RING = WALK == kWalkRing;
    constexpr int NC = 1 << D;          // corners
    constexpr int NO = 1 << (D - 1);    // corners over dims 0..D-2
    constexpr int NQ = NC >= 4 ? NC / 4 : 1;   // 16-byte corner quads per index
    constexpr uint32_t RSB = REPL ? 128u : uint32_t(4 * NC);   // bytes per table index
    __shared__ float s_nlo[NC], s_sc[NC];
    const int P = g.P, LS = g.LS;
    const int lane = threadIdx.x & 31;

    int cc[kMaxDim];
    {
        int64_t r = cell;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            cc[j] = int(r % (g.d[j].n - 1));
            r /= (g.d[j].n - 1);
        }
    }
    // kernel index of corner i (bit D-1-d of i = side along dim d)
    int64_t kbase = 0, kstr[kMaxDim];
    {
        int64_t st = 1;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            kstr[d] = st;
            kbase += int64_t(cc[d]) * st;
            st *= g.d[d].n;
        }
    }
    auto corner_kernel = [&](int i) {
        int64_t k = kbase;
#pragma unroll
        for (int d = 0; d < D; ++d) k += ((i >> (D - 1 - d)) & 1) ? kstr[d] : 0;
        return k;
    };

    // stage the corner tables
    if (REPL) {
        if (NC >= 4) {
            // task (j, q): corners 4q..4q+3 of index j into every copy's quad q
            // AHR: slot s holds corner s mod NC.  GHR: quad q holds the corners
            // (outer 2q, side 0), (outer 2q + 1, side 0), (2q, side 1),
            // (2q + 1, side 1), so that one packed FMA takes the two outer
            // corners' weights at once.
            constexpr int P1 = ADAPTIVE ? 2 : 1, P2 = ADAPTIVE ? 1 : 2;
            for (int t = threadIdx.x; t < P * NQ; t += blockDim.x) {
                const int j = t / NQ, q = t - j * NQ;
                const float4 v = make_float4(__ldcg(lut + corner_kernel(4 * q) * LS + j),
                                             __ldcg(lut + corner_kernel(4 * q + P2) * LS + j),
                                             __ldcg(lut + corner_kernel(4 * q + P1) * LS + j),
                                             __ldcg(lut + corner_kernel(4 * q + 3) * LS + j));
#pragma unroll
                for (int a = 0; a < 8 / NQ; ++a) sts128(tab + j * 32 + (a * NQ + q) * 4, v);
            }
        } else {
            for (int j = threadIdx.x; j < P; j += blockDim.x) {
                const float c0 = __ldcg(lut + corner_kernel(0) * LS + j);
                const float c1 = __ldcg(lut + corner_kernel(1) * LS + j);
#pragma unroll
                for (int a = 0; a < 8; ++a) sts128(tab + j * 32 + a * 4, make_float4(c0, c1, c0, c1));
            }
        }
    } else {
        for (int t = threadIdx.x; t < NC * P; t += blockDim.x) {
            const int j = t / NC, i = t - j * NC;
            // GHR quads hold (2q, 0), (2q + 1, 0), (2q, 1), (2q + 1, 1), as above
            const int c = (ADAPTIVE || NC < 4) ? i : ((i & ~3) | ((i & 1) << 1) | ((i >> 1) & 1));
            tab[t] = __ldcg(lut + corner_kernel(c) * LS + j);
        }
    }
    if (threadIdx.x < NC) {
        const int64_t k = corner_kernel(threadIdx.x);
        s_nlo[threadIdx.x] = -__ldcg(lo_k + k);
        s_sc[threadIdx.x] = __ldcg(scale_k + k);
    }

    int box_lo[kMaxDim], len[kMaxDim];
    int64_t stride[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        int a, b;
        cell_range(g.d[j], cc[j], a, b);
        box_lo[j] = a;
        len[j] = b - a;
        stride[j] = g.d[j].stride;
    }
    int R = 1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) R *= len[j];
    const int r0 = int((int64_t(R) * chunk) / chunks);
    const int r1 = int((int64_t(R) * chunk_end) / chunks);
    __syncthreads();

    // per-dim weight constants: w1 = float(2 x + mb_j) * inv2b_j
    float inv2b[kMaxDim];
    int mb[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Dim &dj = g.d[j];
        inv2b[j] = 1.0f / float(2 * dj.b);
        mb[j] = 2 * dj.p0 - (dj.b - 1) - 2 * dj.b * cc[j];
    }
    const uint32_t tab_s = uint32_t(__cvta_generic_to_shared(tab));
    const float iqk = g.iqk, qkf = g.qkf;

    // lane rotation (REPL): AHR reads corner (t + rot) mod NC at step t;
    // GHR reads quad (s + rot) mod NQ at step s from copy (l / NQ) mod (8 / NQ)
    const int rot = REPL ? (ADAPTIVE ? (lane & (NC - 1)) : (lane & (NQ - 1))) : 0;

    // AHR: per step pair the two corners' ranges, per step the table address
    constexpr int NA = ADAPTIVE ? NC : 1;
    float2 anlo[ADAPTIVE ? NC / 2 : 1], asc[ADAPTIVE ? NC / 2 : 1];
    uint32_t cbase[NA];
    // AHR: the 1/qk of the quantiser folded into the corners' scales when
    // that is exact for all of them (the same decision in every thread)
    bool fold = false;
    if (ADAPTIVE) {
        float nl[NA], sc[NA];
        fold = true;
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            const int c = REPL ? ((t + rot) & (NC - 1)) : t;
            nl[t] = s_nlo[c];
            sc[t] = s_sc[c];
            fold = fold && fold_exact(sc[t], g.qkf);
            const int slot = REPL ? ((lane & ~(NC - 1) & 31) | c) : c;
            cbase[t] = tab_s + 4u * uint32_t(slot) - kBinBias * RSB;
        }
        if (fold) {
#pragma unroll
            for (int t = 0; t < NA; ++t) sc[t] *= g.iqk;
        }
#pragma unroll
        for (int t = 0; t < NA / 2; ++t) {
            anlo[t] = make_float2(nl[2 * t], nl[2 * t + 1]);
            asc[t] = make_float2(sc[2 * t], sc[2 * t + 1]);
        }
    }
    const float gnlo = s_nlo[0], gsc = s_sc[0];
    // GHR: table address of step s
    uint32_t gbase[NQ];
#pragma unroll
    for (int s = 0; s < NQ; ++s) {
        uint32_t off;
        if (REPL) {
            if (NC >= 4) {
                const int qd = (s + rot) & (NQ - 1);
                const int copy = (lane / NQ) & ((8 / NQ) - 1);
                off = 16u * uint32_t(copy * NQ + qd);
            } else {
                off = 8u * uint32_t(lane & 15);
            }
        } else {
            off = 16u * uint32_t(s);
        }
        gbase[s] = tab_s + off - kBinBias * RSB;
    }

    const int L = len[D - 1];
    const int xl = box_lo[D - 1];
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);
    const float inv2b_l = inv2b[D - 1];
    const int mb_l = mb[D - 1];

    // Per-row state: the outer weights in the order this lane reads them.
    //   AHR: w[t] = weight over dims 0..D-2 of corner (t + rot) mod NC, paired;
    //   GHR: (wa[s], wb[s]) = outer weights of the two outer corners of quad
    //        (s + rot) mod NQ (corners 4q..4q+3 = outer 2q, 2q+1 x last 0, 1).
    struct MRow {
        float2 w[ADAPTIVE ? NC / 2 : (NC >= 4 ? NQ : 2)];
    };
    // The outer weight of outer corner o is f0[o_0] * (product over dims
    // 1..D-2, left to right), f0 = (w0, w1) of dim 0: row_weights takes f0
    // as given, so the TMA walk can split off dim 0 (see below).
    auto row_weights = [&](const int *coords, float f0a, float f0b, MRow &st) {
        float wo[NO];
        if constexpr (D >= 2) {
            constexpr int NI = NO / 2;   // corners over dims 1..D-2
            float in_[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) in_[i] = 1.0f;
#pragma unroll
            for (int j = 1; j < D - 1; ++j) {
                const float w1 = float(2 * coords[j] + mb[j]) * inv2b[j];
                const float w0 = 1.0f - w1;
#pragma unroll
                for (int i = 0; i < NI; ++i) in_[i] *= ((i >> (D - 2 - j)) & 1) ? w1 : w0;
            }
#pragma unroll
            for (int o = 0; o < NO; ++o) wo[o] = ((o >> (D - 2)) & 1 ? f0b : f0a) * in_[o & (NI - 1)];
        } else {
            wo[0] = 1.0f;
        }
        if (ADAPTIVE) {
            float a[NA];
#pragma unroll
            for (int c = 0; c < NA; ++c) a[c] = wo[c >> 1];
            if (REPL) rotate_left<NA>(a, rot);
#pragma unroll
            for (int t = 0; t < NA / 2; ++t) st.w[t] = make_float2(a[2 * t], a[2 * t + 1]);
        } else if (NC >= 4) {
            // (outer 2q, outer 2q + 1) weight pairs of the quads, in this lane's order
            float2 pw[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) pw[q] = make_float2(wo[2 * q], wo[2 * q + 1]);
            if (REPL && NQ > 1) rotate_left<NQ>(pw, rot);
#pragma unroll
            for (int q = 0; q < NQ; ++q) st.w[q] = pw[q];
        } else {
            st.w[0] = make_float2(1.0f, 1.0f);
            st.w[1] = st.w[0];
        }
    };
    auto row_fn = [&](const int *coords, int64_t, MRow &st) {
        if constexpr (D >= 2) {
            const float w1 = float(2 * coords[0] + mb[0]) * inv2b[0];
            row_weights(coords, 1.0f - w1, w1, st);
        } else {
            row_weights(coords, 1.0f, 0.0f, st);
        }
    };

    const int rodd = rot & 1;
    const float two_inv2b = 2.0f * inv2b_l;
    // AHR: the step sums (acc.x, acc.y) hold last-dim sides (rodd, 1 - rodd),
    // whose weights at last-dim weight w1 are wab.x * w1 + wab.y and
    // -wab.x * w1 + (1 - wab.y); dwe is their change from one voxel to the next
    const float2 wab = rodd ? make_float2(1.0f, 0.0f) : make_float2(-1.0f, 1.0f);
    const float2 dwe = make_float2(wab.x * two_inv2b, -wab.x * two_inv2b);
    // AHR quad: quantise per corner pair, gather, and weight the two sides
    auto map4a = [&](const MRow &st, const float (&vals)[4], float fbi, float (&res)[4], auto folded) {
        constexpr bool FOLD = decltype(folded)::value;
        const float2 w0 = __ffma2_rn(make_float2(fbi, fbi), make_float2(wab.x, -wab.x),
                                     make_float2(wab.y, 1.0f - wab.y));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float2 acc = make_float2(0.0f, 0.0f);
            const float2 xx = make_float2(vals[e], vals[e]);
#pragma unroll
            for (int t = 0; t < NA / 2; ++t) {
                const uint2 b = FOLD ? qbits2_folded(xx, anlo[t], asc[t], qkf)
                                     : qbits2(xx, anlo[t], asc[t], iqk, qkf);
                const float v0 = lds_f32(b.x * RSB + cbase[2 * t]);
                const float v1 = lds_f32(b.y * RSB + cbase[2 * t + 1]);
                acc = __ffma2_rn(make_float2(v0, v1), st.w[t], acc);
            }
            const float2 we = e == 0 ? w0 : __ffma2_rn(make_float2(float(e), float(e)), dwe, w0);
            res[e] = fmaf(acc.y, we.y, acc.x * we.x);
        }
    };
    // the mapping of the four voxels of a quad (vals) at last-dim weight
    // w1 = fbi + e * two_inv2b for voxel e
    auto map4 = [&](const MRow &st, const float (&vals)[4], float fbi, float (&res)[4]) {
        if constexpr (ADAPTIVE) {
            if (fold)
                map4a(st, vals, fbi, res, std::true_type{});
            else
                map4a(st, vals, fbi, res, std::false_type{});
        } else {
            // GHR: one bin per voxel for all corners
            uint32_t gb[4];
            const float2 nl = make_float2(gnlo, gnlo), sc = make_float2(gsc, gsc);
            const uint2 b01 = qbits2(make_float2(vals[0], vals[1]), nl, sc, iqk, qkf);
            const uint2 b23 = qbits2(make_float2(vals[2], vals[3]), nl, sc, iqk, qkf);
            gb[0] = b01.x;
            gb[1] = b01.y;
            gb[2] = b23.x;
            gb[3] = b23.y;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float w1 = fmaf(float(e), two_inv2b, fbi);
                float a0, a1;   // sums over the outer corners at last-dim side 0 and 1
                if (gb[e] == kBinBias) {
                    // bin 0: every table's first entry is 0, so the voxel maps to 0
                    a0 = 0.0f;
                    a1 = 0.0f;
                } else if (NC >= 4) {
                    float2 acc0 = make_float2(0.0f, 0.0f), acc1 = acc0;   // sides 0 and 1
#pragma unroll
                    for (int s = 0; s < NQ; ++s) {
                        const float4 t4 = lds_f32x4(gb[e] * RSB + gbase[s]);
                        acc0 = __ffma2_rn(make_float2(t4.x, t4.y), st.w[s], acc0);
                        acc1 = __ffma2_rn(make_float2(t4.z, t4.w), st.w[s], acc1);
                    }
                    a0 = acc0.x + acc0.y;
                    a1 = acc1.x + acc1.y;
                } else {
                    const float2 t2 = lds_f32x2(gb[e] * RSB + gbase[0]);
                    a0 = t2.x;
                    a1 = t2.y;
                }
                res[e] = fmaf(w1, a1 - a0, a0);
            }
        }
    };
    auto store4 = [&](int64_t a, int e0, const float (&res)[4]) {
        if (e0 >= 0 && e0 + 4 <= L) {
            __stcs(reinterpret_cast<float4 *>(out + a), make_float4(res[0], res[1], res[2], res[3]));
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e0 + e >= 0 && e0 + e < L) out[a + e] = res[e];
        }
    };

    if constexpr (DOT) {
        float ks = 0.0f, kc = 0.0f;   // Kahan sum of gout * mapped
        auto kadd = [&](float t) {
            const float y = __fsub_rn(t, kc);
            const float s2 = __fadd_rn(ks, y);
            kc = __fsub_rn(__fsub_rn(s2, ks), y);
            ks = s2;
        };
        if ((g.d[D - 1].s & 3) == 0) {
            constexpr int QM = 4;
            struct DSlot {
                float fbi;   // last-dim weight w1 of the slot's first voxel
                int e0;
            };
            const TileShape ts = tile_shape(L, xl & 3, blockDim.x, QM);
            auto slot = [&](int, int e0) {
                DSlot sd;
                sd.e0 = e0;
                sd.fbi = float(2 * (xl + e0) + mb_l) * inv2b_l;
                return sd;
            };
            auto row2 = [&](const int *coords, MRow &st) { row_fn(coords, 0, st); };
            auto quad = [&](MRow &st, const DSlot &sd, int, const float4 &v, const float4 &gq, int64_t) {
                const float vals[4] = {v.x, v.y, v.z, v.w};
                const float gs[4] = {gq.x, gq.y, gq.z, gq.w};
                float res[4];
                map4(st, vals, sd.fbi, res);
                float t = 0.0f;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (sd.e0 + e >= 0 && sd.e0 + e < L) t = fmaf(gs[e], res[e], t);
                kadd(t);
            };
            if constexpr (RING && D >= 3 && std::is_same<T, float>::value) {
                // x and g stream through two cp.async rings behind the tables
                float4 *ring = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(tab) +
                                                          ((map_table_bytes(D, P) + 15) & ~size_t(15)));
                walk_tile_async<D, QM, kDotStages, MRow, DSlot, false, true>(
                    in, stride, box_lo, len, r0, r1, ts, ring, slot, row2, quad, gout);
            } else {
                walk_tile<D, QM, 4, MRow, DSlot, true>(in, gout, stride, box_lo, len, r0, r1, ts, true,
                                                       slot, row2, quad);
            }
        } else {
            auto quad_fn = [&](MRow &st, const QuadRef &q) {
                if (!q.has) return;
                const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
                const float gs[4] = {q.v2.x, q.v2.y, q.v2.z, q.v2.w};
                float res[4];
                map4(st, vals, float(2 * (xl + q.e0) + mb_l) * inv2b_l, res);
                float t = 0.0f;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (q.e0 + e >= 0 && q.e0 + e < L) t = fmaf(gs[e], res[e], t);
                kadd(t);
            };
            walk_box<D, (ADAPTIVE && D >= 3) ? 2 : 4, MRow, true>(in, gout, g.N, stride, box_lo, len, r0,
                                                                  r1, same_align, true, row_fn, quad_fn);
        }
        *dot = make_float2(ks, kc);
        return;
    }

    if constexpr (WALK == kWalkTma) {
        // Warp-specialised tile pipeline: warps 0..7 map (kTmaConsumers
        // threads), warp 8 moves tiles.  Stage s has a "full" barrier (the
        // producer's expect_tx; the TMA load completes it) and an "empty"
        // barrier (one arrival per consumer warp once its results are in the
        // stage).  The producer stores a finished full tile back with TMA, waits
        // for the store to have read the stage, then loads the next tile into it.
        static_assert(D >= 3 && REPL, "TMA tiles: 3- and 4-D cells, replicated tables");
        static_assert(std::is_same<T, float>::value, "TMA tiles: float32 volumes (results in place)");
        constexpr int NS = kTmaStages;
        constexpr int NCW = kTmaConsumers / 32;                 // consumer warps
        constexpr int QT = kTmaTileFloats / 4 / kTmaConsumers;  // quad slots per consumer thread
        constexpr int R = D;                                    // box rank
        const int Bx = tma->bx, By = tma->by, Bz = D == 4 ? tma->bz : 1;
        const int tile_q = (Bx * By * Bz) >> 2;
        const uint32_t tile_bytes = uint32_t(Bx * By * Bz) * 4u;
        constexpr uint32_t kStageBytes = kTmaTileFloats * 4;
        __shared__ __align__(8) uint64_t s_full[NS], s_empty[NS];
        const uint32_t full0 = uint32_t(__cvta_generic_to_shared(s_full));
        const uint32_t empty0 = uint32_t(__cvta_generic_to_shared(s_empty));
        const uint32_t stage0 = (tab_s + uint32_t(map_table_bytes(D, P)) + 127u) & ~127u;
        // tiles of this cell: slices along dim 0 innermost, then blocks along
        // dim D-2, then (4-D) along dim 1; this CTA takes a contiguous range
        const int ny = (len[D - 2] + By - 1) / By;
        const int nz = D == 4 ? (len[1] + Bz - 1) / Bz : 1;
        const int n0 = len[0];
        const int nt_all = n0 * ny * nz;
        const int kb = int((int64_t(nt_all) * chunk) / chunks);
        const int nt = int((int64_t(nt_all) * (chunk + 1)) / chunks) - kb;
        struct Tile {
            int c[R];     // box origin, innermost first
            bool full;    // the box lies inside the cell (TMA store)
        };
        // position of a tile in the cell's order (slice, block along D-2,
        // block along 1); every walker visits its tiles in order, so it steps
        // this forward instead of dividing per tile
        struct TilePos {
            int sl, yb, zb;
        };
        auto tile_pos = [&](int k) {
            const int kk = kb + k;
            const int blk = kk / n0;
            return TilePos{kk - blk * n0, blk % ny, blk / ny};
        };
        auto step = [&](TilePos &q) {
            if (++q.sl == n0) {
                q.sl = 0;
                if (++q.yb == ny) {
                    q.yb = 0;
                    ++q.zb;
                }
            }
        };
        auto tile = [&](const TilePos &q) {
            Tile t;
            const int sl = q.sl, yb = q.yb, zb = q.zb;
            t.c[0] = box_lo[D - 1];
            t.c[1] = box_lo[D - 2] + yb * By;
            if (D == 4) t.c[2] = box_lo[1] + zb * Bz;
            t.c[R - 1] = box_lo[0] + sl;
            t.full = len[D - 1] == Bx && (yb + 1) * By <= len[D - 2] &&
                     (D < 4 || (zb + 1) * Bz <= len[1]);
            return t;
        };
        auto gave_up = [&]() {
            if (tma->status) atomicCAS(tma->status, 0u, uint32_t(MCLAHE_ERR_TIMEOUT));
        };
        if (threadIdx.x == 0) {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                mbar_init(full0 + 8u * i, 1);
                mbar_init(empty0 + 8u * i, NCW);
            }
            mbar_init_fence();
        }
        __syncthreads();
        const int warp = int(threadIdx.x) >> 5;
        if (warp == NCW) {
            // ---- producer (one lane)
            if (lane == 0) {
                TilePos lp = nt > 0 ? tile_pos(0) : TilePos{0, 0, 0};   // next load
                TilePos rp = lp;                                         // next retire
                auto load = [&](int k) {
                    const Tile t = tile(lp);
                    step(lp);
                    const uint32_t st = uint32_t(k % NS);
                    mbar_expect_tx(full0 + 8u * st, tile_bytes);
                    tma_load<R>(stage0 + st * kStageBytes, tma->in, t.c, full0 + 8u * st);
                };
                // tile k - NS is finished when its stage's empty barrier
                // completes its ((k / NS) - 1)-th phase; store it if full
                auto retire = [&](int k) {
                    const uint32_t st = uint32_t(k % NS);
                    if (!mbar_wait_bounded(empty0 + 8u * st, uint32_t(k / NS) & 1u, kTmaWaitLimit))
                        gave_up();
                    const Tile t = tile(rp);
                    step(rp);
                    if (t.full) {
                        tma_store<R>(tma->out, t.c, stage0 + st * kStageBytes);
                        bulk_commit();
                    }
                };
                for (int k = 0; k < nt; ++k) {
                    if (k >= NS) {
                        retire(k - NS);
                        bulk_wait_read<0>();   // the store has read the stage
                    }
                    load(k);
                }
                for (int k = nt > NS ? nt - NS : 0; k < nt; ++k) retire(k);
                bulk_wait_all();
            }
            return;
        }
        // ---- consumers: this thread's quads of a tile, in-tile coordinates
        int qx[QT], qy[QT], qz[QT];
        bool qv[QT];
#pragma unroll
        for (int i = 0; i < QT; ++i) {
            const int qi = int(threadIdx.x) + i * kTmaConsumers;
            qv[i] = qi < tile_q;
            const int e = 4 * qi;
            qx[i] = e % Bx;
            const int rest = e / Bx;
            qy[i] = rest % By;
            qz[i] = rest / By;
        }
        const int lx = len[D - 1];
        // per slot, the row weights without dim 0 (inner) in this lane's order,
        // and which entries take dim 0's w1 (sel): tiles of one block differ
        // only in the slice along dim 0
        constexpr int NW = sizeof(MRow) / sizeof(float2);
        MRow inner[QT];
        uint32_t sel[QT];
        TilePos cq = nt > 0 ? tile_pos(0) : TilePos{0, 0, 0};
        for (int k = 0; k < nt; ++k) {
            const int stg = k % NS;
            if (!mbar_wait_bounded(full0 + 8u * uint32_t(stg), uint32_t(k / NS) & 1u, kTmaWaitLimit))
                gave_up();
            const Tile t = tile(cq);
            const uint32_t sbase = stage0 + uint32_t(stg) * kStageBytes;
            // a new block starts at the first tile and whenever the slice wraps
            if (k == 0 || cq.sl == 0) {
#pragma unroll
                for (int i = 0; i < QT; ++i) {
                    int coords[kMaxDim];
                    coords[0] = t.c[R - 1];
                    if (D == 4) {
                        coords[1] = t.c[2] + qz[i];
                        coords[2] = t.c[1] + qy[i];
                    } else {
                        coords[1] = t.c[1] + qy[i];
                    }
                    MRow s0, s1;
                    row_weights(coords, 1.0f, 0.0f, s0);
                    row_weights(coords, 0.0f, 1.0f, s1);
                    sel[i] = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        // exactly one of the two is the product over dims 1..D-2
                        inner[i].w[w] = make_float2(s0.w[w].x + s1.w[w].x, s0.w[w].y + s1.w[w].y);
                        sel[i] |= (s1.w[w].x != 0.0f ? 1u : 0u) << (2 * w);
                        sel[i] |= (s1.w[w].y != 0.0f ? 1u : 0u) << (2 * w + 1);
                    }
                }
            }
            const float f1 = float(2 * t.c[R - 1] + mb[0]) * inv2b[0], f0 = 1.0f - f1;
#pragma unroll
            for (int i = 0; i < QT; ++i) {
                if (!qv[i]) continue;
                // absolute voxel coordinates of the quad
                const int x = t.c[0] + qx[i], y = t.c[1] + qy[i];
                const int z = D == 4 ? t.c[2] + qz[i] : 0;
                const bool in_cell = qx[i] < lx && y < box_lo[D - 2] + len[D - 2] &&
                                     (D < 4 || z < box_lo[1] + len[1]);
                if (!in_cell) continue;
                const uint32_t qa = sbase + 16u * uint32_t(int(threadIdx.x) + i * kTmaConsumers);
                const float4 v = lds128(qa);
                MRow st;
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    st.w[w] = make_float2(((sel[i] >> (2 * w)) & 1u ? f1 : f0) * inner[i].w[w].x,
                                          ((sel[i] >> (2 * w + 1)) & 1u ? f1 : f0) * inner[i].w[w].y);
                const float vals[4] = {v.x, v.y, v.z, v.w};
                float res[4];
                map4(st, vals, float(2 * x + mb_l) * inv2b_l, res);
                if (t.full) {
                    // in place: the producer stores the tile with one TMA store
                    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(qa), "f"(res[0]),
                                 "f"(res[1]), "f"(res[2]), "f"(res[3])
                                 : "memory");
                } else {
                    int64_t a = x;
                    a += int64_t(t.c[R - 1]) * stride[0];
                    if (D == 4) {
                        a += int64_t(z) * stride[1];
                        a += int64_t(y) * stride[2];
                    } else {
                        a += int64_t(y) * stride[1];
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (qx[i] + e < lx) out[a + e] = res[e];
                }
            }
            if (t.full) fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8u * uint32_t(stg));
            step(cq);
        }
        return;
    }

    if ((g.d[D - 1].s & 3) == 0) {
        // every row starts at the same alignment: fixed quad slots per thread
        constexpr int QM = 4;
        struct MSlot {
            float fbi;   // last-dim weight w1 of the slot's first voxel
            int e0;
        };
        // rows of fewer than 2 QM quads spread over at least two lanes each,
        // so a warp's 16-byte loads and stores cover whole 32-byte sectors of
        // its rows (measured on 128x128x256x32 uint8 with 8-voxel cell rows:
        // the whole forward pass 187 -> 200 Gvoxel/s)
        const int Qrow = ((xl & 3) + L + 3) >> 2;
        const TileShape ts =
            tile_shape(L, xl & 3, blockDim.x, Qrow >= 2 * QM ? QM : (Qrow >= 2 ? Qrow / 2 : 1));
        auto slot = [&](int, int e0) {
            MSlot sd;
            sd.e0 = e0;
            sd.fbi = float(2 * (xl + e0) + mb_l) * inv2b_l;
            return sd;
        };
        auto row2 = [&](const int *coords, MRow &st) { row_fn(coords, 0, st); };
        auto quad = [&](MRow &st, const MSlot &sd, int, const float4 &v, const float4 &, int64_t a) {
            const float vals[4] = {v.x, v.y, v.z, v.w};
            float res[4];
            map4(st, vals, sd.fbi, res);
            store4(a, sd.e0, res);
        };
        if (RING && D >= 3) {
            // rows stream through the cp.async ring behind the tables
            float4 *ring = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(tab) +
                                                      ((map_table_bytes(D, P) + 15) & ~size_t(15)));
            if (ts.head == 0 && ts.QL == QM && L == 4 * ts.LPR * QM) {
                // every slot of every row is a whole quad: no per-slot tests
                auto quad_full = [&](MRow &st, const MSlot &sd, int, const float4 &v, const float4 &,
                                     int64_t a) {
                    const float vals[4] = {v.x, v.y, v.z, v.w};
                    float res[4];
                    map4(st, vals, sd.fbi, res);
                    __stcs(reinterpret_cast<float4 *>(out + a), make_float4(res[0], res[1], res[2], res[3]));
                };
                walk_tile_async<D, QM, kMapStages, MRow, MSlot, true>(in, stride, box_lo, len, r0, r1, ts,
                                                                      ring, slot, row2, quad_full);
            } else {
                walk_tile_async<D, QM, kMapStages, MRow, MSlot>(in, stride, box_lo, len, r0, r1, ts, ring,
                                                                 slot, row2, quad);
            }
        } else if (ts.head == 0 && ts.QL == QM && L == 4 * ts.LPR * QM) {
            auto quad_full = [&](MRow &st, const MSlot &sd, int, const float4 &v, const float4 &,
                                 int64_t a) {
                const float vals[4] = {v.x, v.y, v.z, v.w};
                float res[4];
                map4(st, vals, sd.fbi, res);
                __stcs(reinterpret_cast<float4 *>(out + a), make_float4(res[0], res[1], res[2], res[3]));
            };
            walk_tile<D, QM, 4, MRow, MSlot, false, false, true>(in, nullptr, stride, box_lo, len, r0, r1,
                                                                 ts, true, slot, row2, quad_full);
        } else {
            walk_tile<D, QM, 4, MRow, MSlot, false>(in, nullptr, stride, box_lo, len, r0, r1, ts, true,
                                                    slot, row2, quad);
        }
    } else {
        auto quad_fn = [&](MRow &st, const QuadRef &q) {
            if (!q.has) return;
            const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
            float res[4];
            map4(st, vals, float(2 * (xl + q.e0) + mb_l) * inv2b_l, res);
            store4(q.a, q.e0, res);
        };
        walk_box<D, (ADAPTIVE && D >= 3) ? 2 : 4, MRow>(in, nullptr, g.N, stride, box_lo, len, r0, r1,
                                                        same_align, true, row_fn, quad_fn);
    }
}

}  // namespace mclahe
