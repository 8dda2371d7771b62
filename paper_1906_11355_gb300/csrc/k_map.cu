// k_map.cu -- intensity mapping by multilinear interpolation (Sec. III.C,
// Eq. (12)-(13); Algorithm 1, the interpolation loop).
//
// Voxels that share the same 2^D nearest kernels form an inter-kernel cell
// (the dotted regions of Fig. 2).  Each CTA takes one cell (or a chunk of its
// rows), stages the 2^D neighbouring mapping tables in shared memory, then
// streams its voxels with 128-bit loads and stores, four quads in flight per
// thread.  Each voxel takes its bin under every neighbour's range (one bin for
// a global range), reads the tables at those bins and blends them with the
// Lagrange coefficients
//   out = sum_i prod_j w_{i_j, j} * lut[k0 + i][bin_{k0+i}(x)],
//   w_{1,j} = d_{j0} / b_j,  w_{0,j} = 1 - w_{1,j},
// where d_{j0} = (x_j + p_j0) - (k0_j b_j + (b_j - 1) / 2) is the distance to
// the lower kernel's centre: w_{1,j} = m / (2 b_j) with the integer
// m = 2 (x_j + p_j0) - (b_j - 1) - 2 b_j k0_j in [0, 2 b_j).
//
// Shared-memory layout (bank-conflict-free gathers).  The bins of the voxels
// of a warp are unrelated, so 32 lanes reading the same corner of 32 random
// bins would hit random banks.  Each bin therefore owns one 128-byte row of 32
// slots holding 32 / 2^D copies of its 2^D corner values (slot s = corner
// s mod 2^D), and lane l reads, at step t, the corner (t + l) mod 2^D from
// copy l / 2^D: for every step the 32 lanes touch 32 different banks whatever
// their bins.  With a global range the reads are 16-byte corner quads and the
// rule applies per 8-lane phase.  The lane-dependent corner order is undone by
// per-lane rotated copies of the corner ranges and weights, built once per CTA
// and per row.  Tables too large for this layout (n_bins > 1024) use a plain
// corner-major layout.
//
// Every table has lut[.][0] = 0 (the normalisation subtracts the first CDF
// value), so with a global range a voxel in bin 0 maps to 0 without gathers.
#include "mclahe_internal.cuh"

namespace mclahe {

__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ float4 lds_f32x4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

// Rotate an array of N values left by r (0 <= r < N, N a power of two) with
// log2(N) levels of selects, keeping every index static.
template <int N>
__device__ __forceinline__ void rotate_left(float (&a)[N], int r) {
#pragma unroll
    for (int sh = 1; sh < N; sh <<= 1) {
        const bool on = (r & sh) != 0;
        float t[N];
#pragma unroll
        for (int i = 0; i < N; ++i) t[i] = on ? a[(i + sh) & (N - 1)] : a[i];
#pragma unroll
        for (int i = 0; i < N; ++i) a[i] = t[i];
    }
}

template <int D, bool ADAPTIVE, bool REPL>
__global__ void __launch_bounds__(256) k_map(Geom g, const float *__restrict__ in,
                                             float *__restrict__ out,
                                             const float *__restrict__ lut,
                                             const float *__restrict__ lo_k,
                                             const float *__restrict__ scale_k, int chunks) {
    constexpr int NC = 1 << D;          // corners
    constexpr int NO = 1 << (D - 1);    // corners over dims 0..D-2
    constexpr int NQ = NC >= 4 ? NC / 4 : 1;   // 16-byte corner quads per bin
    extern __shared__ __align__(16) float tab[];
    __shared__ float s_lo[NC], s_sc[NC];
    const int nb = g.nb;
    const int lane = threadIdx.x & 31;

    const int64_t cell = blockIdx.x / chunks;
    const int chunk = blockIdx.x - int(cell * chunks);
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
    if (REPL) {
        // row of 32 slots per bin, slot s holds corner s mod NC
        for (int t = threadIdx.x; t < nb * 32; t += blockDim.x) {
            const int j = t >> 5, c = t & (NC - 1);
            tab[t] = lut[corner_kernel(c) * nb + j];
        }
    } else if (ADAPTIVE) {
        for (int t = threadIdx.x; t < NC * nb; t += blockDim.x) {
            const int i = t / nb, j = t - i * nb;
            tab[t] = lut[corner_kernel(i) * nb + j];
        }
    } else {
        for (int t = threadIdx.x; t < NC * nb; t += blockDim.x) {
            const int j = t / NC, i = t - j * NC;
            tab[t] = lut[corner_kernel(i) * nb + j];
        }
    }
    if (threadIdx.x < NC) {
        const int64_t k = corner_kernel(threadIdx.x);
        s_lo[threadIdx.x] = lo_k[k];
        s_sc[threadIdx.x] = scale_k[k];
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
    const int r1 = int((int64_t(R) * (chunk + 1)) / chunks);
    __syncthreads();

    const float top = float(nb - 1);
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

    // lane rotation (REPL): AHR reads corner (t + rot) mod NC at step t from
    // copy l / NC; GHR reads quad (s + rot) mod NQ at step s from copy
    // (l / NQ) mod (8 / NQ) of its 8-lane phase.
    const int rot = REPL ? (ADAPTIVE ? (lane & (NC - 1)) : (lane & (NQ - 1))) : 0;

    // adaptive ranges and table addresses per step, rotated
    float clo[ADAPTIVE ? NC : 1], csc[ADAPTIVE ? NC : 1];
    uint32_t cbase[ADAPTIVE ? NC : 1];
    const float glo = s_lo[0], gsc = s_sc[0];
    if (ADAPTIVE) {
#pragma unroll
        for (int t = 0; t < NC; ++t) {
            const int c = REPL ? ((t + rot) & (NC - 1)) : t;
            clo[t] = s_lo[c];
            csc[t] = s_sc[c];
            // address of (bin, corner c) = tab + 4 * index; index = bin*32 + slot
            // (REPL) or c*nb + bin; the bits of the quantiser are 2^23 + bin
            if (REPL) {
                const int slot = (lane & ~(NC - 1) & 31) | c;
                cbase[t] = tab_s + 4u * uint32_t(slot) - (kBinBias << 7);
            } else {
                cbase[t] = tab_s + 4u * uint32_t(c * nb) - (kBinBias << 2);
            }
        }
    }
    // GHR: byte offset of this lane's quad slot at step s (REPL)
    uint32_t gslot[NQ];
#pragma unroll
    for (int s = 0; s < NQ; ++s) {
        const int qd = (s + rot) & (NQ - 1);
        const int copy = (lane / NQ) & ((8 / NQ) - 1);
        gslot[s] = 16u * uint32_t(copy * NQ + qd);
    }

    const int L = len[D - 1];
    const int xl = box_lo[D - 1];
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);
    const WalkShape ws = walk_shape(L, xl, same_align, blockDim.x);

    // Per-row state: the outer weights in the order this lane reads them.
    //   AHR: wt[t] = weight over dims 0..D-2 of corner (t + rot) mod NC;
    //   GHR: (wa[s], wb[s]) = outer weights of the two outer corners of quad
    //        (s + rot) mod NQ (corners 4q..4q+3 = outer 2q, 2q+1 x last 0, 1).
    struct MRow {
        float w[ADAPTIVE ? NC : 2 * NQ];
    };
    auto row_fn = [&](const int *coords, int64_t, MRow &st) {
        float wo[NO];
#pragma unroll
        for (int i = 0; i < NO; ++i) wo[i] = 1.0f;
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            const float w1 = float(2 * coords[j] + mb[j]) * inv2b[j];
            const float w0 = 1.0f - w1;
#pragma unroll
            for (int i = 0; i < NO; ++i) wo[i] *= ((i >> (D - 2 - j)) & 1) ? w1 : w0;
        }
        if (ADAPTIVE) {
            float a[ADAPTIVE ? NC : 1];
#pragma unroll
            for (int c = 0; c < NC; ++c) a[c] = wo[c >> 1];
            if (REPL) rotate_left<ADAPTIVE ? NC : 1>(a, rot);
#pragma unroll
            for (int c = 0; c < NC; ++c) st.w[c] = a[c];
        } else if (NC >= 4) {
            // pairs (wo[2q], wo[2q+1]) for quads q = 0..NQ-1, rotated by rot
            float pa[NQ], pb[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                pa[q] = wo[2 * q];
                pb[q] = wo[2 * q + 1];
            }
            if (REPL && NQ > 1) {
                rotate_left<NQ>(pa, rot);
                rotate_left<NQ>(pb, rot);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                st.w[2 * q] = pa[q];
                st.w[2 * q + 1] = pb[q];
            }
        } else {
            st.w[0] = wo[0];
            st.w[1] = wo[0];
        }
    };

    const int rodd = rot & 1;
    auto quad_fn = [&](MRow &st, const QuadRef &q) {
        if (!q.has) return;
        const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
        const float fb = float(2 * (xl + q.e0) + mb[D - 1]);
        float res[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float w1 = (fb + float(2 * e)) * inv2b[D - 1];
            const float w0 = 1.0f - w1;
            float acc = 0.0f;
            if (ADAPTIVE) {
                // even steps read last-dim side (t + rot) & 1, odd steps the other
                float ae = 0.0f, ao = 0.0f;
#pragma unroll
                for (int t = 0; t < NC; ++t) {
                    const uint32_t bits = quantise_bits(vals[e], clo[t], csc[t], top);
                    const float v = REPL ? lds_f32(cbase[t] + (bits << 7)) : lds_f32(cbase[t] + (bits << 2));
                    if (t & 1) ao = fmaf(st.w[t], v, ao);
                    else ae = fmaf(st.w[t], v, ae);
                }
                const float wev = rodd ? w1 : w0, wod = rodd ? w0 : w1;
                acc = fmaf(wev, ae, wod * ao);
            } else {
                const uint32_t bits = quantise_bits(vals[e], glo, gsc, top);
                if (bits != kBinBias) {
                    if (REPL) {
                        const uint32_t row = tab_s + ((bits - kBinBias) << 7);
                        if (NC >= 4) {
                            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                            for (int s = 0; s < NQ; ++s) {
                                const float4 t4 = lds_f32x4(row + gslot[s]);
                                s0 = fmaf(st.w[2 * s], t4.x, fmaf(st.w[2 * s + 1], t4.z, s0));
                                s1 = fmaf(st.w[2 * s], t4.y, fmaf(st.w[2 * s + 1], t4.w, s1));
                            }
                            acc = fmaf(w0, s0, w1 * s1);
                        } else {
                            // D = 1: two corners, 16 copies of 8 bytes per row
                            const uint32_t a2 = row + 8u * uint32_t(lane & 15);
                            acc = fmaf(w0, lds_f32(a2), w1 * lds_f32(a2 + 4));
                        }
                    } else {
                        // plain layout: the NC corners of a bin are adjacent; outer
                        // corner i owns corners 2i (last side 0) and 2i+1 (side 1),
                        // and without rotation st.w[i] is its outer weight
                        const uint32_t row = tab_s + ((bits - kBinBias) * uint32_t(NC)) * 4u;
                        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                        for (int i = 0; i < NO; ++i) {
                            s0 = fmaf(st.w[i], lds_f32(row + 8u * i), s0);
                            s1 = fmaf(st.w[i], lds_f32(row + 8u * i + 4u), s1);
                        }
                        acc = fmaf(w0, s0, w1 * s1);
                    }
                }
            }
            res[e] = acc;
        }
        if (q.e0 >= 0 && q.e0 + 4 <= L) {
            __stcs(reinterpret_cast<float4 *>(out + q.a), make_float4(res[0], res[1], res[2], res[3]));
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int el = q.e0 + e;
                if (el >= 0 && el < L) out[q.a + e] = res[e];
            }
        }
    };

    if (ws.ru == 1)
        walk_rows<D, 1, MRow>(in, g.N, stride, box_lo, len, r0, r1, ws, true, row_fn, quad_fn);
    else if (ws.ru == 2)
        walk_rows<D, 2, MRow>(in, g.N, stride, box_lo, len, r0, r1, ws, true, row_fn, quad_fn);
    else
        walk_rows<D, 4, MRow>(in, g.N, stride, box_lo, len, r0, r1, ws, true, row_fn, quad_fn);
}

// The replicated layout needs 128 bytes per bin.
static bool use_repl(const Geom &g) { return size_t(g.nb) * 128 <= 160 * 1024; }

size_t map_smem_bytes(const Geom &g) {
    return use_repl(g) ? size_t(g.nb) * 128 : (size_t(1) << g.D) * g.nb * sizeof(float);
}

template <int D, bool A, bool REPL>
static cudaError_t launch_map_t(const mclahe_plan_s &p, const float *in, float *out,
                                const unsigned char *ws, cudaStream_t st, unsigned grid,
                                size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_map<D, A, REPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    k_map<D, A, REPL><<<grid, p.t.map_threads, smem, st>>>(
        p.g, in, out, reinterpret_cast<const float *>(ws + p.ws.lut),
        reinterpret_cast<const float *>(ws + p.ws.lo), reinterpret_cast<const float *>(ws + p.ws.scale),
        p.t.map_chunks);
    return cudaGetLastError();
}

template <int D>
static cudaError_t launch_map_d(const mclahe_plan_s &p, const float *in, float *out,
                                const unsigned char *ws, cudaStream_t st) {
    const Geom &g = p.g;
    int64_t cells = 1;
    for (int j = 0; j < D; ++j) cells *= (g.d[j].n - 1);
    const unsigned grid = unsigned(cells * p.t.map_chunks);
    const size_t smem = map_smem_bytes(g);
    const bool repl = use_repl(g);
    if (g.mode == MCLAHE_RANGE_ADAPTIVE)
        return repl ? launch_map_t<D, true, true>(p, in, out, ws, st, grid, smem)
                    : launch_map_t<D, true, false>(p, in, out, ws, st, grid, smem);
    return repl ? launch_map_t<D, false, true>(p, in, out, ws, st, grid, smem)
                : launch_map_t<D, false, false>(p, in, out, ws, st, grid, smem);
}

cudaError_t launch_map(const mclahe_plan_s &p, const float *in, float *out,
                       const unsigned char *ws, cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_map_d<1>(p, in, out, ws, st);
        case 2: return launch_map_d<2>(p, in, out, ws, st);
        case 3: return launch_map_d<3>(p, in, out, ws, st);
        case 4: return launch_map_d<4>(p, in, out, ws, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
