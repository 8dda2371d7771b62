// k_bwd.cu -- reverse mode of the forward pass (mclahe_backward) with respect
// to the mapping tables and the clip limit.  The paper does not differentiate
// MCLAHE; the derivatives below are those of Algorithm 1 as the forward pass
// evaluates it.
//
// The output is linear in the tables (Sec. III.C, Eq. (12)-(13)), so
//   dL/dlut[k][j] = sum over voxels v and corners i with k0(v) + i = k and
//                   bin_k(v) = j of g_v * c_i(v).
// Three launches:
//   k_gmax    the largest |g| of the upstream gradient (the fixed-point scale);
//   k_adj     one CTA per chunk of an inter-kernel cell: streams the input and
//             the upstream gradient, accumulates g * c_i into the cell's 2^D
//             corner tables in shared memory and adds them, copies summed, to
//             the cell's table-gradient sums in global memory (64-bit integer
//             atomics: exact, so the order of the chunks does not matter).
//             The sums are exact integers: each term is rounded to a
//             fixed-point integer f with
//             |f| < 2^30 (scale 2^E from max |g|) and added as two 32-bit
//             words, hi = f >> 15 and lo = f & 0x7fff, into separate
//             accumulators (32-bit integer shared-memory reductions run several
//             times faster than float ones, and the result does not depend on
//             the order); with at most 65535 voxels per chunk neither word's
//             sum can overflow.  Lane-rotated copies keep the reductions
//             conflict-free whatever the bins;
//   k_lutbwd  one CTA per kernel: sums the integer sums of the cells around
//             the kernel (exact), scales them to float once, folds the padded
//             table indices, stores dL/dlut, and takes the reverse of clip,
//             redistribute, cumulative sum and normalisation:
//               dL/dT = (1/den) [sum_j g_j (A_j - A_0 - j N_c/nb)
//                                + (A_0 - N_c/nb) sum_j g_j lut_j],
//             den = C_{nb-1} - C_0, A_j the clipped bins up to j (0 for a
//             constant CDF);
//   k_clipgrad one CTA: dL/dclip = V * sum_k dL/dT_k in a fixed order (0 when
//             the clip limit given lies outside [0, 1], where the forward
//             clamps it).
#include <algorithm>

#include "hist_impl.cuh"
#include "map_impl.cuh"   // rotate_left

namespace mclahe {

// Accumulator layout of k_adj.  REPL: [corner][index][copy] with 32 / 2^D
// copies; lane l adds, at step t, to corner (t + l) mod 2^D in copy l / 2^D,
// so the 32 lanes of a warp always touch 32 different words in 32 different
// banks (the index is shared or not); the lane rotation is undone by rotated
// per-lane weights and ranges, as in the mapping pass.  Plain: [corner][index].
__host__ __device__ inline bool adj_repl(int P) { return size_t(P) * 128 <= 160 * 1024; }
// bytes of one accumulator array (hi or lo words)
__host__ __device__ inline size_t adj_words_bytes(int D, int P) {
    return adj_repl(P) ? size_t(P) * 128 : (size_t(1) << D) * size_t(P) * sizeof(uint32_t);
}
__host__ __device__ inline size_t adj_smem(int D, int P) { return 2 * adj_words_bytes(D, P); }

// Fixed-point exponent E of a launch: max|g| * 2^E < 2^30 (0 if g is all zero).
__device__ __forceinline__ int adj_exponent(uint32_t gmax_key) {
    const float gmax = __uint_as_float(gmax_key);
    if (!(gmax > 0.0f)) return 0;
    int e;
    frexpf(gmax, &e);   // gmax < 2^e
    return min(max(30 - e, -126), 126);
}

// the largest |g| as an order-preserving key (|g| as bits: non-negative floats
// order as unsigned integers)
__global__ void __launch_bounds__(256) k_gmax(const float *__restrict__ g, int64_t n,
                                              uint32_t *__restrict__ key) {
    float m = 0.0f;
    const int64_t nq = n >> 2;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nq; q += stride) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(g) + q);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int64_t t = (nq << 2) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride)
        m = fmaxf(m, fabsf(g[t]));
    const uint32_t k = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if ((threadIdx.x & 31) == 0) atomicMax(key, k);
}

template <int D, bool ADAPTIVE, bool REPL>
__global__ void __launch_bounds__(256, 2) k_adj(Geom g, const float *__restrict__ in,
                                                const float *__restrict__ gout,
                                                const float *__restrict__ lo_k,
                                                const float *__restrict__ scale_k,
                                                unsigned long long *__restrict__ sums, int chunks,
                                                const uint32_t *__restrict__ gmax_key) {
    constexpr int NC = 1 << D;
    constexpr int NO = 1 << (D - 1);
    constexpr int RC = REPL ? 32 / NC : 1;      // copies
    extern __shared__ __align__(16) uint32_t acc[];   // hi words, then lo words
    __shared__ float s_nlo[NC], s_sc[NC];
    const int P = g.P, LS = g.LS;
    const int lane = threadIdx.x & 31;
    const int64_t cell = blockIdx.x / chunks;
    const int chunk = int(blockIdx.x - cell * chunks);

    int cc[kMaxDim];
    {
        int64_t r = cell;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            cc[j] = int(r % (g.d[j].n - 1));
            r /= (g.d[j].n - 1);
        }
    }
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
    {
        uint4 *z = reinterpret_cast<uint4 *>(acc);
        const int n4 = int(2 * NC * P * RC / 4);
        for (int i = threadIdx.x; i < n4; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = n4 * 4 + threadIdx.x; i < 2 * NC * P * RC; i += blockDim.x) acc[i] = 0u;
    }
    if (threadIdx.x < NC) {
        int64_t k = kbase;
#pragma unroll
        for (int d = 0; d < D; ++d) k += ((threadIdx.x >> (D - 1 - d)) & 1) ? kstr[d] : 0;
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
    const int r1 = int((int64_t(R) * (chunk + 1)) / chunks);
    __syncthreads();

    float inv2b[kMaxDim];
    int mb[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Dim &dj = g.d[j];
        inv2b[j] = 1.0f / float(2 * dj.b);
        mb[j] = 2 * dj.p0 - (dj.b - 1) - 2 * dj.b * cc[j];
    }
    const uint32_t acc_s = uint32_t(__cvta_generic_to_shared(acc));
    const uint32_t lo_off = uint32_t(NC * P * RC) * 4u;   // the lo words behind the hi words
    const int E = adj_exponent(__ldcg(gmax_key));
    const float fscale = ldexpf(1.0f, E);
    const float iqk = g.iqk, qkf = g.qkf;
    const int rot = REPL ? (lane & (NC - 1)) : 0;
    const int copy = REPL ? (lane / NC) : 0;
    constexpr uint32_t IB = uint32_t(4 * RC);   // bytes per table index
    // per step t: corner (t + rot) mod NC, its range and accumulator base
    float nl[NC], sc[NC];
    uint32_t cbase[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) {
        const int c = (t + rot) & (NC - 1);
        nl[t] = s_nlo[c];
        sc[t] = s_sc[c];
        cbase[t] = acc_s + uint32_t(c * P) * IB + 4u * uint32_t(copy) - kBinBias * IB;
    }
    const int L = len[D - 1];
    const int xl = box_lo[D - 1];
    const float inv2b_l = inv2b[D - 1];
    const float two_inv2b = 2.0f * inv2b_l;
    const int mb_l = mb[D - 1];
    const int rodd = rot & 1;

    // per row: the outer weight of the corner each step handles
    struct BRow {
        float w[NC];
    };
    auto row_fn = [&](const int *coords, BRow &st) {
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
        float a[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) a[c] = wo[c >> 1];
        if (REPL) rotate_left<NC>(a, rot);
#pragma unroll
        for (int c = 0; c < NC; ++c) st.w[c] = a[c];
    };
    // adds g * c_i for the voxel (x, g) at last-dim weight w1
    auto add = [&](const BRow &st, float x, float gv, float w1) {
        const float gw1 = gv * w1, gw0 = gv - gw1;
        const float ge = rodd ? gw1 : gw0, go = rodd ? gw0 : gw1;   // even / odd steps
        uint32_t bins[NC];
        if (ADAPTIVE && NC >= 2) {
            // the corners' bins two at a time (packed; the same roundings as qbits1)
#pragma unroll
            for (int t = 0; t < NC; t += 2) {
                const uint2 b2 = qbits2(make_float2(x, x), make_float2(nl[t], nl[t + 1]),
                                        make_float2(sc[t], sc[t + 1]), iqk, qkf);
                bins[t] = b2.x;
                bins[t + 1] = b2.y;
            }
        } else {
            const uint32_t b0 = qbits1(x, nl[0], sc[0], iqk, qkf);
#pragma unroll
            for (int t = 0; t < NC; ++t) bins[t] = b0;
        }
#pragma unroll
        for (int t = 0; t < NC; ++t) {
            const float v = st.w[t] * ((t & 1) ? go : ge);
            const int f = __float2int_rn(v * fscale);   // |f| < 2^30
            const uint32_t a = bins[t] * IB + cbase[t];
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(uint32_t(f >> 15)) : "memory");
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a + lo_off), "r"(uint32_t(f & 0x7fff))
                         : "memory");
        }
    };
    if ((g.d[D - 1].s & 3) == 0) {
        struct BSlot {
            float fbi;   // last-dim weight w1 of the slot's first voxel
            int e0;
        };
        const TileShape ts = tile_shape(L, xl & 3, blockDim.x, 4);
        auto slot = [&](int, int e0) {
            BSlot sd;
            sd.e0 = e0;
            sd.fbi = float(2 * (xl + e0) + mb_l) * inv2b_l;
            return sd;
        };
        auto quad = [&](BRow &st, const BSlot &sd, int, const float4 &v, const float4 &gq, int64_t) {
            const float vals[4] = {v.x, v.y, v.z, v.w};
            const float gs[4] = {gq.x, gq.y, gq.z, gq.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (sd.e0 + e >= 0 && sd.e0 + e < L) add(st, vals[e], gs[e], fmaf(float(e), two_inv2b, sd.fbi));
        };
        if (ts.head == 0 && ts.QL == 4 && L == 16 * ts.LPR) {
            // every slot of every row is a whole quad: no per-voxel tests
            auto quad_full = [&](BRow &st, const BSlot &sd, int, const float4 &v, const float4 &gq,
                                 int64_t) {
                add(st, v.x, gq.x, sd.fbi);
                add(st, v.y, gq.y, fmaf(1.0f, two_inv2b, sd.fbi));
                add(st, v.z, gq.z, fmaf(2.0f, two_inv2b, sd.fbi));
                add(st, v.w, gq.w, fmaf(3.0f, two_inv2b, sd.fbi));
            };
            walk_tile<D, 4, 2, BRow, BSlot, true, false, true>(in, gout, stride, box_lo, len, r0, r1, ts,
                                                               true, slot, row_fn, quad_full);
        } else {
            walk_tile<D, 4, 2, BRow, BSlot, true>(in, gout, stride, box_lo, len, r0, r1, ts, true, slot,
                                                  row_fn, quad);
        }
    } else {
        auto row64 = [&](const int *coords, int64_t, BRow &st) { row_fn(coords, st); };
        auto quad_fn = [&](BRow &st, const QuadRef &q) {
            if (!q.has) return;
            const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
            const float gs[4] = {q.v2.x, q.v2.y, q.v2.z, q.v2.w};
            const float fbi = float(2 * (xl + q.e0) + mb_l) * inv2b_l;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (q.e0 + e >= 0 && q.e0 + e < L) add(st, vals[e], gs[e], fmaf(float(e), two_inv2b, fbi));
        };
        walk_box<D, 4, BRow, true>(in, gout, g.N, stride, box_lo, len, r0, r1, false, true, row64,
                                   quad_fn);
    }
    __syncthreads();
    // the chunk's sums, copies summed, added to the cell's integer sums
    unsigned long long *dst = sums + size_t(cell) * NC * LS;
    for (int i = threadIdx.x; i < NC * P; i += blockDim.x) {
        const int c = i / P, j = i - c * P;
        const uint32_t *hi = acc + (size_t(c) * P + j) * RC;
        const uint32_t *lo = hi + NC * P * RC;
        int64_t tot = 0;
#pragma unroll
        for (int q = 0; q < RC; ++q) tot += int64_t(int32_t(hi[q])) * 32768 + int64_t(lo[q]);
        if (tot != 0) atomicAdd(dst + size_t(c) * LS + j, static_cast<unsigned long long>(tot));
    }
}

// Deterministic block sum (fixed shuffle tree, then warps in order); the
// result is valid in thread 0.
__device__ __forceinline__ float block_sum(float v) {
    __shared__ float s_w[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    float s = 0.0f;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += s_w[w];
    __syncthreads();
    return s;
}

template <int D>
__global__ void __launch_bounds__(256) k_lutbwd(Geom g, const uint32_t *__restrict__ hist,
                                                const float *__restrict__ lut,
                                                const unsigned long long *__restrict__ sums,
                                                const uint32_t *__restrict__ gmax_key,
                                                const float *__restrict__ d_clip,
                                                float *__restrict__ d_grad_lut,
                                                float *__restrict__ dT) {
    constexpr int NC = 1 << D;
    extern __shared__ __align__(16) float G[];   // P floats, then nb counts
    const int nb = g.nb, P = g.P, LS = g.LS;
    uint32_t *h = reinterpret_cast<uint32_t *>(G + P);
    const int64_t k = blockIdx.x;
    int kk[kMaxDim];
    {
        int64_t r = k;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            kk[j] = int(r % g.d[j].n);
            r /= g.d[j].n;
        }
    }
    // the cell that has kernel k as its corner c (if it exists)
    int64_t cell_of[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        int64_t cell = 0;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int cd = kk[d] - ((c >> (D - 1 - d)) & 1);
            ok &= (cd >= 0) && (cd <= g.d[d].n - 2);
            cell = cell * (g.d[d].n - 1) + cd;
        }
        cell_of[c] = ok ? cell : -1;
    }
    // dL/dlut: the integer sums of the (up to 2^D) cells around the kernel,
    // added exactly, then scaled to float once
    const float inv = ldexpf(1.0f, -adj_exponent(__ldcg(gmax_key)));
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        int64_t t = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (cell_of[c] >= 0) t += int64_t(__ldcg(sums + (cell_of[c] * NC + c) * LS + j));
        G[j] = float(t) * inv;
    }
    for (int j = threadIdx.x; j < nb; j += blockDim.x) h[j] = hist[k * nb + j];
    __syncthreads();
    if (threadIdx.x == 0) {   // padded indices >= nb stand for the last bin
        float s = G[nb - 1];
        for (int j = nb; j < P; ++j) s += G[j];
        G[nb - 1] = s;
    }
    __syncthreads();
    if (d_grad_lut)
        for (int j = threadIdx.x; j < nb; j += blockDim.x) d_grad_lut[k * nb + j] = G[j];
    const LutStats st = lut_stats(h, nb, g.V, load_clip(d_clip, g.clip));
    const float ncb = float(st.N_c) / float(nb);
    float s1 = 0.0f, s2 = 0.0f;
    int64_t Aj = st.pa;
    for (int j = st.j0; j < st.j1; ++j) {
        if (int64_t(h[j]) > st.tf) Aj += 1;
        s1 = fmaf(G[j], float(Aj - st.A0) - float(j) * ncb, s1);
        s2 = fmaf(G[j], lut[k * LS + j], s2);
    }
    s1 = block_sum(s1);
    s2 = block_sum(s2);
    if (threadIdx.x == 0)
        dT[k] = st.flat ? 0.0f : (s1 + (float(st.A0) - ncb) * s2) / st.den;
}

__global__ void __launch_bounds__(256) k_clipgrad(const float *__restrict__ dT, int64_t K,
                                                  int64_t V, const float *__restrict__ d_clip,
                                                  float plan_clip, float *__restrict__ out) {
    float s = 0.0f;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) s += dT[k];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        const float raw = d_clip ? *d_clip : plan_clip;
        out[0] = (raw >= 0.0f && raw <= 1.0f) ? float(V) * s : 0.0f;
    }
}

size_t bwd_sum_words(const Geom &g) { return size_t(n_cells(g)) * (size_t(1) << g.D) * size_t(g.LS); }
// the scatter's sums, max |g| key and dL/dT, or the gather's tables and
// partials (k_bwd_gather.cu), whichever is larger: both start at the scratch
size_t bwd_scratch_bytes(const Geom &g, int chunks) {
    return std::max(8 * bwd_sum_words(g) + 16 + sizeof(float) * size_t(g.K), bwd_gather_bytes(g, chunks));
}

template <int D>
static cudaError_t launch_bwd_d(const mclahe_plan_s &p, const float *in, const float *gout,
                                unsigned char *ws, const float *d_clip, float *d_grad_lut,
                                float *d_grad_clip, cudaStream_t st) {
    const Geom &g = p.g;
    const int chunks = p.t.bwd_chunks;
    // scratch: integer sums, the max |g| key (cleared together), dL/dT
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(ws + p.ws.scratch);
    uint32_t *gmax_key = reinterpret_cast<uint32_t *>(sums + bwd_sum_words(g));
    float *dT = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(gmax_key) + 16);
    const size_t smem_adj = adj_smem(D, g.P);
    const unsigned grid = unsigned(n_cells(g) * chunks);
    const bool repl = adj_repl(g.P);
    const float *lo = reinterpret_cast<const float *>(ws + p.ws.lo);
    const float *sc = reinterpret_cast<const float *>(ws + p.ws.scale);
    cudaError_t e = cudaMemsetAsync(sums, 0, 8 * bwd_sum_words(g) + sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    {
        const int64_t nq = (g.N >> 2) + 1;
        const int blocks = int(std::min<int64_t>((nq + 255) / 256, int64_t(device_sms()) * 4));
        k_gmax<<<blocks, 256, 0, st>>>(gout, g.N, gmax_key);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
#define MCLAHE_ADJ(A, R)                                                                       \
    e = ensure_smem(reinterpret_cast<const void *>(k_adj<D, A, R>), size_t(smem_adj));          \
    if (e != cudaSuccess) return e;                                                            \
    k_adj<D, A, R><<<grid, 256, smem_adj, st>>>(g, in, gout, lo, sc, sums, chunks, gmax_key);
    if (g.mode == MCLAHE_RANGE_ADAPTIVE) {
        if (repl) { MCLAHE_ADJ(true, true) } else { MCLAHE_ADJ(true, false) }
    } else {
        if (repl) { MCLAHE_ADJ(false, true) } else { MCLAHE_ADJ(false, false) }
    }
#undef MCLAHE_ADJ
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem_lb = size_t(g.P) * sizeof(float) + size_t(g.nb) * sizeof(uint32_t);
    e = ensure_smem(reinterpret_cast<const void *>(k_lutbwd<D>), size_t(smem_lb));
    if (e != cudaSuccess) return e;
    k_lutbwd<D><<<unsigned(g.K), 256, smem_lb, st>>>(
        g, reinterpret_cast<const uint32_t *>(ws + p.ws.hist), reinterpret_cast<const float *>(ws + p.ws.lut),
        sums, gmax_key, d_clip, d_grad_lut, dT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (d_grad_clip) {
        k_clipgrad<<<1, 256, 0, st>>>(dT, g.K, g.V, d_clip, g.clip, d_grad_clip);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_backward(const mclahe_plan_s &p, const float *in, const float *gout,
                            unsigned char *ws, const float *d_clip, float *d_grad_lut,
                            float *d_grad_clip, cudaStream_t st) {
    // the clip-limit gradient alone: the gather form (no table gradients needed)
    if (!d_grad_lut && d_grad_clip) return launch_backward_gather(p, in, gout, ws, d_clip, d_grad_clip, st);
    switch (p.g.D) {
        case 1: return launch_bwd_d<1>(p, in, gout, ws, d_clip, d_grad_lut, d_grad_clip, st);
        case 2: return launch_bwd_d<2>(p, in, gout, ws, d_clip, d_grad_lut, d_grad_clip, st);
        case 3: return launch_bwd_d<3>(p, in, gout, ws, d_clip, d_grad_lut, d_grad_clip, st);
        case 4: return launch_bwd_d<4>(p, in, gout, ws, d_clip, d_grad_lut, d_grad_clip, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_backward(mclahe_plan_t p, const float *d_in,
                                         const float *d_grad_out, void *d_ws, size_t ws_bytes,
                                         const float *d_clip, float *d_grad_lut,
                                         float *d_grad_clip, mclahe_stream_t stream) {
    mclahe_status s = check_forward_args(p, d_in, d_grad_out, d_ws, ws_bytes);
    if (s != MCLAHE_OK) return s;
    if (!d_grad_lut && !d_grad_clip) return MCLAHE_ERR_INVALID_ARG;
    cudaError_t e = launch_backward(*p, d_in, d_grad_out, static_cast<unsigned char *>(d_ws), d_clip,
                                    d_grad_lut, d_grad_clip, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}

namespace mclahe {
// k_bwd_gather.cu: the gather form over n_vol volumes of one plan (host arrays
// of device pointers; d_clip nullable, else n_vol clip limits; d_grad_clip
// n_vol floats)
cudaError_t launch_backward_gather_many(const mclahe_plan_s &p, int n_vol, const float *const *in,
                                        const float *const *gout, void *const *ws,
                                        const float *d_clip, float *d_grad_clip, cudaStream_t st);
}  // namespace mclahe

extern "C" mclahe_status mclahe_backward_batch(mclahe_plan_t p, int n_vol, const float *const *d_in,
                                               const float *const *d_grad_out, void *const *d_ws,
                                               size_t ws_bytes, const float *d_clip,
                                               float *d_grad_clip, mclahe_stream_t stream) {
    if (!p || n_vol < 0 || !d_grad_clip || (n_vol > 0 && (!d_in || !d_grad_out || !d_ws)))
        return MCLAHE_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_grad_clip) & 3) return MCLAHE_ERR_INVALID_ARG;
    if (d_clip && (reinterpret_cast<uintptr_t>(d_clip) & 3)) return MCLAHE_ERR_INVALID_ARG;
    for (int v = 0; v < n_vol; ++v) {
        const mclahe_status s = check_forward_args(p, d_in[v], d_grad_out[v], d_ws[v], ws_bytes);
        if (s != MCLAHE_OK) return s;
        for (int u = 0; u < v; ++u)
            if (d_ws[u] == d_ws[v]) return MCLAHE_ERR_INVALID_ARG;
    }
    if (n_vol == 0) return MCLAHE_OK;
    const cudaError_t e = launch_backward_gather_many(*p, n_vol, d_in, d_grad_out, d_ws, d_clip,
                                                      d_grad_clip, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MCLAHE_OK : MCLAHE_ERR_CUDA;
}
