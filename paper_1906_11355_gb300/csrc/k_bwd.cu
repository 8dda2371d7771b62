// k_bwd.cu -- reverse mode of the forward pass (mclahe_backward) with respect
// to the mapping tables and the clip limit.  The paper does not differentiate
// MCLAHE; the derivatives below are those of Algorithm 1 as the forward pass
// evaluates it.
//
// The output is linear in the tables (Sec. III.C, Eq. (12)-(13)), so
//   dL/dlut[k][j] = sum over voxels v and corners i with k0(v) + i = k and
//                   bin_k(v) = j of g_v * c_i(v).
// Three launches:
//   k_adj     one CTA per chunk of an inter-kernel cell: streams the input and
//             the upstream gradient, accumulates g * c_i into the cell's 2^D
//             corner tables in shared memory (float reductions) and writes
//             them as the chunk's partial table gradients;
//   k_lutbwd  one CTA per kernel: sums the partials of the cells around the
//             kernel in a fixed order (deterministic), folds the padded table
//             indices, stores dL/dlut, and takes the reverse of clip,
//             redistribute, cumulative sum and normalisation:
//               dL/dT = (1/den) [sum_j g_j (A_j - A_0 - j N_c/nb)
//                                + (A_0 - N_c/nb) sum_j g_j lut_j],
//             den = C_{nb-1} - C_0, A_j the clipped bins up to j (0 for a
//             constant CDF);
//   k_clipgrad one CTA: dL/dclip = V * sum_k dL/dT_k in a fixed order (0 when
//             the clip limit given lies outside [0, 1], where the forward
//             clamps it).
#include "hist_impl.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(256) k_adj(Geom g, const float *__restrict__ in,
                                             const float *__restrict__ gout,
                                             const float *__restrict__ lo_k,
                                             const float *__restrict__ scale_k,
                                             float *__restrict__ part, int chunks) {
    constexpr int NC = 1 << D;
    constexpr int NO = 1 << (D - 1);
    extern __shared__ __align__(16) float acc[];   // NC x P, corner-major
    __shared__ float s_nlo[NC], s_sc[NC];
    const int P = g.P, LS = g.LS;
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
    for (int i = threadIdx.x; i < NC * P; i += blockDim.x) acc[i] = 0.0f;
    if (threadIdx.x < NC) {
        int64_t k = kbase;
#pragma unroll
        for (int d = 0; d < D; ++d) k += ((threadIdx.x >> (D - 1 - d)) & 1) ? kstr[d] : 0;
        s_nlo[threadIdx.x] = -lo_k[k];
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

    float inv2b[kMaxDim];
    int mb[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Dim &dj = g.d[j];
        inv2b[j] = 1.0f / float(2 * dj.b);
        mb[j] = 2 * dj.p0 - (dj.b - 1) - 2 * dj.b * cc[j];
    }
    const uint32_t acc_s = uint32_t(__cvta_generic_to_shared(acc));
    const float iqk = g.iqk, qkf = g.qkf;
    float nl[NC], sc[NC];
    uint32_t cbase[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        nl[c] = s_nlo[c];
        sc[c] = s_sc[c];
        cbase[c] = acc_s + 4u * uint32_t(c * P) - kBinBias * 4u;
    }
    const int L = len[D - 1];
    const int xl = box_lo[D - 1];
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);
    const float inv2b_l = inv2b[D - 1];
    const int mb_l = mb[D - 1];

    struct BRow {
        float wo[NO];
    };
    auto row_fn = [&](const int *coords, int64_t, BRow &st) {
#pragma unroll
        for (int i = 0; i < NO; ++i) st.wo[i] = 1.0f;
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            const float w1 = float(2 * coords[j] + mb[j]) * inv2b[j];
            const float w0 = 1.0f - w1;
#pragma unroll
            for (int i = 0; i < NO; ++i) st.wo[i] *= ((i >> (D - 2 - j)) & 1) ? w1 : w0;
        }
    };
    auto quad_fn = [&](BRow &st, const QuadRef &q) {
        if (!q.has) return;
        const float vals[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
        const float gs[4] = {q.v2.x, q.v2.y, q.v2.z, q.v2.w};
        const float fb = float(2 * (xl + q.e0) + mb_l);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int el = q.e0 + e;
            if (el < 0 || el >= L) continue;
            const float w1 = (fb + float(2 * e)) * inv2b_l;
            const float w0 = 1.0f - w1;
            const float gw0 = gs[e] * w0, gw1 = gs[e] * w1;
            const uint32_t gbits = ADAPTIVE ? 0u : qbits1(vals[e], nl[0], sc[0], iqk, qkf);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint32_t b = ADAPTIVE ? qbits1(vals[e], nl[c], sc[c], iqk, qkf) : gbits;
                const float v = st.wo[c >> 1] * ((c & 1) ? gw1 : gw0);
                asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(b * 4u + cbase[c]), "f"(v)
                             : "memory");
            }
        }
    };
    walk_box<D, 4, BRow, true>(in, gout, g.N, stride, box_lo, len, r0, r1, same_align, true,
                               row_fn, quad_fn);
    __syncthreads();
    float *dst = part + (cell * chunks + chunk) * NC * LS;
    for (int i = threadIdx.x; i < NC * LS; i += blockDim.x) {
        const int c = i / LS, j = i - c * LS;
        dst[i] = j < P ? acc[c * P + j] : 0.0f;
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
                                                const float *__restrict__ part, int chunks,
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
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (cell_of[c] < 0) continue;
            const float *p = part + (cell_of[c] * chunks * NC + c) * LS + j;
            for (int ch = 0; ch < chunks; ++ch) s += p[int64_t(ch) * NC * LS];
        }
        G[j] = s;
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

size_t bwd_partial_floats(const Geom &g, int chunks) {
    return size_t(n_cells(g)) * size_t(chunks) * (size_t(1) << g.D) * size_t(g.LS);
}

template <int D>
static cudaError_t launch_bwd_d(const mclahe_plan_s &p, const float *in, const float *gout,
                                unsigned char *ws, const float *d_clip, float *d_grad_lut,
                                float *d_grad_clip, cudaStream_t st) {
    const Geom &g = p.g;
    const int chunks = p.t.bwd_chunks;
    float *part = reinterpret_cast<float *>(ws + p.ws.scratch);
    float *dT = part + bwd_partial_floats(g, chunks);
    const size_t smem_adj = (size_t(1) << D) * g.P * sizeof(float);
    const unsigned grid = unsigned(n_cells(g) * chunks);
    cudaError_t e;
    if (g.mode == MCLAHE_RANGE_ADAPTIVE) {
        e = cudaFuncSetAttribute(k_adj<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_adj));
        if (e != cudaSuccess) return e;
        k_adj<D, true><<<grid, 256, smem_adj, st>>>(g, in, gout, reinterpret_cast<const float *>(ws + p.ws.lo),
                                                    reinterpret_cast<const float *>(ws + p.ws.scale), part, chunks);
    } else {
        e = cudaFuncSetAttribute(k_adj<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_adj));
        if (e != cudaSuccess) return e;
        k_adj<D, false><<<grid, 256, smem_adj, st>>>(g, in, gout, reinterpret_cast<const float *>(ws + p.ws.lo),
                                                     reinterpret_cast<const float *>(ws + p.ws.scale), part, chunks);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem_lb = size_t(g.P) * sizeof(float) + size_t(g.nb) * sizeof(uint32_t);
    e = cudaFuncSetAttribute(k_lutbwd<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_lb));
    if (e != cudaSuccess) return e;
    k_lutbwd<D><<<unsigned(g.K), 256, smem_lb, st>>>(
        g, reinterpret_cast<const uint32_t *>(ws + p.ws.hist), reinterpret_cast<const float *>(ws + p.ws.lut),
        part, chunks, d_clip, d_grad_lut, dT);
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
