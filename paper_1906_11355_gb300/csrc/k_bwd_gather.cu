// k_bwd_gather.cu -- the clip-limit gradient of the forward pass without the
// table gradients (mclahe_backward with d_grad_lut = NULL): a gather instead
// of the adjoint's scatter.
//
// With G[k][j] = dL/dlut[k][j] = sum over voxels v and corners i with
// k0(v) + i = k, bin_k(v) = j of g_v c_i(v) (Sec. III.C, Eq. (12)-(13)), the
// clip-limit gradient is
//   dL/dclip = V sum_k sum_j G[k][j] D[k][j],  D[k][j] = d lut_kj / dT,
// and reordering the double sum over voxels gives
//   dL/dclip = V sum_v g_v sum_i c_i(v) D[k0(v) + i][bin(v)],
// that is, the mapping pass of Sec. III.C with the tables D in place of the
// mapping tables, dotted with the upstream gradient.  Three launches:
//   k_dtab      one CTA per kernel: D[k][j] from the kernel's histogram and
//               table (the reverse of clip, redistribute, cumulative sum and
//               normalisation of Algorithm 1):
//                 D_j = [(A_j - A_0 - j N_c/nb) + lut_j (A_0 - N_c/nb)] / den,
//               den = C_{nb-1} - C_0, A_j the clipped bins up to j, 0 for a
//               constant CDF; padded indices >= nb - 1 repeat D_{nb-1};
//   k_mapdot    one CTA per chunk of a cell: every voxel's interpolated D
//               times g_v, summed per thread (compensated), per block in
//               double in a fixed tree, one partial per CTA;
//   k_clipsum   one CTA: the partials in a fixed order, times V (0 when the
//               clip limit given lies outside [0, 1], where the forward
//               clamps it).
// No atomics: the result depends only on the launch shape (deterministic).
#include <algorithm>

#include "hist_impl.cuh"
#include "map_impl.cuh"

namespace mclahe {

__global__ void __launch_bounds__(256) k_dtab(Geom g, const uint32_t *__restrict__ hist,
                                              const float *__restrict__ lut,
                                              const float *__restrict__ d_clip,
                                              float *__restrict__ dtab) {
    extern __shared__ __align__(16) uint32_t h[];   // nb counts
    __shared__ float s_last;
    const int nb = g.nb, LS = g.LS;
    const int64_t k = blockIdx.x;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) h[j] = __ldcg(hist + k * nb + j);
    __syncthreads();
    const LutStats st = lut_stats(h, nb, g.V, load_clip(d_clip, g.clip));
    const float ncb = __fdiv_rn(float(st.N_c), float(nb));
    const float c2 = __fsub_rn(float(st.A0), ncb);
    int64_t Aj = st.pa;
    for (int j = st.j0; j < st.j1; ++j) {
        if (int64_t(h[j]) > st.tf) Aj += 1;
        float d = 0.0f;
        if (!st.flat) {
            const float a = __fsub_rn(float(Aj - st.A0), __fmul_rn(float(j), ncb));
            d = __fdiv_rn(__fadd_rn(a, __fmul_rn(__ldcg(lut + k * LS + j), c2)), st.den);
        }
        dtab[k * LS + j] = d;
        if (j == nb - 1) s_last = d;
    }
    __syncthreads();
    for (int j = nb + int(threadIdx.x); j < LS; j += blockDim.x) dtab[k * LS + j] = s_last;
}

// Deterministic block sum in double (fixed shuffle tree, then the warps in
// order); valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double s_w[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += s_w[w];
    __syncthreads();
    return s;
}

template <int D, bool ADAPTIVE, bool REPL>
__global__ void __launch_bounds__(256, D >= 4 && ADAPTIVE ? 1 : 2)
    k_mapdot(Geom g, const float *__restrict__ in, const float *__restrict__ gout,
             const float *__restrict__ dtab, const float *__restrict__ lo_k,
             const float *__restrict__ scale_k, int chunks, double *__restrict__ partial) {
    extern __shared__ __align__(16) float tab[];
    const int64_t cell = blockIdx.x / chunks;
    const int chunk = int(blockIdx.x - cell * chunks);
    float2 kd;
    map_cell<D, ADAPTIVE, REPL, kWalkLsu, true>(g, in, nullptr, dtab, lo_k, scale_k, cell, chunk,
                                                chunks, tab, nullptr, -1, gout, &kd);
    const double s = block_sum_d(double(kd.x) - double(kd.y));
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_clipsum(const double *__restrict__ partial, int n,
                                                 int64_t V, const float *__restrict__ d_clip,
                                                 float plan_clip, float *__restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    s = block_sum_d(s);
    if (threadIdx.x == 0) {
        const float raw = d_clip ? *d_clip : plan_clip;
        out[0] = (raw >= 0.0f && raw <= 1.0f) ? float(double(V) * s) : 0.0f;
    }
}

// Scratch of the gather: D tables [K][LS] floats, then one double per CTA.
size_t bwd_gather_bytes(const Geom &g, int chunks) {
    const size_t tab = (sizeof(float) * size_t(g.K) * g.LS + 255) & ~size_t(255);
    return tab + sizeof(double) * size_t(n_cells(g)) * size_t(chunks);
}

template <int D>
static cudaError_t launch_gather_d(const mclahe_plan_s &p, const float *in, const float *gout,
                                   unsigned char *ws, const float *d_clip, float *d_grad_clip,
                                   cudaStream_t st) {
    const Geom &g = p.g;
    const int chunks = p.t.bwd_chunks;
    float *dtab = reinterpret_cast<float *>(ws + p.ws.scratch);
    double *partial = reinterpret_cast<double *>(
        ws + p.ws.scratch + ((sizeof(float) * size_t(g.K) * g.LS + 255) & ~size_t(255)));
    const size_t smem_h = sizeof(uint32_t) * size_t(g.nb);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_dtab), smem_h);
    if (e != cudaSuccess) return e;
    k_dtab<<<unsigned(g.K), 256, smem_h, st>>>(g, reinterpret_cast<const uint32_t *>(ws + p.ws.hist),
                                               reinterpret_cast<const float *>(ws + p.ws.lut), d_clip,
                                               dtab);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned grid = unsigned(n_cells(g) * chunks);
    const size_t smem = map_smem_for(D, g.P, false);
    const float *lo = reinterpret_cast<const float *>(ws + p.ws.lo);
    const float *sc = reinterpret_cast<const float *>(ws + p.ws.scale);
    const bool a = g.mode == MCLAHE_RANGE_ADAPTIVE, repl = map_repl_fits(g.P);
#define MCLAHE_DOT(A, R)                                                                    \
    e = ensure_smem(reinterpret_cast<const void *>(k_mapdot<D, A, R>), smem);              \
    if (e != cudaSuccess) return e;                                                         \
    k_mapdot<D, A, R><<<grid, 256, smem, st>>>(g, in, gout, dtab, lo, sc, chunks, partial);
    if (a) {
        if (repl) { MCLAHE_DOT(true, true) } else { MCLAHE_DOT(true, false) }
    } else {
        if (repl) { MCLAHE_DOT(false, true) } else { MCLAHE_DOT(false, false) }
    }
#undef MCLAHE_DOT
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_clipsum<<<1, 256, 0, st>>>(partial, int(grid), g.V, d_clip, g.clip, d_grad_clip);
    return cudaGetLastError();
}

cudaError_t launch_backward_gather(const mclahe_plan_s &p, const float *in, const float *gout,
                                   unsigned char *ws, const float *d_clip, float *d_grad_clip,
                                   cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_gather_d<1>(p, in, gout, ws, d_clip, d_grad_clip, st);
        case 2: return launch_gather_d<2>(p, in, gout, ws, d_clip, d_grad_clip, st);
        case 3: return launch_gather_d<3>(p, in, gout, ws, d_clip, d_grad_clip, st);
        case 4: return launch_gather_d<4>(p, in, gout, ws, d_clip, d_grad_clip, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
