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
// Each launch covers up to 32 volumes of one plan (blockIdx.y), so a batch of
// small volumes fills the GPU in three launches (mclahe_backward_batch).
// No atomics: the result depends only on the launch shape (deterministic).
#include <algorithm>

#include "hist_impl.cuh"
#include "map_impl.cuh"

namespace mclahe {

// The volumes of one launch (blockIdx.y): the same plan, each its own input,
// upstream gradient, workspace and clip-limit slot.
constexpr int kBwdVols = 32;
struct BwdVols {
    const float *in[kBwdVols];
    const float *gout[kBwdVols];
    unsigned char *ws[kBwdVols];
    float *gclip[kBwdVols];
};

// Where the gather's scratch lies in a workspace.
struct GatherLayout {
    size_t hist, lut, lo, scale, dtab, partial;
};

__global__ void __launch_bounds__(256) k_dtab(Geom g, const __grid_constant__ BwdVols v, GatherLayout L,
                                              const float *__restrict__ d_clip) {
    extern __shared__ __align__(16) uint32_t h[];   // nb counts
    __shared__ float s_last;
    const int nb = g.nb, LS = g.LS;
    const int64_t k = blockIdx.x;
    unsigned char *ws = v.ws[blockIdx.y];
    const uint32_t *hist = reinterpret_cast<const uint32_t *>(ws + L.hist);
    const float *lut = reinterpret_cast<const float *>(ws + L.lut);
    float *dtab = reinterpret_cast<float *>(ws + L.dtab);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) h[j] = __ldcg(hist + k * nb + j);
    __syncthreads();
    const LutStats st = lut_stats(h, nb, g.V, load_clip(d_clip ? d_clip + blockIdx.y : nullptr, g.clip));
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
    k_mapdot(Geom g, const __grid_constant__ BwdVols v, GatherLayout L, int chunks) {
    extern __shared__ __align__(16) float tab[];
    const int64_t cell = blockIdx.x / chunks;
    const int chunk = int(blockIdx.x - cell * chunks);
    const unsigned char *ws = v.ws[blockIdx.y];
    float2 kd;
    map_cell<D, ADAPTIVE, REPL, D >= 3 ? kWalkRing : kWalkLsu, true>(
        g, v.in[blockIdx.y], nullptr, reinterpret_cast<const float *>(ws + L.dtab),
        reinterpret_cast<const float *>(ws + L.lo), reinterpret_cast<const float *>(ws + L.scale), cell,
        chunk, chunks, tab, nullptr, -1, v.gout[blockIdx.y], &kd);
    const double s = block_sum_d(double(kd.x) - double(kd.y));
    if (threadIdx.x == 0)
        reinterpret_cast<double *>(v.ws[blockIdx.y] + L.partial)[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_clipsum(const __grid_constant__ BwdVols v, GatherLayout L, int n,
                                                 int64_t V, const float *__restrict__ d_clip,
                                                 float plan_clip) {
    const double *partial = reinterpret_cast<const double *>(v.ws[blockIdx.x] + L.partial);
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    s = block_sum_d(s);
    if (threadIdx.x == 0) {
        const float raw = d_clip ? d_clip[blockIdx.x] : plan_clip;
        v.gclip[blockIdx.x][0] = (raw >= 0.0f && raw <= 1.0f) ? float(double(V) * s) : 0.0f;
    }
}

// Scratch of the gather: D tables [K][LS] floats, then one double per CTA.
size_t bwd_gather_bytes(const Geom &g, int chunks) {
    const size_t tab = (sizeof(float) * size_t(g.K) * g.LS + 255) & ~size_t(255);
    return tab + sizeof(double) * size_t(n_cells(g)) * size_t(chunks);
}

static GatherLayout gather_layout(const mclahe_plan_s &p) {
    GatherLayout L;
    L.hist = p.ws.hist;
    L.lut = p.ws.lut;
    L.lo = p.ws.lo;
    L.scale = p.ws.scale;
    L.dtab = p.ws.scratch;
    L.partial = p.ws.scratch + ((sizeof(float) * size_t(p.g.K) * p.g.LS + 255) & ~size_t(255));
    return L;
}

// One launch of each kernel over nv (<= kBwdVols) volumes; d_clip (nullable)
// points at the first of their clip limits.
template <int D>
static cudaError_t launch_gather_d(const mclahe_plan_s &p, const BwdVols &v, int nv,
                                   const float *d_clip, cudaStream_t st) {
    const Geom &g = p.g;
    const int chunks = p.t.bwd_chunks;
    const GatherLayout L = gather_layout(p);
    const size_t smem_h = sizeof(uint32_t) * size_t(g.nb);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_dtab), smem_h);
    if (e != cudaSuccess) return e;
    k_dtab<<<dim3(unsigned(g.K), unsigned(nv)), 256, smem_h, st>>>(g, v, L, d_clip);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned grid = unsigned(n_cells(g) * chunks);
    const size_t smem = dot_smem_for(D, g.P);
    const bool a = g.mode == MCLAHE_RANGE_ADAPTIVE, repl = map_repl_fits(g.P);
#define MCLAHE_DOT(A, R)                                                                    \
    e = ensure_smem(reinterpret_cast<const void *>(k_mapdot<D, A, R>), smem);              \
    if (e != cudaSuccess) return e;                                                         \
    k_mapdot<D, A, R><<<dim3(grid, unsigned(nv)), 256, smem, st>>>(g, v, L, chunks);
    if (a) {
        if (repl) { MCLAHE_DOT(true, true) } else { MCLAHE_DOT(true, false) }
    } else {
        if (repl) { MCLAHE_DOT(false, true) } else { MCLAHE_DOT(false, false) }
    }
#undef MCLAHE_DOT
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_clipsum<<<unsigned(nv), 256, 0, st>>>(v, L, int(grid), g.V, d_clip, g.clip);
    return cudaGetLastError();
}

static cudaError_t launch_gather(const mclahe_plan_s &p, const BwdVols &v, int nv, const float *d_clip,
                                 cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_gather_d<1>(p, v, nv, d_clip, st);
        case 2: return launch_gather_d<2>(p, v, nv, d_clip, st);
        case 3: return launch_gather_d<3>(p, v, nv, d_clip, st);
        case 4: return launch_gather_d<4>(p, v, nv, d_clip, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_backward_gather(const mclahe_plan_s &p, const float *in, const float *gout,
                                   unsigned char *ws, const float *d_clip, float *d_grad_clip,
                                   cudaStream_t st) {
    BwdVols v{};
    v.in[0] = in;
    v.gout[0] = gout;
    v.ws[0] = ws;
    v.gclip[0] = d_grad_clip;
    return launch_gather(p, v, 1, d_clip, st);
}

cudaError_t launch_backward_gather_many(const mclahe_plan_s &p, int n_vol, const float *const *in,
                                        const float *const *gout, void *const *ws,
                                        const float *d_clip, float *d_grad_clip, cudaStream_t st) {
    for (int v0 = 0; v0 < n_vol; v0 += kBwdVols) {
        const int nv = std::min(kBwdVols, n_vol - v0);
        BwdVols v{};
        for (int i = 0; i < nv; ++i) {
            v.in[i] = in[v0 + i];
            v.gout[i] = gout[v0 + i];
            v.ws[i] = static_cast<unsigned char *>(ws[v0 + i]);
            v.gclip[i] = d_grad_clip + v0 + i;
        }
        const cudaError_t e = launch_gather(p, v, nv, d_clip ? d_clip + v0 : nullptr, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mclahe
