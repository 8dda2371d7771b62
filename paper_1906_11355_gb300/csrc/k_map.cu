// k_map.cu -- intensity mapping by multilinear interpolation (Sec. III.C,
// Eq. (12)-(13); Algorithm 1, the interpolation loop).
//
// Voxels that share the same 2^D nearest kernels form an inter-kernel cell
// (the dotted regions of Fig. 2).  Each CTA takes one cell (or a chunk of its
// rows), stages the 2^D neighbouring mapping tables in shared memory, then
// streams its voxels: 128-bit loads, the bin of each voxel under every
// neighbour's range (one bin for a global range), the table values at those
// bins, and the Lagrange blend
//   out = sum_i prod_j w_{i_j, j} * lut[k0 + i][bin_{k0+i}(x)],
//   w_{1,j} = d_{j0} / b_j,  w_{0,j} = 1 - w_{1,j},
// where d_{j0} = (x_j + p_j0) - (k0_j b_j + (b_j - 1) / 2) is the distance to
// the lower kernel's centre.
#include "mclahe_internal.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(256) k_map(Geom g, const float *__restrict__ in,
                                             float *__restrict__ out,
                                             const float *__restrict__ lut,
                                             const float *__restrict__ lo_k,
                                             const float *__restrict__ scale_k, int chunks) {
    constexpr int NC = 1 << D;          // corners
    constexpr int NO = 1 << (D - 1);    // corners over dims 0..D-2
    extern __shared__ float tab[];      // [NC][nb]
    __shared__ float s_lo[NC], s_sc[NC];
    const int nb = g.nb;

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
    // stage the neighbouring kernels' tables; corner i has bit (D-1-j) = side along dim j
    for (int t = threadIdx.x; t < NC * nb; t += blockDim.x) {
        const int i = t / nb, j = t - i * nb;
        int64_t k = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) k = k * g.d[d].n + cc[d] + ((i >> (D - 1 - d)) & 1);
        tab[t] = lut[k * nb + j];
        if (j == 0) {
            s_lo[i] = lo_k[k];
            s_sc[i] = scale_k[k];
        }
    }

    int lo[kMaxDim], len[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        int a, b;
        cell_range(g.d[j], cc[j], a, b);
        lo[j] = a;
        len[j] = b - a;
    }
    int R = 1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) R *= len[j];
    const int r0 = int((int64_t(R) * chunk) / chunks);
    const int r1 = int((int64_t(R) * (chunk + 1)) / chunks);
    __syncthreads();

    const float top = float(nb - 1);
    const float glo = s_lo[0], gsc = s_sc[0];
    // last-dim weight: w1 = m / (2b), m = 2(x + p0) - (b - 1) - 2b c
    const Dim dl = g.d[D - 1];
    const float inv2b_l = 1.0f / float(2 * dl.b);
    const int mbase_l = 2 * dl.p0 - (dl.b - 1) - 2 * dl.b * cc[D - 1];

    const int L = len[D - 1];
    const int xl = lo[D - 1];
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);
    const int Q = (((same_align ? (xl & 3) : 3) + L + 3) >> 2);
    int lpr = 1;
    while (lpr < Q && lpr < 32) lpr <<= 1;
    const int groups = blockDim.x / lpr;
    const int grp = threadIdx.x / lpr, gl = threadIdx.x - grp * lpr;

    RowIter<D> it;
    it.init(len, r0 + grp, groups);
    for (int r = r0 + grp; r < r1; r += groups) {
        int64_t row_start = xl;
        float wo[NO];
#pragma unroll
        for (int i = 0; i < NO; ++i) wo[i] = 1.0f;
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            const Dim &dj = g.d[j];
            const int x = lo[j] + it.c[j];
            row_start += int64_t(x) * dj.stride;
            const int m = 2 * (x + dj.p0) - (dj.b - 1) - 2 * dj.b * cc[j];
            const float w1 = __fdiv_rn(float(m), float(2 * dj.b));
            const float w0 = 1.0f - w1;
#pragma unroll
            for (int i = 0; i < NO; ++i) wo[i] *= ((i >> (D - 2 - j)) & 1) ? w1 : w0;
        }
        const int64_t qbase = row_start & ~int64_t(3);
        for (int q = gl; q < Q; q += lpr) {
            const int64_t a = qbase + 4 * int64_t(q);
            bool ok[4];
            bool all = true, any = false;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ok[e] = (a + e >= row_start) && (a + e < row_start + L);
                all &= ok[e];
                any |= ok[e];
            }
            if (!any) continue;
            float v[4];
            const bool vec = a + 4 <= g.N;
            if (vec) {
                const float4 t = __ldcs(reinterpret_cast<const float4 *>(in + a));
                v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = ok[e] ? in[a + e] : 0.0f;
            }
            float res[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = int(a + e - row_start) + xl;
                const float w1 = float(2 * x + mbase_l) * inv2b_l;
                const float w0 = 1.0f - w1;
                float acc = 0.0f;
                if (ADAPTIVE) {
#pragma unroll
                    for (int i = 0; i < NO; ++i) {
                        const int c0 = 2 * i, c1 = 2 * i + 1;
                        const int b0 = quantise(v[e], s_lo[c0], s_sc[c0], top);
                        const int b1 = quantise(v[e], s_lo[c1], s_sc[c1], top);
                        acc += wo[i] * (w0 * tab[c0 * nb + b0] + w1 * tab[c1 * nb + b1]);
                    }
                } else {
                    const int bn = quantise(v[e], glo, gsc, top);
#pragma unroll
                    for (int i = 0; i < NO; ++i)
                        acc += wo[i] * (w0 * tab[(2 * i) * nb + bn] + w1 * tab[(2 * i + 1) * nb + bn]);
                }
                res[e] = acc;
            }
            if (all && vec) {
                __stcs(reinterpret_cast<float4 *>(out + a), make_float4(res[0], res[1], res[2], res[3]));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (ok[e]) out[a + e] = res[e];
            }
        }
        it.next();
    }
}

template <int D>
static cudaError_t launch_map_d(const mclahe_plan_s &p, const float *in, float *out,
                                const unsigned char *ws, cudaStream_t st) {
    const Geom &g = p.g;
    int64_t cells = 1;
    for (int j = 0; j < D; ++j) cells *= (g.d[j].n - 1);
    const int chunks = p.t.map_chunks;
    const unsigned grid = unsigned(cells * chunks);
    const size_t smem = size_t(1 << D) * g.nb * sizeof(float);
    const float *lut = reinterpret_cast<const float *>(ws + p.ws.lut);
    const float *lo = reinterpret_cast<const float *>(ws + p.ws.lo);
    const float *sc = reinterpret_cast<const float *>(ws + p.ws.scale);
    cudaError_t e;
    if (g.mode == MCLAHE_RANGE_ADAPTIVE) {
        e = cudaFuncSetAttribute(k_map<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_map<D, true><<<grid, p.t.map_threads, smem, st>>>(g, in, out, lut, lo, sc, chunks);
    } else {
        e = cudaFuncSetAttribute(k_map<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_map<D, false><<<grid, p.t.map_threads, smem, st>>>(g, in, out, lut, lo, sc, chunks);
    }
    return cudaGetLastError();
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
