// k_hist.cu -- per-kernel intensity histograms (Algorithm 1, histogram step).
//
// The padded volume of Sec. III.B is never built.  Each CTA takes one kernel
// (or one chunk of its rows) and reads the kernel's footprint in the original
// volume: the original voxels with at least one mirror image inside the
// kernel.  A voxel counts once per image (its multiplicity, a product of
// per-dimension factors in {1, 2, 3}), which gives exactly the histogram of
// the padded kernel while every voxel is read from HBM about once.
//
// Loads are 128-bit and coalesced along the contiguous dimension; bins are
// privatised per CTA in shared memory; equal bins within a warp are merged
// with __match_any_sync before the shared-memory atomic; the CTA's bins are
// merged into the global table with integer atomics, which makes the result
// independent of the order in which CTAs finish.
#include "mclahe_internal.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(256) k_hist(Geom g, const float *__restrict__ in,
                                              const uint32_t *__restrict__ keys,
                                              uint32_t *__restrict__ hist, int chunks) {
    extern __shared__ uint32_t sh[];
    const int nb = g.nb;
    const int64_t k = blockIdx.x / chunks;
    const int chunk = blockIdx.x - int(k * chunks);

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

    float lo, hi;
    if (ADAPTIVE) {
        keys_to_range(keys[2 * k], keys[2 * k + 1], lo, hi);
    } else if (g.has_range) {
        lo = g.range_lo;
        hi = g.range_hi;
    } else {
        keys_to_range(keys[0], keys[1], lo, hi);
    }
    const float scale = range_scale(lo, hi, nb);
    const float top = float(nb - 1);

    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();

    // Row layout: rows of the footprint box along dims 0..D-2, each row L
    // contiguous elements starting at xl along dim D-1.  A row is covered by
    // aligned quads; rows start at the same alignment when the row stride is
    // a multiple of 4 (or there is one row).
    const int L = len[D - 1];
    const int xl = f[D - 1].lo;
    const bool same_align = (D == 1) || ((g.d[D >= 2 ? D - 2 : 0].stride & 3) == 0);
    const int Q = (((same_align ? (xl & 3) : 3) + L + 3) >> 2);  // quads per row (bound)
    int lpr = 1;
    while (lpr < Q && lpr < 32) lpr <<= 1;                         // lanes per row
    const int groups = blockDim.x / lpr;
    const int grp = threadIdx.x / lpr, gl = threadIdx.x - grp * lpr;
    const int row_steps = (r1 - r0 + groups - 1) / groups;          // block-uniform
    const int quad_steps = (Q + lpr - 1) / lpr;
    const int lane = threadIdx.x & 31;

    RowIter<D> it;
    it.init(len, r0 + grp, groups);
    for (int rs = 0; rs < row_steps; ++rs) {
        const int r = r0 + grp + rs * groups;
        const bool row_ok = r < r1;
        int64_t row_start = xl;
        int wo = 1;  // multiplicity over dims 0..D-2
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            const int x = f[j].lo + it.c[j];
            row_start += int64_t(x) * g.d[j].stride;
            wo *= f[j].mult(x);
        }
        const int64_t qbase = row_start & ~int64_t(3);
        for (int qs = 0; qs < quad_steps; ++qs) {
            const int q = gl + qs * lpr;
            const int64_t a = qbase + 4 * int64_t(q);
            float v[4];
            int w[4];
            bool any = false;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t idx = a + e;
                const bool ok = row_ok && q < Q && idx >= row_start && idx < row_start + L;
                w[e] = ok ? wo * f[D - 1].mult(int(idx - row_start) + xl) : 0;
                any |= ok;
            }
            if (any) {
                if (a + 4 <= g.N) {
                    const float4 t = __ldg(reinterpret_cast<const float4 *>(in + a));
                    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e] = (w[e] > 0) ? in[a + e] : 0.0f;
                }
            }
            // weights above one only occur near the volume's faces
            const bool unit = __all_sync(0xffffffffu, w[0] <= 1 && w[1] <= 1 && w[2] <= 1 && w[3] <= 1);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int bin = (w[e] > 0) ? quantise(v[e], lo, scale, top) : -1;
                if (unit) {
                    const unsigned peers = __match_any_sync(0xffffffffu, bin);
                    if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&sh[bin], __popc(peers));
                } else if (bin >= 0) {
                    atomicAdd(&sh[bin], uint32_t(w[e]));
                }
            }
        }
        it.next();
    }
    __syncthreads();
    uint32_t *gh = hist + k * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const uint32_t c = sh[i];
        if (c) atomicAdd(&gh[i], c);
    }
}

template <int D>
static cudaError_t launch_hist_d(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                 cudaStream_t st) {
    const Geom &g = p.g;
    const uint32_t *keys = reinterpret_cast<const uint32_t *>(ws + p.ws.keys);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + p.ws.hist);
    const int chunks = p.t.hist_chunks;
    const unsigned grid = unsigned(g.K * chunks);
    const size_t smem = size_t(g.nb) * sizeof(uint32_t);
    if (g.mode == MCLAHE_RANGE_ADAPTIVE)
        k_hist<D, true><<<grid, p.t.hist_threads, smem, st>>>(g, in, keys, hist, chunks);
    else
        k_hist<D, false><<<grid, p.t.hist_threads, smem, st>>>(g, in, keys, hist, chunks);
    return cudaGetLastError();
}

cudaError_t launch_hist(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                        cudaStream_t st) {
    switch (p.g.D) {
        case 1: return launch_hist_d<1>(p, in, ws, st);
        case 2: return launch_hist_d<2>(p, in, ws, st);
        case 3: return launch_hist_d<3>(p, in, ws, st);
        case 4: return launch_hist_d<4>(p, in, ws, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
