// mclahe_internal.cuh -- geometry, launch shapes and device helpers shared by the
// sm_103a kernels of the MCLAHE hot path.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mclahe.h"

namespace mclahe {

constexpr int kMaxDim = 4;
constexpr int kMaxBins = 4096;
constexpr size_t kWsAlign = 256;

// Unsigned 32-bit division by a runtime constant d >= 1 with one multiply-high
// (round-up method of Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994).  Exact for every 32-bit dividend.
struct FastDiv {
    uint32_t d, m, l;
    __host__ __device__ FastDiv() : d(1), m(0), l(0) {}
    __host__ explicit FastDiv(uint32_t div) : d(div) {
        l = 0;
        while ((uint64_t(1) << l) < div) ++l;           // l = ceil(log2 d)
        m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - div)) / div + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t x) const {
        if (d == 1) return x;
        uint32_t t = __umulhi(m, x);
        return (t + ((x - t) >> 1)) >> (l - 1);
    }
};

// Per-dimension geometry of the padded volume (Sec. III.B, Eq. (1)-(2)).
struct Dim {
    int32_t s;      // extent of the original volume
    int32_t b;      // kernel size
    int32_t p0;     // padding before
    int32_t p1;     // padding after
    int32_t n;      // kernels along this dim, (s + p) / b
    int32_t pad_;
    int64_t stride; // element stride of the original volume
};

// Everything a kernel needs about one volume; passed by value.
struct Geom {
    int32_t D;          // dimensionality, 1..4
    int32_t nb;         // n_bins
    int32_t mode;       // mclahe_range_mode
    int32_t has_range;  // GHR with a caller-given range
    float range_lo, range_hi;
    float clip;         // plan's clip limit
    int32_t pad_;
    int64_t K;          // kernels
    int64_t V;          // voxels per kernel
    int64_t N;          // voxels of the original volume
    Dim d[kMaxDim];
};

// Launch shapes chosen by the heuristic or the autotuner.
struct Tuning {
    int hist_threads;   // threads per histogram CTA
    int hist_chunks;    // CTAs per kernel in the range/histogram passes
    int map_threads;    // threads per mapping CTA
    int map_chunks;     // CTAs per inter-kernel cell in the mapping pass
};

// Workspace layout (byte offsets, kWsAlign aligned).
struct Layout {
    size_t status, keys, hist, lo, scale, lut, scratch, total;
    size_t keys_count;  // uint32 keys (2 for GHR, 2K for AHR)
    size_t scratch_bytes;
};

}  // namespace mclahe

struct mclahe_plan_s {
    mclahe::Geom g;
    mclahe::Tuning t;
    mclahe::Layout ws;
    int64_t pad[mclahe::kMaxDim];
    void *graph_cache;  // batch-mode graph owned by the first plan of a batch
};

namespace mclahe {

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Order-preserving map of a float to an unsigned key (for atomic min/max).
__device__ __forceinline__ uint32_t float_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Histogram range from the min key (stored complemented) and the max key.
__device__ __forceinline__ void keys_to_range(uint32_t nmin_key, uint32_t max_key, float &lo,
                                              float &hi) {
    lo = key_float(~nmin_key);
    hi = key_float(max_key);
}

// fp32 scale of a histogram range: n_bins / (hi - lo), 0 when hi <= lo.
__device__ __forceinline__ float range_scale(float lo, float hi, int nb) {
    return (hi > lo) ? __fdiv_rn(float(nb), __fsub_rn(hi, lo)) : 0.0f;
}

// Bin quantiser: clamp(floor(fp32(fp32(x - lo) * scale)), 0, nb - 1), each
// operation rounded to nearest with no contraction.  Clamping before the
// floor gives the same integer because the bounds are integers; NaN goes to
// bin 0.
__device__ __forceinline__ int quantise(float x, float lo, float scale, float top) {
    float y = __fmul_rn(__fsub_rn(x, lo), scale);
    y = fminf(fmaxf(y, 0.0f), top);
    return __float2int_rd(y);
}

// The same quantiser returning the bits of the float 2^23 + bin: after the
// clamp, y lies in [0, nb - 1], where adding 2^23 rounded down is exactly
// 2^23 + floor(y) (the float spacing there is 1).  Callers fold the constant
// 0x4B000000 into their address arithmetic, which avoids the quarter-rate
// float-to-int conversion.
constexpr uint32_t kBinBias = 0x4B000000u;   // bits of 2^23
__device__ __forceinline__ uint32_t quantise_bits(float x, float lo, float scale, float top) {
    float y = __fmul_rn(__fsub_rn(x, lo), scale);
    y = fminf(fmaxf(y, 0.0f), top);
    return __float_as_uint(__fadd_rd(y, 8388608.0f));
}

// Footprint of kernel k along one dimension: the original indices whose
// mirror images (Sec. III.B) fall in the padded interval [k*b, k*b + b).
// Multiplicity = number of images of x in that interval (0..3).
struct Foot {
    int32_t lo, hi;          // union, [lo, hi)
    int32_t ml, mh;          // main image
    int32_t ll, lh;          // reflected at the start
    int32_t rl, rh;          // reflected at the end
    __device__ __forceinline__ int mult(int x) const {
        return int(x >= ml && x < mh) + int(x >= ll && x < lh) + int(x >= rl && x < rh);
    }
};

__device__ __forceinline__ Foot footprint(const Dim &d, int k) {
    Foot f;
    const int P0 = k * d.b, P1 = P0 + d.b;          // padded interval
    f.ml = max(P0 - d.p0, 0);
    f.mh = min(P1 - d.p0, d.s);
    if (f.mh < f.ml) f.mh = f.ml;
    // padded P < p0 maps to x = p0 - 1 - P
    if (P0 < d.p0) {
        f.ll = d.p0 - min(P1, d.p0);
        f.lh = d.p0 - P0;
    } else {
        f.ll = f.lh = 0;
    }
    // padded P >= p0 + s maps to x = 2s - 1 - (P - p0)
    if (P1 > d.p0 + d.s) {
        f.rl = 2 * d.s - (P1 - d.p0);
        f.rh = 2 * d.s - max(P0 - d.p0, d.s);
    } else {
        f.rl = f.rh = 0;
    }
    f.lo = f.ml;
    f.hi = f.mh;
    if (f.lh > f.ll) {
        f.lo = min(f.lo, f.ll);
        f.hi = max(f.hi, f.lh);
    }
    if (f.rh > f.rl) {
        f.lo = min(f.lo, f.rl);
        f.hi = max(f.hi, f.rh);
    }
    return f;
}

// Original-index range [lo, hi) of inter-kernel cell c along one dimension:
// the voxels whose lower neighbouring kernel (largest k with centre
// k*b + (b-1)/2 <= x + p0, Sec. III.C) is c.
__device__ __forceinline__ void cell_range(const Dim &d, int c, int &lo, int &hi) {
    lo = c * d.b + d.b / 2 - d.p0;
    hi = lo + d.b;
    lo = min(max(lo, 0), d.s);
    hi = min(max(hi, 0), d.s);
}

// Iterator over the rows (all dims but the last) of a box, advancing by a
// fixed number of rows each step (mixed-radix add with carry).
template <int D>
struct RowIter {
    int c[kMaxDim];     // coordinates inside the box, dims 0..D-2
    int len[kMaxDim];
    int adv[kMaxDim];   // the step in the box's mixed radix
    __device__ __forceinline__ void init(const int *box_len, int start, int step) {
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            len[j] = box_len[j];
            c[j] = start % len[j];
            start /= len[j];
            adv[j] = step % len[j];
            step /= len[j];
        }
    }
    __device__ __forceinline__ void next() {
        int carry = 0;
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            int v = c[j] + adv[j] + carry;
            carry = v >= len[j];
            c[j] = carry ? v - len[j] : v;
        }
    }
};

// ---------------------------------------------------------------------------
// Row walker: the CTA visits rows [r0, r1) of a box (rows = all dims but the
// last, each row L contiguous elements from element xl of the last dim) in
// aligned 128-bit quads.  Every thread takes four quads per step, issuing the
// four loads before using them:
//   RU = 1: four quads of one row (lpr lanes share a row),
//   RU = 2: two quads from each of two rows (rows of at most 2 quads),
//   RU = 4: one quad from each of four rows (rows of 1 quad).
// The step count is the same for all threads of the block, so warp-wide
// primitives may be used inside.
// ---------------------------------------------------------------------------
struct WalkShape {
    int Q;      // quads per row (upper bound, including the alignment head)
    int ru;     // rows per thread step (1, 2 or 4)
    int lpr;    // lanes per row (RU = 1), else 1
    int ql;     // quads per lane per row (RU = 1)
    int G;      // row groups of the block (blockDim / lpr)
};

__device__ __forceinline__ WalkShape walk_shape(int L, int xl, bool same_align, int nthreads) {
    WalkShape w;
    w.Q = (((same_align ? (xl & 3) : 3) + L + 3) >> 2);
    if (w.Q <= 1) {
        w.ru = 4;
        w.lpr = 1;
        w.ql = 1;
    } else if (w.Q == 2) {
        w.ru = 2;
        w.lpr = 1;
        w.ql = 2;
    } else {
        w.ru = 1;
        const int want = (w.Q + 3) >> 2;
        int lpr = 1;
        while (lpr < want && lpr < 32) lpr <<= 1;
        w.lpr = lpr;
        w.ql = (w.Q + lpr - 1) / lpr;
    }
    w.G = nthreads / w.lpr;
    return w;
}

// One quad handed to the consumer: its four values, the element offset of its
// first element inside the row (may be negative for the alignment head), and
// its element address.
struct QuadRef {
    float4 v;
    int e0;
    int64_t a;
    bool has;   // overlaps the row
};

__device__ __forceinline__ float4 load_quad4(const float *__restrict__ in, int64_t a, int64_t N,
                                             bool has, bool stream) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (has) {
        if (a + 4 <= N) {
            v = stream ? __ldcs(reinterpret_cast<const float4 *>(in + a))
                       : __ldg(reinterpret_cast<const float4 *>(in + a));
        } else {
            v.x = in[a];
            if (a + 1 < N) v.y = in[a + 1];
            if (a + 2 < N) v.z = in[a + 2];
        }
    }
    return v;
}

// Walks the rows of a box.  row_fn(const int *coords, int64_t row_start, S &state)
// prepares per-row state S; quad_fn(S &state, const QuadRef &q) consumes one
// quad.  Template parameter RU must equal shape.ru.
template <int D, int RU, typename S, typename RowFn, typename QuadFn>
__device__ __forceinline__ void walk_rows(const float *__restrict__ in, int64_t N,
                                          const int64_t *stride, const int *box_lo,
                                          const int *box_len, int r0, int r1,
                                          const WalkShape &w, bool stream, RowFn row_fn,
                                          QuadFn quad_fn) {
    const int L = box_len[D - 1];
    const int xl = box_lo[D - 1];
    const int grp = threadIdx.x / w.lpr, gl = threadIdx.x & (w.lpr - 1);
    const int rows = r1 - r0;
    const int row_steps = (rows + w.G * RU - 1) / (w.G * RU);
    RowIter<D> it;
    it.init(box_len, r0 + grp, w.G);
    for (int rs = 0; rs < row_steps; ++rs) {
        S st[RU];
        int64_t start[RU];
        bool row_ok[RU];
#pragma unroll
        for (int ru = 0; ru < RU; ++ru) {
            const int r = grp + (rs * RU + ru) * w.G;
            row_ok[ru] = r < rows;
            int64_t s = xl;
            int coords[kMaxDim];
#pragma unroll
            for (int j = 0; j < D - 1; ++j) {
                coords[j] = box_lo[j] + it.c[j];
                s += int64_t(coords[j]) * stride[j];
            }
            start[ru] = s;
            row_fn(coords, s, st[ru]);
            it.next();
        }
        const int qsteps = (RU == 1) ? (w.ql + 3) >> 2 : 1;
        for (int qs = 0; qs < qsteps; ++qs) {
            QuadRef q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ru = (RU == 1) ? 0 : (RU == 2 ? (u >> 1) : u);
                const int qi = (RU == 1) ? (gl + (qs * 4 + u) * w.lpr) : (RU == 2 ? (u & 1) : 0);
                const int64_t qbase = start[ru] & ~int64_t(3);
                const int head = int(start[ru] - qbase);
                q[u].e0 = 4 * qi - head;
                q[u].a = qbase + 4 * int64_t(qi);
                const bool inl = (RU == 1) ? ((qs * 4 + u) < w.ql) : true;
                q[u].has = row_ok[ru] && inl && q[u].e0 < L && q[u].e0 + 4 > 0;
                q[u].v = load_quad4(in, q[u].a, N, q[u].has, stream);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ru = (RU == 1) ? 0 : (RU == 2 ? (u >> 1) : u);
                quad_fn(st[ru], q[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------
cudaError_t launch_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                         cudaStream_t st);
cudaError_t launch_hist(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                        const float *d_clip, cudaStream_t st);
cudaError_t launch_map(const mclahe_plan_s &p, const float *in, float *out,
                       const unsigned char *ws, cudaStream_t st);

// plan.cu
int device_sms();
int64_t n_cells(const Geom &g);
Tuning default_tuning(const Geom &g);
Layout make_layout(const Geom &g);
mclahe_status check_forward_args(const mclahe_plan_s *p, const void *in, const void *out,
                                 const void *ws, size_t ws_bytes);
mclahe_status forward_impl(const mclahe_plan_s &p, const float *in, float *out, unsigned char *ws,
                           const float *d_clip, cudaStream_t st);

// batch.cu
void release_graph_cache(mclahe_plan_s *p);

}  // namespace mclahe
