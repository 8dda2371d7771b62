// mclahe_internal.cuh -- geometry, launch shapes and device helpers shared by the
// sm_103a kernels of the MCLAHE hot path.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>

#include "mclahe.h"

namespace mclahe {

constexpr int kMaxDim = 4;
constexpr int kMaxBins = 4096;
constexpr size_t kWsAlign = 256;
constexpr int kMaxPieces = 5;     // constant-multiplicity pieces of a footprint per dim

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
//
// Table geometry.  The bin quantiser (see qbits below) yields an index in
// [0, qk], qk = the smallest power of two >= n_bins - 1, where every index
// >= n_bins - 1 stands for the last bin.  Mapping tables are therefore stored
// with P = qk + 1 entries (entries n_bins .. qk repeat entry n_bins - 1), in
// rows of LS >= P floats (LS a multiple of 4).
struct Geom {
    int32_t D;          // dimensionality, 1..4
    int32_t nb;         // n_bins
    int32_t mode;       // mclahe_range_mode
    int32_t has_range;  // GHR with a caller-given range
    float range_lo, range_hi;
    float clip;         // plan's clip limit
    int32_t qk;         // power of two >= nb - 1
    float qkf;          // qk as a float
    float iqk;          // 1 / qk (exact)
    int32_t P;          // table entries, qk + 1
    int32_t LS;         // table row stride in floats, P rounded up to 4
    int64_t K;          // kernels
    int64_t V;          // voxels per kernel
    int64_t N;          // voxels of the original volume
    Dim d[kMaxDim];
};

// Launch shapes chosen by the heuristic or the autotuner.
struct Tuning {
    int hist_threads;   // threads per histogram CTA (256; 512 for 4-D volumes)
    int hist_chunks;    // CTAs per kernel (cluster size) in the histogram pass
    int hist_copies;    // lane copies of the shared-memory histograms (1 .. 32)
    int hist_group;     // kernels along the last dimension per histogram work item
    int hist_shares;    // shares per work item in the flat histogram pass (0: one
                        // cluster of hist_chunks CTAs per work item)
    int map_threads;    // threads per mapping CTA
    int map_chunks;     // CTAs per inter-kernel cell in the mapping pass
    int map_tma;        // 1: stream 3- and 4-D cells as TMA tiles (where map_tma_box allows)
    int map_flat;       // 1: map_chunks shares per cell dealt out to a persistent grid
    int hist_walk;      // rows of the histogram pass: 0 cp.async ring, 1 TMA tiles (where
                        // hist_tma_box allows), 2 per-thread loads (least shared memory),
                        // 3 the kernel's footprint staged in shared memory (one kernel per
                        // cluster, where hist_staged_fits allows)
    int bwd_chunks;     // CTAs per inter-kernel cell in the backward pass (fixed by the plan)
    int range_pass;     // 1: an adaptive plan's per-kernel ranges come from k_range_kernels
                        // (one streaming sweep) before a cluster-form histogram pass,
                        // instead of a sweep of each footprint inside it (where
                        // range_pass_fits allows)
};

// Workspace layout (byte offsets, kWsAlign aligned).
struct Layout {
    size_t status, keys, tickets, hist, lo, scale, lut, scratch, total;
    size_t keys_count;  // uint32 range keys: the global range, then one pair per kernel
    size_t scratch_bytes;
};

}  // namespace mclahe

struct mclahe_plan_s {
    mclahe::Geom g;
    mclahe::Tuning t;
    mclahe::Layout ws;
    int64_t pad[mclahe::kMaxDim];
    int tuned;          // launch shapes come from mclahe_autotune
    mutable int flat_ctas = 0;   // grid of the last flat histogram launch
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

// ---------------------------------------------------------------------------
// Bin quantiser.  The reading of the histogram step of Algorithm 1 is
//   bin(x) = clamp(floor(y), 0, nb - 1),  y = fp32(fp32(x - lo) * scale),
// each operation rounded to nearest.  It is evaluated as
//   t = min(max(fp32(y * 2^-k), 0), 1)      (mul.rn.sat; exact scaling)
//   bits = fp32_rd(t * 2^k + 2^23)          (one fma rounded down)
// where 2^k = qk >= nb - 1.  Multiplying by a power of two is exact whenever
// the result is a normal number, and when it is not, y < 1 and both forms give
// index 0; so t * 2^k = clamp(y, 0, 2^k) exactly, and adding 2^23 rounded
// down gives the float 2^23 + floor(clamp(y, 0, 2^k)), whose bits are
// kBinBias + index with index in [0, qk].  Every index >= nb - 1 stands for
// bin nb - 1 (tables are padded, histograms fold them).  NaN saturates to 0.
// The pair form runs two values through the packed f32x2 instructions.
// ---------------------------------------------------------------------------
constexpr uint32_t kBinBias = 0x4B000000u;   // bits of 2^23
constexpr float kTwo23 = 8388608.0f;

__device__ __forceinline__ float mul_sat(float a, float b) {
    float r;
    asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

struct QRange {
    float nlo;     // -lo
    float sc;      // scale
};

// Two values under two (possibly equal) ranges: returns kBinBias + index.
__device__ __forceinline__ uint2 qbits2(float2 x, float2 nlo, float2 sc, float iqk, float qkf) {
    float2 y = __fmul2_rn(__fadd2_rn(x, nlo), sc);
    y.x = mul_sat(y.x, iqk);
    y.y = mul_sat(y.y, iqk);
    y = __ffma2_rd(y, make_float2(qkf, qkf), make_float2(kTwo23, kTwo23));
    return make_uint2(__float_as_uint(y.x), __float_as_uint(y.y));
}

// qbits2 with the 2^-k of iqk folded into the scale (scq = sc * iqk).  Equal
// to qbits2 whenever scq is exact, that is, sc is zero, infinite, NaN or
// |sc| >= 2^-126 * qk, so that sc * 2^-k is a normal number before rounding
// (fold_exact; testing the rounded product instead would pass scales whose
// product rounds up to the smallest normal): 1/qk is a power of two, so
// rounding (x - lo) * scq equals rounding (x - lo) * sc and then scaling by
// 1/qk in the normal range, and a product below the normal range is bin 0
// either way.
__device__ __forceinline__ uint2 qbits2_folded(float2 x, float2 nlo, float2 scq, float qkf) {
    float2 y = __fadd2_rn(x, nlo);
    y.x = mul_sat(y.x, scq.x);
    y.y = mul_sat(y.y, scq.y);
    y = __ffma2_rd(y, make_float2(qkf, qkf), make_float2(kTwo23, kTwo23));
    return make_uint2(__float_as_uint(y.x), __float_as_uint(y.y));
}

__device__ __forceinline__ bool fold_exact(float sc, float qkf) {
    return sc == 0.0f || !(fabsf(sc) < 1.17549435e-38f * qkf);   // 2^-126 * qk, exact
}

__device__ __forceinline__ uint32_t qbits1(float x, float nlo, float sc, float iqk, float qkf) {
    float y = __fmul_rn(__fadd_rn(x, nlo), sc);
    y = mul_sat(y, iqk);
    return __float_as_uint(__fmaf_rd(y, qkf, kTwo23));
}

// ---------------------------------------------------------------------------
// Footprint of kernel k along one dimension: the original indices whose
// mirror images (Sec. III.B) fall in the padded interval [k*b, k*b + b).
// Multiplicity = number of images of x in that interval (0..3).
// ---------------------------------------------------------------------------
struct Foot {
    int32_t lo, hi;          // union, [lo, hi)
    int32_t ml, mh;          // main image
    int32_t ll, lh;          // reflected at the start
    int32_t rl, rh;          // reflected at the end
    __host__ __device__ __forceinline__ int mult(int x) const {
        return int(x >= ml && x < mh) + int(x >= ll && x < lh) + int(x >= rl && x < rh);
    }
};

__host__ __device__ __forceinline__ int imin_(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int imax_(int a, int b) { return a > b ? a : b; }

__host__ __device__ __forceinline__ Foot footprint(const Dim &d, int k) {
    Foot f;
    const int P0 = k * d.b, P1 = P0 + d.b;          // padded interval
    f.ml = imax_(P0 - d.p0, 0);
    f.mh = imin_(P1 - d.p0, d.s);
    if (f.mh < f.ml) f.mh = f.ml;
    // padded P < p0 maps to x = p0 - 1 - P
    if (P0 < d.p0) {
        f.ll = d.p0 - imin_(P1, d.p0);
        f.lh = d.p0 - P0;
    } else {
        f.ll = f.lh = 0;
    }
    // padded P >= p0 + s maps to x = 2s - 1 - (P - p0)
    if (P1 > d.p0 + d.s) {
        f.rl = 2 * d.s - (P1 - d.p0);
        f.rh = 2 * d.s - imax_(P0 - d.p0, d.s);
    } else {
        f.rl = f.rh = 0;
    }
    f.lo = f.ml;
    f.hi = f.mh;
    if (f.lh > f.ll) {
        f.lo = imin_(f.lo, f.ll);
        f.hi = imax_(f.hi, f.lh);
    }
    if (f.rh > f.rl) {
        f.lo = imin_(f.lo, f.rl);
        f.hi = imax_(f.hi, f.rh);
    }
    return f;
}

// The footprint split into intervals of constant nonzero multiplicity.
struct Pieces {
    int n;
    int a[kMaxPieces], e[kMaxPieces], m[kMaxPieces];   // [a, e) with multiplicity m
};

__host__ __device__ __forceinline__ Pieces footprint_pieces(const Dim &d, int k) {
    Pieces p;
    {   // interior kernel: one piece, the main image, multiplicity 1
        const int a = k * d.b - d.p0;
        if (a >= 0 && a + d.b <= d.s) {
            p.n = 1;
            p.a[0] = a;
            p.e[0] = a + d.b;
            p.m[0] = 1;
            return p;
        }
    }
    const Foot f = footprint(d, k);
    int bp[8];
    int nbp = 0;
    const int cand[8] = {f.lo, f.hi, f.ml, f.mh, f.ll, f.lh, f.rl, f.rh};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int v = cand[i];
        bool dup = v < f.lo || v > f.hi;
        for (int j = 0; j < nbp; ++j) dup |= (bp[j] == v);
        if (!dup) {
            int j = nbp++;
            while (j > 0 && bp[j - 1] > v) {   // insertion sort
                bp[j] = bp[j - 1];
                --j;
            }
            bp[j] = v;
        }
    }
    p.n = 0;
    for (int i = 0; i + 1 < nbp; ++i) {
        const int m = f.mult(bp[i]);
        if (m > 0 && p.n < kMaxPieces) {
            p.a[p.n] = bp[i];
            p.e[p.n] = bp[i + 1];
            p.m[p.n] = m;
            ++p.n;
        }
    }
    return p;
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

// Quotient and remainder of small non-negative integers (a < 2^24, 1 <= d <
// 2^24) through a float reciprocal, corrected to the exact integer result.
__device__ __forceinline__ int small_div(int a, int d, int &rem) {
    int q = __float2int_rz(__int2float_rz(a) * __frcp_rn(__int2float_rn(d)));
    int r = a - q * d;
    if (r < 0) {
        q -= 1;
        r += d;
    } else if (r >= d) {
        q += 1;
        r -= d;
    }
    rem = r;
    return q;
}

// Iterator over the rows (all dims but the last) of a box, advancing by a
// fixed number of rows each step (mixed-radix add with carry).  Row indices
// stay below 2^24 (the plan bounds a footprint's rows).
template <int D>
struct RowIter {
    int c[kMaxDim];     // coordinates inside the box, dims 0..D-2
    int len[kMaxDim];
    int adv[kMaxDim];   // the step in the box's mixed radix
    __device__ __forceinline__ void init(const int *box_len, int start, int step) {
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            len[j] = box_len[j];
            int r;
            start = small_div(start, len[j], r);
            c[j] = r;
            step = small_div(step, len[j], r);
            adv[j] = r;
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
// aligned 128-bit quads.  Every thread takes U quads per step (U = 2 or 4),
// issuing the U loads before using them:
//   RU = 1: U quads of one row (lpr lanes share a row),
//   RU = 2: U/2 quads from each of two rows (rows of at most U/2 quads),
//   RU = 4: one quad from each of four rows (U = 4, rows of 1 quad).
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

__device__ __forceinline__ WalkShape walk_shape(int L, int xl, bool same_align, int nthreads,
                                                int U) {
    WalkShape w;
    w.Q = (((same_align ? (xl & 3) : 3) + L + 3) >> 2);
    if (w.Q * 2 <= U) {
        w.ru = U / w.Q >= 4 ? 4 : 2;   // Q = 1: U rows; Q = 2, U = 4: two rows
        if (w.ru > U) w.ru = U;
        w.lpr = 1;
        w.ql = U / w.ru;
    } else {
        w.ru = 1;
        const int want = (w.Q + U - 1) / U;
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
    float4 v2;  // the same quad of the second input (walkers with two inputs)
    int e0;
    int64_t a;
    bool has;   // overlaps the row
};

// ---------------------------------------------------------------------------
// Input elements.  Volumes are float32, or unsigned 8- or 16-bit integers whose
// intensities are the integers themselves (converted to fp32 exactly).  A quad
// is four consecutive elements starting on a multiple of 4 (16, 8 or 4 bytes,
// aligned); every helper returns fp32 values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 u16x4(uint2 w) {
    return make_float4(float(w.x & 0xffffu), float(w.x >> 16), float(w.y & 0xffffu), float(w.y >> 16));
}
__device__ __forceinline__ float4 u8x4(uint32_t w) {
    return make_float4(float(w & 0xffu), float((w >> 8) & 0xffu), float((w >> 16) & 0xffu), float(w >> 24));
}
// the quad at p (read-only path; `cs`: streaming, evict first)
__device__ __forceinline__ float4 ldq(const float *p, bool cs) {
    return cs ? __ldcs(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ float4 ldq(const uint16_t *p, bool cs) {
    return u16x4(cs ? __ldcs(reinterpret_cast<const uint2 *>(p)) : __ldg(reinterpret_cast<const uint2 *>(p)));
}
__device__ __forceinline__ float4 ldq(const uint8_t *p, bool cs) {
    return u8x4(cs ? __ldcs(reinterpret_cast<const unsigned int *>(p))
                   : __ldg(reinterpret_cast<const unsigned int *>(p)));
}
__device__ __forceinline__ float ld1(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const uint16_t *p) { return float(__ldg(p)); }
__device__ __forceinline__ float ld1(const uint8_t *p) { return float(__ldg(p)); }
template <typename T>
constexpr uint32_t quad_bytes() { return 4u * uint32_t(sizeof(T)); }

template <typename T>
__device__ __forceinline__ float4 load_quad4(const T *__restrict__ in, int64_t a, int64_t N,
                                             bool has, bool stream) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (has) {
        if (a + 4 <= N) {
            v = ldq(in + a, stream);
        } else {
            v.x = ld1(in + a);
            if (a + 1 < N) v.y = ld1(in + a + 1);
            if (a + 2 < N) v.z = ld1(in + a + 2);
        }
    }
    return v;
}

// Walks the rows of a box.  row_fn(const int *coords, int64_t row_start, S &state)
// prepares per-row state S; quad_fn(S &state, const QuadRef &q) consumes one
// quad.  Template parameter RU must equal shape.ru.  With TWO, the same quads
// of a second array in2 (same layout) are loaded into QuadRef::v2.
template <int D, int U, int RU, typename S, bool TWO, typename T, typename RowFn, typename QuadFn>
__device__ __forceinline__ void walk_rows(const T *__restrict__ in,
                                          const float *__restrict__ in2, int64_t N,
                                          const int64_t *stride, const int *box_lo,
                                          const int *box_len, int r0, int r1,
                                          const WalkShape &w, bool stream, RowFn row_fn,
                                          QuadFn quad_fn) {
    constexpr int QPR = U / RU;   // quads per row and step (RU > 1)
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
        const int qsteps = (RU == 1) ? (w.ql + U - 1) / U : 1;
        for (int qs = 0; qs < qsteps; ++qs) {
            QuadRef q[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int ru = (RU == 1) ? 0 : u / QPR;
                const int qi = (RU == 1) ? (gl + (qs * U + u) * w.lpr) : (u % QPR);
                const int64_t qbase = start[ru] & ~int64_t(3);
                const int head = int(start[ru] - qbase);
                q[u].e0 = 4 * qi - head;
                q[u].a = qbase + 4 * int64_t(qi);
                const bool inl = (RU == 1) ? ((qs * U + u) < w.ql) : true;
                q[u].has = row_ok[ru] && inl && q[u].e0 < L && q[u].e0 + 4 > 0;
                q[u].v = load_quad4(in, q[u].a, N, q[u].has, stream);
                if (TWO) q[u].v2 = load_quad4(in2, q[u].a, N, q[u].has, true);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int ru = (RU == 1) ? 0 : u / QPR;
                quad_fn(st[ru], q[u]);
            }
        }
    }
}

// Dispatch of walk_rows on the shape's RU.
template <int D, int U, typename S, bool TWO = false, typename T, typename RowFn, typename QuadFn>
__device__ __forceinline__ void walk_box(const T *__restrict__ in,
                                         const float *__restrict__ in2, int64_t N,
                                         const int64_t *stride, const int *box_lo,
                                         const int *box_len, int r0, int r1, bool same_align,
                                         bool stream, RowFn row_fn, QuadFn quad_fn) {
    const WalkShape ws = walk_shape(box_len[D - 1], box_lo[D - 1], same_align, blockDim.x, U);
    if (ws.ru == 1)
        walk_rows<D, U, 1, S, TWO, T>(in, in2, N, stride, box_lo, box_len, r0, r1, ws, stream,
                                   row_fn, quad_fn);
    else if (U >= 4 && ws.ru == 4)
        walk_rows<D, U, (U >= 4 ? 4 : 1), S, TWO, T>(in, in2, N, stride, box_lo, box_len, r0, r1, ws,
                                                  stream, row_fn, quad_fn);
    else
        walk_rows<D, U, 2, S, TWO, T>(in, in2, N, stride, box_lo, box_len, r0, r1, ws, stream,
                                   row_fn, quad_fn);
}

// ---------------------------------------------------------------------------
// Tile walker: for a box whose rows all start at the same alignment mod 4
// (the row stride a multiple of 4, or a single row), every thread owns fixed
// quad slots of every row it visits: LPR lanes share a row, lane gl takes the
// quads gl, gl + LPR, ..., gl + (QL - 1) LPR of it.  A slot's position in the
// row, and so its masks and anything the consumer derives from it, is the
// same in every row; slot_fn(i, e0) runs once per slot (e0 = element offset
// of the slot's first element in the row, possibly negative) and returns the
// slot's data SD, row_fn(coords, state) runs once per row, and
// quad_fn(state, slot data, i, v, v2, a) once per loaded quad (a = element
// address of the quad's first element).  Loads are issued
// U at a time; every loop is unrolled, so slot data stay in registers.  With
// PF, rows that fit one load batch are software-pipelined: the next row's
// loads are issued before the current row is consumed.  QL <= QMAX is required: boxes with rows longer
// than 4 * 32 * QMAX - 3 elements must be split along the last dimension.
// ---------------------------------------------------------------------------
// A type carried as a value (to name a local type in a generic lambda).
template <typename T>
struct Tag {
    using type = T;
};

struct TileShape {
    int head;   // first row element's offset in its aligned quad
    int Q;      // quads per row
    int LPR;    // lanes per row (power of two <= 32)
    int QL;     // quads per lane per row
    int G;      // rows in flight per block
};

__device__ __forceinline__ TileShape tile_shape(int L, int head, int nthreads, int qmax) {
    TileShape t;
    t.head = head;
    t.Q = (head + L + 3) >> 2;
    int lpr = 1;
    while (lpr < 32 && lpr * qmax < t.Q) lpr <<= 1;
    t.LPR = lpr;
    t.QL = (t.Q + lpr - 1) / lpr;
    t.G = nthreads / lpr;
    return t;
}

// FULL: every slot of every row is a whole quad inside the box (checked by the
// caller): no per-slot tests.
template <int D, int QMAX, int U, typename S, typename SD, bool TWO, bool PF = false,
          bool FULL = false, typename T, typename SlotFn, typename RowFn, typename QuadFn>
__device__ __forceinline__ void walk_tile(const T *__restrict__ in,
                                          const float *__restrict__ in2, const int64_t *stride,
                                          const int *box_lo, const int *box_len, int r0, int r1,
                                          const TileShape &t, bool stream, SlotFn slot_fn,
                                          RowFn row_fn, QuadFn quad_fn) {
    static_assert(QMAX % U == 0, "QMAX must be a multiple of U");
    const int gl = threadIdx.x & (t.LPR - 1), grp = threadIdx.x / t.LPR;
    const int L = box_len[D - 1];
    bool ok[QMAX];
    SD sd[QMAX];
#pragma unroll
    for (int i = 0; i < QMAX; ++i) {
        const int e0 = 4 * (gl + i * t.LPR) - t.head;
        ok[i] = i < t.QL && e0 < L && e0 + 4 > 0;
        sd[i] = slot_fn(i, e0);
    }
    const int64_t step = 4 * int64_t(t.LPR);
    RowIter<D> it;
    it.init(box_len, r0 + grp, t.G);
    // the next row of this thread: its coordinates and first quad address
    auto next_row = [&](int *coords, int64_t &a0) {
        int64_t start = box_lo[D - 1];
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            coords[j] = box_lo[j] + it.c[j];
            start += int64_t(coords[j]) * stride[j];
        }
        it.next();
        a0 = start - t.head + 4 * gl;
    };
    auto load = [&](int64_t a0, int i0, float4 (&v)[U], float4 (&v2)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (FULL || ok[i0 + u]) {
                v[u] = ldq(in + a0 + (i0 + u) * step, stream);
                if (TWO) v2[u] = __ldcs(reinterpret_cast<const float4 *>(in2 + a0 + (i0 + u) * step));
            }
        }
    };
    if (PF && t.QL <= U) {
        // one load batch per row: the next row's loads are in flight while
        // this row is consumed
        int r = r0 + grp;
        if (r >= r1) return;
        int cc[kMaxDim];
        int64_t ac;
        float4 v[U], v2[U];
        next_row(cc, ac);
        load(ac, 0, v, v2);
        for (;;) {
            const int rn = r + t.G;
            int cn[kMaxDim];
            int64_t an = 0;
            float4 vn[U], vn2[U];
            if (rn < r1) {
                next_row(cn, an);
                load(an, 0, vn, vn2);
            }
            S st;
            row_fn(cc, st);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (FULL || ok[u]) quad_fn(st, sd[u], u, v[u], v2[u], ac + u * step);
            if (rn >= r1) break;
            r = rn;
            ac = an;
#pragma unroll
            for (int j = 0; j < D - 1; ++j) cc[j] = cn[j];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = vn[u];
                if (TWO) v2[u] = vn2[u];
            }
        }
        return;
    }
    for (int r = r0 + grp; r < r1; r += t.G) {
        int coords[kMaxDim];
        int64_t a0;
        next_row(coords, a0);
        S st;
        row_fn(coords, st);
#pragma unroll
        for (int i0 = 0; i0 < QMAX; i0 += U) {
            if (i0 < t.QL) {
                float4 v[U], v2[U];
                load(a0, i0, v, v2);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (FULL || ok[i0 + u]) quad_fn(st, sd[i0 + u], i0 + u, v[u], v2[u], a0 + (i0 + u) * step);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Asynchronous tile walker: the same fixed quad slots as walk_tile, but each
// thread's quads are copied global -> shared with cp.async (16 bytes per
// copy, no registers held while in flight) into a per-thread ring of ST row
// stages, ST - 1 rows ahead of the row being consumed; the consumer reads its
// own stage back with 128-bit shared loads.  Ring layout [stage][slot][thread]
// (consecutive lanes, consecutive 16 bytes: conflict-free).  The ring holds
// ST * QMAX * blockDim float4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// the quad at src copied to shared memory at dst (16, 8 or 4 bytes), and the
// fp32 values of a quad copied there
__device__ __forceinline__ void cpq(uint32_t dst, const float *src) { cp_async16(dst, src); }
__device__ __forceinline__ void cpq(uint32_t dst, const uint16_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cpq(uint32_t dst, const uint8_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
template <typename T>
__device__ __forceinline__ float4 ldsq(uint32_t addr) {
    if constexpr (sizeof(T) == 4) {
        return lds128(addr);
    } else if constexpr (sizeof(T) == 2) {
        uint2 w;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(w.x), "=r"(w.y) : "r"(addr));
        return u16x4(w);
    } else {
        uint32_t w;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w) : "r"(addr));
        return u8x4(w);
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// FULL: the caller has checked that every slot of every row is a whole quad
// inside the box (head 0, L = 4 * LPR * QMAX): no per-slot tests.
// TWO: a second float32 volume in2 of the same layout streams through a second
// ring right behind the first (ring + ST * QMAX * blockDim float4); quad_fn
// gets its quad as the second value.
template <int D, int QMAX, int ST, typename S, typename SD, bool FULL = false, bool TWO = false,
          typename T, typename SlotFn, typename RowFn, typename QuadFn>
__device__ __forceinline__ void walk_tile_async(const T *__restrict__ in, const int64_t *stride,
                                                const int *box_lo, const int *box_len, int r0,
                                                int r1, const TileShape &t, float4 *ring,
                                                SlotFn slot_fn, RowFn row_fn, QuadFn quad_fn,
                                                const float *__restrict__ in2 = nullptr) {
    const int gl = threadIdx.x & (t.LPR - 1), grp = threadIdx.x / t.LPR;
    const int L = box_len[D - 1];
    const int nt = blockDim.x;
    bool ok[QMAX];
    SD sd[QMAX];
#pragma unroll
    for (int i = 0; i < QMAX; ++i) {
        const int e0 = 4 * (gl + i * t.LPR) - t.head;
        ok[i] = i < t.QL && e0 < L && e0 + 4 > 0;
        sd[i] = slot_fn(i, e0);
    }
    const int64_t step = 4 * int64_t(t.LPR);
    const int first = r0 + grp;
    const int nk = first < r1 ? (r1 - first + t.G - 1) / t.G : 0;
    const uint32_t ring_s = uint32_t(__cvta_generic_to_shared(ring));
    auto slot_addr = [&](int stage, int i) {
        return ring_s + 16u * uint32_t((stage * QMAX + i) * nt + int(threadIdx.x));
    };
    RowIter<D> iss, con;   // rows being issued and rows being consumed
    iss.init(box_len, first, t.G);
    con.init(box_len, first, t.G);
    auto row_addr = [&](RowIter<D> &it, int *coords) {
        int64_t start = box_lo[D - 1];
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            coords[j] = box_lo[j] + it.c[j];
            start += int64_t(coords[j]) * stride[j];
        }
        it.next();
        return start - t.head + 4 * gl;
    };
    const uint32_t ring2_off = 16u * uint32_t(ST * QMAX * nt);
    auto issue = [&](int stage) {
        int coords[kMaxDim];
        const int64_t a0 = row_addr(iss, coords);
#pragma unroll
        for (int i = 0; i < QMAX; ++i)
            if (FULL || ok[i]) {
                cpq(slot_addr(stage, i), in + a0 + i * step);
                if (TWO) cp_async16(slot_addr(stage, i) + ring2_off, in2 + a0 + i * step);
            }
    };
#pragma unroll
    for (int k = 0; k < ST - 1; ++k) {
        if (k < nk) issue(k);
        cp_async_commit();
    }
    int stage_c = 0, stage_i = ST - 1;
    for (int k = 0; k < nk; ++k) {
        if (k + ST - 1 < nk) issue(stage_i);
        cp_async_commit();
        cp_async_wait<ST - 1>();   // row k has landed
        int coords[kMaxDim];
        const int64_t a0 = row_addr(con, coords);
        S st;
        row_fn(coords, st);
#pragma unroll
        for (int i = 0; i < QMAX; ++i)
            if (FULL || ok[i]) {
                const float4 v = ldsq<T>(slot_addr(stage_c, i));
                const float4 v2 = TWO ? lds128(slot_addr(stage_c, i) + ring2_off) : v;
                quad_fn(st, sd[i], i, v, v2, a0 + i * step);
            }
        stage_c = (stage_c + 1 == ST) ? 0 : stage_c + 1;
        stage_i = (stage_i + 1 == ST) ? 0 : stage_i + 1;
    }
    cp_async_wait<0>();
}

// shared-memory access by 32-bit shared-window address
__device__ __forceinline__ void red_shared_add(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ float2 lds_f32x2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}
__device__ __forceinline__ float4 lds_f32x4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

// ---------------------------------------------------------------------------
// Host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------
// k_range.cu: the per-kernel ranges of an adaptive plan in one sweep
bool range_pass_fits(const Geom &g);
cudaError_t launch_range_kernels(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                                 cudaStream_t st);
// whether a plan's histogram pass takes its adaptive ranges from that sweep
// (the cluster form with a ring, TMA or per-thread walk)
inline bool uses_range_pass(const mclahe_plan_s &p) {
    return p.t.range_pass && p.g.mode == MCLAHE_RANGE_ADAPTIVE && p.t.hist_shares == 0 &&
           p.t.hist_walk != 3 && range_pass_fits(p.g);
}
cudaError_t launch_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                         cudaStream_t st);
cudaError_t launch_hist(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                        const float *d_clip, cudaStream_t st);
cudaError_t launch_map(const mclahe_plan_s &p, const float *in, float *out,
                       const unsigned char *ws, cudaStream_t st);
cudaError_t launch_backward(const mclahe_plan_s &p, const float *in, const float *gout,
                            unsigned char *ws, const float *d_clip, float *d_grad_lut,
                            float *d_grad_clip, cudaStream_t st);
// backward scratch: int64 table-gradient sums [cells][2^D][LS], the max |g|
// key (and padding), dL/dT[K]
size_t bwd_sum_words(const Geom &g);
size_t bwd_scratch_bytes(const Geom &g, int chunks);
// k_bwd_gather.cu: the clip-limit gradient alone (d lut/dT tables interpolated
// like the mapping pass and dotted with the upstream gradient) and its scratch
size_t bwd_gather_bytes(const Geom &g, int chunks);
cudaError_t launch_backward_gather(const mclahe_plan_s &p, const float *in, const float *gout,
                                   unsigned char *ws, const float *d_clip, float *d_grad_clip,
                                   cudaStream_t st);
// Dynamic shared memory of a histogram CTA for a row walk (0: per-thread
// loads, the batched launch; 1: the cp.async row ring; 2: TMA tiles), and of
// the flat form's range pass.
size_t hist_smem_bytes(const Geom &g, int copies, int group, int walk = 1, int threads = 256);
size_t hist_range_smem_bytes(int group, int walk, int threads);
// the row-walk code of hist_smem_bytes for a plan's hist_walk (0 ring, 1 TMA tiles,
// 2 per-thread loads)
inline int hist_walk_code(int hist_walk) { return hist_walk == 0 ? 1 : hist_walk == 1 ? 2 : 0; }
bool hist_tma_box(const Geom &g, int group, int &bx, int &by);
// the staged walk (hist_walk = 3): fits for R copies and clusters of C CTAs
// (2- to 4-D, last extent a multiple of 4), with its shared-memory bytes
bool hist_staged_fits(const Geom &g, int R, int C, size_t *bytes);
// Tensor map of a float32 volume (dims innermost first) with box[0..D-1]
// elements per tile (tma_host.cu).
cudaError_t encode_tensor_map(CUtensorMap *m, const float *ptr, const Geom &g, const int *box);
cudaError_t launch_hist_range(const mclahe_plan_s &p, const float *in, unsigned char *ws,
                              cudaStream_t st);
int64_t hist_items(const Geom &g, int group);
size_t map_smem_bytes(const Geom &g);
bool map_tma_box(const Geom &g, int &bx, int &by, int &bz);
bool map_replicated(const Geom &g);

// launch_cache.cu: raise a kernel's dynamic shared-memory limit (once per
// device, kernel and size) and cached occupancy (CTAs per SM)
cudaError_t ensure_smem(const void *func, size_t bytes);
cudaError_t cached_occupancy(const void *func, int threads, size_t smem, int *per_sm);

// batch.cu
void batch_forget_plan(const mclahe_plan_s *p);

// plan.cu
int device_sms();
int64_t n_cells(const Geom &g);
Tuning default_tuning(const Geom &g);
Layout make_layout(const Geom &g, const Tuning &t);
mclahe_status check_forward_args(const mclahe_plan_s *p, const void *in, const void *out,
                                 const void *ws, size_t ws_bytes);
mclahe_status forward_impl(const mclahe_plan_s &p, const float *in, float *out, unsigned char *ws,
                           const float *d_clip, cudaStream_t st);

}  // namespace mclahe
