// hist_staged.cuh -- the histogram pass with the kernel's footprint staged in
// shared memory (Algorithm 1: histogram, clip, redistribute, CDF,
// normalisation; Sec. III.D: the adaptive range), one thread-block cluster
// per kernel.
//
// With an adaptive range every kernel's voxels are needed twice: once for the
// kernel's minimum and maximum and once, under that range, for the histogram.
// Streaming them from global memory twice costs a second sweep (from L2 at
// best).  Here cluster rank r copies its share of the footprint box (rows
// [R r / C, R (r + 1) / C) of the box, every row whole) into its own shared
// memory with cp.async -- all copies in flight at once -- so the volume is
// read from DRAM once: the minimum and maximum are reduced from shared memory,
// exchanged across the cluster through distributed shared memory, and the
// histogram is binned from shared memory.  The footprint of kernel k along a
// dimension is the interval of original indices whose mirror images
// (Sec. III.B) fall in the padded kernel, each with its multiplicity (the
// number of its images inside the kernel); a voxel adds the product of its
// multiplicities over the dimensions, which gives exactly the histogram of the
// padded kernel.  The copies, clip and table phases are those of the cluster
// form (sum_copies, merge_and_build).
#pragma once

#include "hist_impl.cuh"

namespace mclahe {

// Shared memory of a staged CTA: the histogram words of one kernel, then the
// staged quads of its rows.
constexpr int kStagedQmax = 4;      // quad slots per thread and row (rows of at most
                                    // 4 * 32 * kStagedQmax - 3 elements)
constexpr int kStagedBatches = 4;   // cp.async groups per thread (rows in order)
struct StagedShape {
    int rows_max;   // footprint rows of the largest kernel (all dims but the last)
    int Q;          // quads per staged row (the widest footprint row, from its 16-byte boundary)
};

__host__ __device__ inline size_t staged_data_offset_words(int P, int R) {
    return (hist_smem_words(P, R, 1) + 3) & ~size_t(3);
}
// ... then one weight word per staged row and one multiplicity word per quad
// position of a row
__host__ __device__ inline size_t staged_smem_bytes(int P, int R, int C, const StagedShape &sh) {
    const size_t rows = (size_t(sh.rows_max) + C - 1) / C;
    return staged_data_offset_words(P, R) * 4 + rows * size_t(sh.Q) * 16 + rows * 4 + size_t(sh.Q) * 4;
}

template <int D, bool ADAPTIVE, typename T = float>
__device__ __forceinline__ void hist_staged(const Geom &g, const T *__restrict__ in,
                                            const uint32_t *__restrict__ keys,
                                            const float *__restrict__ d_clip,
                                            uint32_t *__restrict__ hist, float *__restrict__ lut,
                                            float *__restrict__ lo_out, float *__restrict__ scale_out,
                                            int64_t kidx, int R, uint32_t *sh) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int nb = g.nb, P = g.P;
    const int lane = threadIdx.x & 31;
    const int nt = blockDim.x;

    // the kernel's coordinates and footprint box
    __shared__ Foot s_f[kMaxDim];
    if (threadIdx.x < D) {
        int64_t r = kidx;
        int k = 0;
        for (int j = D - 1; j >= int(threadIdx.x); --j) {
            k = int(r % g.d[j].n);
            r /= g.d[j].n;
        }
        s_f[threadIdx.x] = footprint(g.d[threadIdx.x], k);
    }
    // smem: copies [P][R], counts [P], keys [2], -lo, scale, lo; data; row weights
    uint32_t *cnt = sh + size_t(P) * R;
    uint32_t *s_keys = cnt + P;
    float *s_nlo = reinterpret_cast<float *>(s_keys + 2);
    float *s_sc = s_nlo + 1;
    float *s_lo = s_sc + 1;
    float4 *data = reinterpret_cast<float4 *>(sh + staged_data_offset_words(P, R));
    {
        uint4 *z = reinterpret_cast<uint4 *>(sh);
        const int nw = int(hist_smem_words(P, R, 1));
        for (int i = threadIdx.x; i < nw / 4; i += nt) z[i] = make_uint4(0, 0, 0, 0);
        for (int i = (nw / 4) * 4 + threadIdx.x; i < nw; i += nt) sh[i] = 0;
    }
    __syncthreads();
    int blo[kMaxDim], blen[kMaxDim];
    int64_t stride[kMaxDim];
    int rows = 1;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        blo[j] = s_f[j].lo;
        blen[j] = s_f[j].hi - s_f[j].lo;
        stride[j] = g.d[j].stride;
        if (j < D - 1) rows *= blen[j];
    }
    const int r0 = int((int64_t(rows) * rank) / C), r1 = int((int64_t(rows) * (rank + 1)) / C);
    const int nr = r1 - r0;
    const int Lb = blen[D - 1], xa = blo[D - 1] & ~3, head = blo[D - 1] - xa;
    // Thread t takes the flat quads t, t + nt, ... of the CTA's rows (row rr =
    // q / Q, quad qi = q mod Q: consecutive threads copy consecutive 16-byte
    // quads) and later reads back only the quads it copied itself, so waiting
    // for its own cp.async groups replaces a block barrier.  Row, quad and the
    // row's coordinates advance incrementally (no division in the loops).
    const int Q = (head + Lb + 3) >> 2;
    const int nq = nr * Q;
    const int myq = nq > int(threadIdx.x) ? (nq - 1 - int(threadIdx.x)) / nt + 1 : 0;
    int dq;
    const int drr = small_div(nt, Q, dq);
    const uint32_t d0 = uint32_t(__cvta_generic_to_shared(data));
    const Foot fl = s_f[D - 1];
    uint32_t *roww = reinterpret_cast<uint32_t *>(data + size_t(nq));   // [nr] outer weights
    uint32_t *qmult = roww + nr;   // [Q] per quad position: the common last-dim
                                   // multiplicity of its four voxels, 0 if they
                                   // differ or leave the footprint
    // position of this thread's k-th quad: (rr, qi) and the row's box
    // coordinates; step() moves to the (k+1)-th
    struct Pos {
        int rr, qi;
        int c[kMaxDim];
    };
    auto start = [&](Pos &ps) {
        ps.rr = small_div(int(threadIdx.x), Q, ps.qi);
        int rest = r0 + ps.rr;
#pragma unroll
        for (int j = D - 2; j >= 0; --j) rest = small_div(rest, blen[j], ps.c[j]);
    };
    auto advance_rows = [&](Pos &ps, int k) {   // k >= 0 rows forward
        ps.rr += k;
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            ps.c[j] += k;
            k = 0;
            while (ps.c[j] >= blen[j]) {
                ps.c[j] -= blen[j];
                ++k;
            }
        }
    };
    auto step = [&](Pos &ps) {
        ps.qi += dq;
        int k = drr;
        if (ps.qi >= Q) {
            ps.qi -= Q;
            ++k;
        }
        advance_rows(ps, k);
    };
    // batch b of this thread's quads: [myq b / NB, myq (b + 1) / NB), one cp.async group each
    constexpr int NB = kStagedBatches;

    // ---- stage
    {
        Pos ps;
        start(ps);
        int k = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int kend = (myq * (b + 1)) / NB;
            for (; k < kend; ++k) {
                int64_t a = xa + 4 * ps.qi;
#pragma unroll
                for (int j = 0; j < D - 1; ++j) a += int64_t(blo[j] + ps.c[j]) * stride[j];
                cpq(d0 + 16u * uint32_t(int(threadIdx.x) + k * nt), in + a);
                step(ps);
            }
            cp_async_commit();
        }
        // row weights and quad multiplicities (read after the next block barrier)
        for (int i = threadIdx.x; i < nr; i += nt) {
            int rest = r0 + i, c;
            uint32_t w = 1;
#pragma unroll
            for (int j = D - 2; j >= 0; --j) {
                rest = small_div(rest, blen[j], c);
                w *= uint32_t(s_f[j].mult(blo[j] + c));
            }
            roww[i] = w;
        }
        for (int q = threadIdx.x; q < Q; q += nt) {
            int m[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int e0 = 4 * q - head + e;
                m[e] = (e0 >= 0 && e0 < Lb) ? fl.mult(blo[D - 1] + e0) : 0;
            }
            qmult[q] = (m[0] == m[1] && m[1] == m[2] && m[2] == m[3]) ? uint32_t(m[0]) : 0u;
        }
    }

    // wait for this thread's copy groups up to batch b (all of them for b < 0)
    auto wait_batch = [&](int b) {
        switch (NB - 1 - b) {
            case 3: cp_async_wait<3>(); break;
            case 2: cp_async_wait<2>(); break;
            case 1: cp_async_wait<1>(); break;
            default: cp_async_wait<0>(); break;
        }
    };

    // ---- adaptive range: min/max of the staged voxels, batch by batch as
    // they land, then across the cluster
    if (ADAPTIVE) {
        float mn = INFINITY, mx = -INFINITY;
        int k = 0, qi;
        small_div(int(threadIdx.x), Q, qi);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            wait_batch(b);
            const int kend = (myq * (b + 1)) / NB;
            for (; k < kend; ++k) {
                const float4 v = ldsq<T>(d0 + 16u * uint32_t(int(threadIdx.x) + k * nt));
                const int e0 = 4 * qi - head;
                if (e0 >= 0 && e0 + 4 <= Lb) {
                    mn = min3f(mn, v.x, v.y);
                    mn = min3f(mn, v.z, v.w);
                    mx = max3f(mx, v.x, v.y);
                    mx = max3f(mx, v.z, v.w);
                } else {
                    const float vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (e0 + e >= 0 && e0 + e < Lb) {
                            mn = fminf(mn, vals[e]);
                            mx = fmaxf(mx, vals[e]);
                        }
                }
                qi += dq;
                if (qi >= Q) qi -= Q;
            }
        }
        const bool has = mn <= mx;
        const uint32_t kmn = __reduce_max_sync(0xffffffffu, has ? ~float_key(mn) : 0u);
        const uint32_t kmx = __reduce_max_sync(0xffffffffu, has ? float_key(mx) : 0u);
        if (lane == 0 && (kmn | kmx)) {
            atomicMax(&s_keys[0], kmn);
            atomicMax(&s_keys[1], kmx);
        }
        if (C > 1) cluster.sync(); else __syncthreads();   // every CTA's keys are complete
        if (threadIdx.x == 0) {
            uint32_t ka = 0, kb = 0;
            for (int c = 0; c < C; ++c) {
                const uint32_t *rk = C > 1 ? cluster.map_shared_rank(s_keys, c) : s_keys;
                ka = max(ka, rk[0]);
                kb = max(kb, rk[1]);
            }
            float lo, hi;
            keys_to_range(ka, kb, lo, hi);
            s_lo[0] = lo;
            s_nlo[0] = -lo;
            s_sc[0] = range_scale(lo, hi, nb);
        }
    } else if (threadIdx.x == 0) {
        float lo, hi;
        if (g.has_range) {
            lo = g.range_lo;
            hi = g.range_hi;
        } else {
            keys_to_range(__ldcg(keys), __ldcg(keys + 1), lo, hi);
        }
        s_lo[0] = lo;
        s_nlo[0] = -lo;
        s_sc[0] = range_scale(lo, hi, nb);
    }
    __syncthreads();

    // ---- histogram of the staged voxels (R lane copies), batch by batch
    {
        const uint32_t r4 = uint32_t(4 * R);
        const uint32_t base = uint32_t(__cvta_generic_to_shared(sh)) + 4u * uint32_t(lane & (R - 1)) -
                              kBinBias * r4;
        const float2 n2 = make_float2(s_nlo[0], s_nlo[0]), s2 = make_float2(s_sc[0], s_sc[0]);
        const float iqk = g.iqk, qkf = g.qkf;
        int k = 0, qi, rr = small_div(int(threadIdx.x), Q, qi);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (!ADAPTIVE) wait_batch(b);
            const int kend = (myq * (b + 1)) / NB;
            for (; k < kend; ++k) {
                const float4 v = ldsq<T>(d0 + 16u * uint32_t(int(threadIdx.x) + k * nt));
                const uint32_t w = roww[rr], mq = qmult[qi];
                const uint2 b01 = qbits2(make_float2(v.x, v.y), n2, s2, iqk, qkf);
                const uint2 b23 = qbits2(make_float2(v.z, v.w), n2, s2, iqk, qkf);
                const uint32_t bits[4] = {b01.x, b01.y, b23.x, b23.y};
                if (mq != 0) {
                    const uint32_t wq = w * mq;
#pragma unroll
                    for (int e = 0; e < 4; ++e) red_shared_add(bits[e] * r4 + base, wq);
                } else {
                    const int e0 = 4 * qi - head;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int m = (e0 + e >= 0 && e0 + e < Lb) ? fl.mult(blo[D - 1] + e0 + e) : 0;
                        if (m > 0) red_shared_add(bits[e] * r4 + base, w * uint32_t(m));
                    }
                }
                rr += drr;
                qi += dq;
                if (qi >= Q) {
                    qi -= Q;
                    ++rr;
                }
            }
        }
    }
    __syncthreads();
    sum_copies(sh, cnt, 1, P, R, nb);
    if (C > 1) cluster.sync(); else __syncthreads();   // every CTA's counts are complete
    merge_and_build(g, sh, cnt, s_lo, s_sc, 1, C, rank, hist, lut, lo_out, scale_out, kidx, d_clip);
}

}  // namespace mclahe
