// batch_impl.cuh -- device side of mclahe_batch: the persistent kernel that
// runs range, kernel and cell tiles of many volumes (see batch.cu for the
// work list and the launch), shared by the per-dimensionality translation
// units batch_k2.cu, batch_k3.cu and batch_k4.cu.
#pragma once

#include "hist_impl.cuh"
#include "map_impl.cuh"

namespace mclahe {

constexpr int kGroupVol = 64;                 // volumes per persistent launch
constexpr int kMaxStage = 3 * kGroupVol;
constexpr uint32_t kWaitSpins = 1u << 22;     // default polls: ~ seconds with the back-off below

struct BVol {
    Geom g;
    const float *in;
    float *out;
    uint32_t *hist;
    float *lut, *lo, *scale;
    uint32_t *keys;          // global range keys (min complemented, max)
    const float *clip;       // nullable
    int32_t R;               // histogram lane copies
    int32_t G;               // kernels per histogram item along the last dimension
    int64_t n_hist;          // histogram items
    int32_t mgroups;         // cell tiles per cell (each split over the cluster)
    int64_t n_range;         // range tiles (0: no range pass)
    int64_t range_len;       // voxels per range tile
};

struct BParams {
    int n_vol, n_stage;
    unsigned long long *next;   // work counter
    uint32_t *done;             // per volume: range tiles done, kernel tiles done
    uint32_t *status;           // batch status word
    uint32_t wait_polls;        // polls before a wait gives up
    uint32_t target_bias;       // added to every wait target (0; non-zero only to test the
                                // timeout path: no counter reaches the raised target)
    int64_t stage_start[kMaxStage + 1];
    int32_t stage_kind[kMaxStage];   // 0 range, 1 kernel, 2 cell
    int32_t stage_vol[kMaxStage];
    BVol v[kGroupVol];
};

static_assert(sizeof(BParams) <= 32000, "batch parameters must fit the kernel parameter space");

// Thread 0 waits (bounded: at most `polls` polls) until *ctr >= target; then
// the block proceeds.  A wait that gives up records MCLAHE_ERR_TIMEOUT, and
// every later wait of the launch returns at once.
__device__ __forceinline__ void wait_ready(const uint32_t *ctr, uint32_t target, uint32_t *status,
                                           uint32_t polls) {
    if (threadIdx.x == 0) {
        uint32_t spins = 0, ns = 32;
        for (;;) {
            if (*reinterpret_cast<volatile uint32_t *>(status) != 0) break;   // an earlier give-up
            uint32_t v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (++spins > polls) {
                atomicCAS(status, 0u, uint32_t(MCLAHE_ERR_TIMEOUT));
                break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
        }
    }
    __syncthreads();
}

// Publish one finished tile: every thread's global writes are done first.
__device__ __forceinline__ void signal_done(uint32_t *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

__device__ __forceinline__ void range_tile(const BVol &V, int64_t idx, int rank, int C) {
    __shared__ float s_mn[32], s_mx[32];
    const int64_t a0 = idx * V.range_len, a1 = min(V.g.N, a0 + V.range_len);
    const int64_t len = a1 - a0;
    const int64_t b0 = a0 + (len * rank) / C, b1 = a0 + (len * (rank + 1)) / C;
    float mn = INFINITY, mx = -INFINITY;
    // aligned middle in 128-bit loads, ends element by element
    const int64_t q0 = (b0 + 3) & ~int64_t(3), q1 = max(q0, b1 & ~int64_t(3));
    for (int64_t i = q0 + 4 * int64_t(threadIdx.x); i < q1; i += 4 * int64_t(blockDim.x)) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(V.in + i));
        mn = min3f(mn, v.x, v.y);
        mn = min3f(mn, v.z, v.w);
        mx = max3f(mx, v.x, v.y);
        mx = max3f(mx, v.z, v.w);
    }
    for (int64_t i = b0 + threadIdx.x; i < min(q0, b1); i += blockDim.x) {
        mn = fminf(mn, V.in[i]);
        mx = fmaxf(mx, V.in[i]);
    }
    for (int64_t i = max(q1, b0) + threadIdx.x; i < b1; i += blockDim.x) {
        mn = fminf(mn, V.in[i]);
        mx = fmaxf(mx, V.in[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_mn[warp] = mn;
        s_mx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < int(blockDim.x >> 5); ++w) {
            mn = fminf(mn, s_mn[w]);
            mx = fmaxf(mx, s_mx[w]);
        }
        if (b1 > b0) {
            atomicMax(&V.keys[0], ~float_key(mn));
            atomicMax(&V.keys[1], float_key(mx));
        }
    }
}

template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(256, D <= 2 ? 3 : ((D >= 4 && ADAPTIVE) ? 1 : 2)) k_batch(const __grid_constant__ BParams bp) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ unsigned long long s_item;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int64_t total = bp.stage_start[bp.n_stage];
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(bp.next, 1ull);
        cluster.sync();
        const int64_t item = int64_t(*cluster.map_shared_rank(&s_item, 0));
        cluster.sync();   // every CTA has read the tile before rank 0 takes the next
        if (item >= total) break;
        int lo = 0, hi = bp.n_stage - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.stage_start[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int vi = bp.stage_vol[lo];
        const BVol &V = bp.v[vi];
        const int64_t idx = item - bp.stage_start[lo];
        switch (bp.stage_kind[lo]) {
            case 0:
                range_tile(V, idx, rank, C);
                signal_done(&bp.done[2 * vi]);
                break;
            case 1:
                if (V.n_range > 0) wait_ready(&bp.done[2 * vi], uint32_t(V.n_range * C) + bp.target_bias, bp.status,
                                           bp.wait_polls);
                hist_group<D, ADAPTIVE>(V.g, V.in, V.keys, V.clip, V.hist, V.lut, V.lo, V.scale, idx,
                                        V.G, V.R, smem);
                if (rank == 0) signal_done(&bp.done[2 * vi + 1]);
                break;
            default: {
                wait_ready(&bp.done[2 * vi + 1], uint32_t(V.n_hist) + bp.target_bias, bp.status,
                           bp.wait_polls);
                const int64_t cell = idx / V.mgroups;
                const int grp = int(idx - cell * V.mgroups);
                map_cell<D, ADAPTIVE, true, false>(V.g, V.in, V.out, V.lut, V.lo, V.scale, cell,
                                            grp * C + rank, V.mgroups * C,
                                            reinterpret_cast<float *>(smem));
                break;
            }
        }
    }
}

template <int D, bool A>
cudaError_t launch_batch_t(const BParams &bp, int C, size_t smem, cudaStream_t st) {
    auto kern = k_batch<D, A>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), size_t(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C);
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    const int64_t items = bp.stage_start[bp.n_stage];
    const int64_t grid_clusters = nclusters < items ? nclusters : (items > 0 ? items : 1);
    cfg.gridDim = dim3(unsigned(grid_clusters * C));
    return cudaLaunchKernelEx(&cfg, kern, bp);
}

cudaError_t launch_batch_d2(const BParams &bp, bool adaptive, int C, size_t smem, cudaStream_t st);
cudaError_t launch_batch_d3(const BParams &bp, bool adaptive, int C, size_t smem, cudaStream_t st);
cudaError_t launch_batch_d4(const BParams &bp, bool adaptive, int C, size_t smem, cudaStream_t st);

// launches one group's persistent kernel (batch_k<D>.cu)
cudaError_t launch_batch_group(const BParams &bp, int D, bool adaptive, int C, size_t smem,
                               cudaStream_t st);

}  // namespace mclahe
