// k_map_impl.cuh -- kernels and launcher templates of the mapping pass of one
// volume: one CTA per chunk of an inter-kernel cell (Sec. III.C, Eq.
// (12)-(13); the work of a CTA is in map_impl.cuh), for float32 volumes
// (k_map.cu) and unsigned integer volumes (k_map_u16.cu, k_map_u8.cu).
#pragma once

#include <algorithm>
#include <type_traits>
#include <cuda.h>

#include "map_impl.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE, bool REPL, typename T = float>
__global__ void __launch_bounds__(256, D >= 4 ? (ADAPTIVE ? 1 : 2) : (ADAPTIVE && D == 3 ? 2 : 3)) k_map(Geom g, const T *__restrict__ in,
                                             float *__restrict__ out,
                                             const float *__restrict__ lut,
                                             const float *__restrict__ lo_k,
                                             const float *__restrict__ scale_k, int chunks, int64_t cell0) {
    extern __shared__ __align__(16) float tab[];
    const int64_t b = blockIdx.x / chunks;
    const int chunk = int(blockIdx.x - b * chunks);
    map_cell<D, ADAPTIVE, REPL, kWalkRing, false, T>(g, in, out, lut, lo_k, scale_k, cell0 + b, chunk, chunks,
                                                     tab);
}

// TMA tiles (kWalkTma): the whole cell row along the last dim, as many rows
// along dims D-2 and (4-D) 1 as fit in kTmaTileFloats, dividing the kernel
// size so interior cells split into whole tiles.
template <int D, bool ADAPTIVE>
__global__ void __launch_bounds__(kTmaConsumers + 32, D >= 4 ? (ADAPTIVE ? 1 : 2) : 2)
    k_map_tma(Geom g, const __grid_constant__ CUtensorMap tm_in,
              const __grid_constant__ CUtensorMap tm_out, const float *__restrict__ in,
              float *__restrict__ out, const float *__restrict__ lut,
              const float *__restrict__ lo_k, const float *__restrict__ scale_k, int chunks, int bx,
              int by, int bz, uint32_t *status) {
    extern __shared__ __align__(128) float tab[];
    const MapTma t{&tm_in, &tm_out, bx, by, bz, status};
    const int64_t cell = blockIdx.x / chunks;
    const int chunk = int(blockIdx.x - cell * chunks);
    map_cell<D, ADAPTIVE, true, kWalkTma>(g, in, out, lut, lo_k, scale_k, cell, chunk, chunks, tab, &t);
}

// Flat form: every cell is cut into `shares` equal row shares, and the shares
// of all cells are dealt out in order to a persistent grid (one wave), so the
// CTAs' work is equal whatever the number of cells; a CTA restages the corner
// tables when its range moves to the next cell.
template <int D, bool ADAPTIVE, bool REPL>
__global__ void __launch_bounds__(256, D >= 4 ? (ADAPTIVE ? 1 : 2) : (ADAPTIVE && D == 3 ? 2 : 3))
    k_map_flat(Geom g, const float *__restrict__ in, float *__restrict__ out,
               const float *__restrict__ lut, const float *__restrict__ lo_k,
               const float *__restrict__ scale_k, int shares, int64_t total) {
    extern __shared__ __align__(16) float tab[];
    const int64_t b0 = total * blockIdx.x / gridDim.x;
    const int64_t b1 = total * (blockIdx.x + 1) / gridDim.x;
    for (int64_t s = b0; s < b1;) {
        const int64_t cell = s / shares;
        const int c0 = int(s - cell * shares);
        const int64_t rest = b1 - cell * shares;
        const int c1 = rest < shares ? int(rest) : shares;
        map_cell<D, ADAPTIVE, REPL>(g, in, out, lut, lo_k, scale_k, cell, c0, shares, tab, nullptr, c1);
        s = cell * shares + c1;
        __syncthreads();   // the tables are restaged for the next cell
    }
}

static inline size_t map_tma_smem(const Geom &g) {
    return map_table_bytes(g.D, g.P) + 128 + size_t(kTmaStages) * kTmaTileFloats * sizeof(float);
}

template <int D, bool A>
static cudaError_t launch_map_tma_t(const mclahe_plan_s &p, const float *in, float *out,
                                    const unsigned char *ws, cudaStream_t st, unsigned grid, int bx,
                                    int by, int bz) {
    const size_t smem = map_tma_smem(p.g);
    CUtensorMap m_in, m_out;
    const int box[4] = {bx, by, p.g.D == 4 ? bz : 1, 1};
    cudaError_t e = encode_tensor_map(&m_in, in, p.g, box);
    if (e == cudaSuccess) e = encode_tensor_map(&m_out, out, p.g, box);
    if (e == cudaSuccess)
        e = ensure_smem(reinterpret_cast<const void *>(k_map_tma<D, A>), smem);
    if (e != cudaSuccess) return e;
    k_map_tma<D, A><<<grid, kTmaConsumers + 32, smem, st>>>(
        p.g, m_in, m_out, in, out, reinterpret_cast<const float *>(ws + p.ws.lut),
        reinterpret_cast<const float *>(ws + p.ws.lo), reinterpret_cast<const float *>(ws + p.ws.scale),
        p.t.map_chunks, bx, by, bz, reinterpret_cast<uint32_t *>(const_cast<unsigned char *>(ws) + p.ws.status));
    return cudaGetLastError();
}

template <int D, bool A, bool REPL>
static cudaError_t launch_map_flat_t(const mclahe_plan_s &p, const float *in, float *out,
                                     const unsigned char *ws, cudaStream_t st, size_t smem) {
    auto kern = k_map_flat<D, A, REPL>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cached_occupancy(reinterpret_cast<const void *>(kern), p.t.map_threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t total = n_cells(p.g) * p.t.map_chunks;
    const unsigned grid = unsigned(std::min<int64_t>(total, int64_t(per_sm) * device_sms()));
    kern<<<grid, p.t.map_threads, smem, st>>>(
        p.g, in, out, reinterpret_cast<const float *>(ws + p.ws.lut),
        reinterpret_cast<const float *>(ws + p.ws.lo), reinterpret_cast<const float *>(ws + p.ws.scale),
        p.t.map_chunks, total);
    return cudaGetLastError();
}

template <int D, bool A, bool REPL, typename T>
static cudaError_t launch_map_t(const mclahe_plan_s &p, const T *in, float *out,
                                const unsigned char *ws, cudaStream_t st, unsigned grid,
                                size_t smem, int64_t cell0, bool full) {
    if constexpr (std::is_same<T, float>::value) {
        if (p.t.map_flat && full) return launch_map_flat_t<D, A, REPL>(p, in, out, ws, st, smem);
    }
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_map<D, A, REPL, T>), smem);
    if (e != cudaSuccess) return e;
    k_map<D, A, REPL, T><<<grid, p.t.map_threads, smem, st>>>(
        p.g, in, out, reinterpret_cast<const float *>(ws + p.ws.lut),
        reinterpret_cast<const float *>(ws + p.ws.lo), reinterpret_cast<const float *>(ws + p.ws.scale),
        p.t.map_chunks, cell0);
    return cudaGetLastError();
}

// cells [cell0, cell0 + ncells) (all by default; a part of the cells always
// takes the per-cell grid with per-thread walks)
template <int D, typename T>
static cudaError_t launch_map_d(const mclahe_plan_s &p, const T *in, float *out,
                                const unsigned char *ws, cudaStream_t st, int64_t cell0 = 0,
                                int64_t ncells = -1) {
    const Geom &g = p.g;
    const bool full = cell0 == 0 && (ncells < 0 || ncells == n_cells(g));
    const unsigned grid = unsigned((full ? n_cells(g) : ncells) * p.t.map_chunks);
    int bx, by, bz;
    if constexpr (D >= 3 && std::is_same<T, float>::value) {
        if (full && p.t.map_tma && map_tma_box(g, bx, by, bz))
            return g.mode == MCLAHE_RANGE_ADAPTIVE
                       ? launch_map_tma_t<D, true>(p, in, out, ws, st, grid, bx, by, bz)
                       : launch_map_tma_t<D, false>(p, in, out, ws, st, grid, bx, by, bz);
    }
    const size_t smem = map_smem_bytes(g);
    const bool repl = map_replicated(g);
    if (g.mode == MCLAHE_RANGE_ADAPTIVE)
        return repl ? launch_map_t<D, true, true, T>(p, in, out, ws, st, grid, smem, cell0, full)
                    : launch_map_t<D, true, false, T>(p, in, out, ws, st, grid, smem, cell0, full);
    return repl ? launch_map_t<D, false, true, T>(p, in, out, ws, st, grid, smem, cell0, full)
                : launch_map_t<D, false, false, T>(p, in, out, ws, st, grid, smem, cell0, full);
}

template <typename T>
static cudaError_t launch_map_any(const mclahe_plan_s &p, const T *in, float *out,
                                  const unsigned char *ws, cudaStream_t st, int64_t cell0 = 0,
                                  int64_t ncells = -1) {
    switch (p.g.D) {
        case 1: return launch_map_d<1>(p, in, out, ws, st, cell0, ncells);
        case 2: return launch_map_d<2>(p, in, out, ws, st, cell0, ncells);
        case 3: return launch_map_d<3>(p, in, out, ws, st, cell0, ncells);
        case 4: return launch_map_d<4>(p, in, out, ws, st, cell0, ncells);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mclahe
