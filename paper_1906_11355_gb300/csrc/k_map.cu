// k_map.cu -- launcher of the mapping pass of one volume: one CTA per chunk of
// an inter-kernel cell (Sec. III.C, Eq. (12)-(13); the work of a CTA is in
// map_impl.cuh).
#include "map_impl.cuh"

namespace mclahe {

template <int D, bool ADAPTIVE, bool REPL>
__global__ void __launch_bounds__(256, D >= 4 ? (ADAPTIVE ? 1 : 2) : (ADAPTIVE && D == 3 ? 2 : 3)) k_map(Geom g, const float *__restrict__ in,
                                             float *__restrict__ out,
                                             const float *__restrict__ lut,
                                             const float *__restrict__ lo_k,
                                             const float *__restrict__ scale_k, int chunks) {
    extern __shared__ __align__(16) float tab[];
    const int64_t cell = blockIdx.x / chunks;
    const int chunk = int(blockIdx.x - cell * chunks);
    map_cell<D, ADAPTIVE, REPL>(g, in, out, lut, lo_k, scale_k, cell, chunk, chunks, tab);
}

bool map_replicated(const Geom &g) { return map_repl_fits(g.P); }
size_t map_smem_bytes(const Geom &g) { return map_smem_for(g.D, g.P); }

template <int D, bool A, bool REPL>
static cudaError_t launch_map_t(const mclahe_plan_s &p, const float *in, float *out,
                                const unsigned char *ws, cudaStream_t st, unsigned grid,
                                size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_map<D, A, REPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    k_map<D, A, REPL><<<grid, p.t.map_threads, smem, st>>>(
        p.g, in, out, reinterpret_cast<const float *>(ws + p.ws.lut),
        reinterpret_cast<const float *>(ws + p.ws.lo), reinterpret_cast<const float *>(ws + p.ws.scale),
        p.t.map_chunks);
    return cudaGetLastError();
}

template <int D>
static cudaError_t launch_map_d(const mclahe_plan_s &p, const float *in, float *out,
                                const unsigned char *ws, cudaStream_t st) {
    const Geom &g = p.g;
    const unsigned grid = unsigned(n_cells(g) * p.t.map_chunks);
    const size_t smem = map_smem_bytes(g);
    const bool repl = map_replicated(g);
    if (g.mode == MCLAHE_RANGE_ADAPTIVE)
        return repl ? launch_map_t<D, true, true>(p, in, out, ws, st, grid, smem)
                    : launch_map_t<D, true, false>(p, in, out, ws, st, grid, smem);
    return repl ? launch_map_t<D, false, true>(p, in, out, ws, st, grid, smem)
                : launch_map_t<D, false, false>(p, in, out, ws, st, grid, smem);
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
