// k_map.cu -- the mapping pass of one float32 volume (Sec. III.C, Eq.
// (12)-(13); kernels and launch templates in k_map_impl.cuh): table layout,
// TMA box and the launch.
#include "k_map_impl.cuh"

namespace mclahe {

bool map_replicated(const Geom &g) { return map_repl_fits(g.P); }
size_t map_smem_bytes(const Geom &g) { return map_smem_for(g.D, g.P); }

static int largest_divisor_at_most(int n, int cap) {
    for (int d = std::min(n, cap); d > 1; --d)
        if (n % d == 0) return d;
    return 1;
}

// Whether the TMA walk applies (3- and 4-D, replicated tables, every cell
// row starting on a 16-byte boundary, rows of 16-byte multiples), and its box.
bool map_tma_box(const Geom &g, int &bx, int &by, int &bz) {
    if (g.D < 3 || !map_repl_fits(g.P)) return false;
    const Dim &dl = g.d[g.D - 1];
    if (dl.s % 4 != 0 || dl.b % 4 != 0 || dl.b > 256) return false;
    for (int c = 0; c + 1 < dl.n; ++c) {
        const int lo = std::min(std::max(c * dl.b + dl.b / 2 - dl.p0, 0), dl.s);
        if (lo % 4 != 0) return false;
    }
    bx = dl.b;
    by = largest_divisor_at_most(g.d[g.D - 2].b, std::min(256, kTmaTileFloats / bx));
    bz = g.D == 4 ? largest_divisor_at_most(g.d[1].b, std::min(256, kTmaTileFloats / (bx * by))) : 1;
    return true;
}

cudaError_t launch_map(const mclahe_plan_s &p, const float *in, float *out,
                       const unsigned char *ws, cudaStream_t st) {
    return launch_map_any(p, in, out, ws, st);
}

cudaError_t launch_map_cells(const mclahe_plan_s &p, const float *in, float *out,
                             const unsigned char *ws, cudaStream_t st, int64_t cell0, int64_t ncells) {
    return launch_map_any(p, in, out, ws, st, cell0, ncells);
}

}  // namespace mclahe
