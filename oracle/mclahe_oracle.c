/*
 * mclahe_oracle.c -- plain, slow CPU reference of Multidimensional Contrast
 * Limited Adaptive Histogram Equalization (MCLAHE; Stimper, Bauer, Ernstorfer,
 * Schoelkopf, Xian, arXiv:1906.11355).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Everything is computed in FP64, except the bin quantiser, which the paper
 * leaves unspecified ("histogram(b, n_bins)", Algorithm 1) and which is fixed
 * here in IEEE FP32 with round-to-nearest and no contraction (see orc_bin), so
 * that histograms computed elsewhere can be compared bit for bit.
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes):
 *   R1  padding length: Eq. (1), p = 2b - 1 - ((s - 1) mod b).  Algorithm 1
 *       prints "+" in its first step; only "-" makes s + p a multiple of b.
 *   R2  symmetric padding (Sec. III.B): edge-inclusive mirror, padded index
 *       j < 0 -> -1 - j, j >= s -> 2s - 1 - j.  Requires 1 <= b <= s.
 *   R3  global histogram range (Sec. III.D): [min, max] of the input, or a
 *       caller-supplied [lo, hi].
 *   R4  bin quantiser: scale = fp32(nb) / fp32(hi - lo) (0 when hi <= lo),
 *       bin = clamp(floor(fp32(fp32(x - lo) * scale)), 0, nb - 1).
 *   R5  clip limit (Algorithm 1 parameters): threshold T = clip_limit * V,
 *       V = voxels per kernel, real valued.
 *   R6  redistribution (Algorithm 1): one pass; the excess above T is added
 *       in equal shares E / nb to every bin, clipped ones included.
 *   R7  kernel centre along dim j: k * b_j + (b_j - 1) / 2 in padded
 *       coordinates; the voxel at original index x sits at x + p_j0.
 *   R8  normalisation (Algorithm 1): (cdf - min cdf) / (max cdf - min cdf);
 *       when max == min the mapping is identically 0.
 *   R9  output is the interpolated mapping in [0, 1], not rescaled.
 *
 * Build: cc -std=c11 -O2 -fPIC -shared -ffp-contract=off -fopenmp
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

/* Threads of the OpenMP loops below (n < 1: all processors); timing only,
 * the results do not depend on it. */
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }

#define ORC_MAXDIM 4

typedef struct {
    int ndim;
    int64_t s[ORC_MAXDIM];   /* original shape                       */
    int64_t b[ORC_MAXDIM];   /* kernel size                          */
    int64_t p[ORC_MAXDIM];   /* total padding, Eq. (1)               */
    int64_t p0[ORC_MAXDIM];  /* padding before, Eq. (2)              */
    int64_t p1[ORC_MAXDIM];  /* padding after, Eq. (2)               */
    int64_t ps[ORC_MAXDIM];  /* padded shape s + p                   */
    int64_t n[ORC_MAXDIM];   /* kernels per dim, (s + p) / b         */
    int64_t n_kernels;       /* product of n                         */
    int64_t V;               /* voxels per kernel, product of b      */
    int64_t n_voxels;        /* product of s                         */
    int64_t n_padded;        /* product of ps                        */
} orc_geom;

/* Sec. III.B, Eq. (1) and Eq. (2); Algorithm 1, first step (reading R1). */
static int geom_init(orc_geom *g, int ndim, const int64_t *shape, const int64_t *ksize)
{
    if (ndim < 1 || ndim > ORC_MAXDIM) return -1;
    g->ndim = ndim;
    g->n_kernels = 1;
    g->V = 1;
    g->n_voxels = 1;
    g->n_padded = 1;
    for (int j = 0; j < ndim; ++j) {
        int64_t s = shape[j], b = ksize[j];
        if (s < 1 || b < 1 || b > s) return -1;   /* reading R2 */
        g->s[j] = s;
        g->b[j] = b;
        g->p[j] = 2 * b - 1 - ((s - 1) % b);
        g->p0[j] = g->p[j] / 2;
        g->p1[j] = (g->p[j] + 1) / 2;
        g->ps[j] = s + g->p[j];
        g->n[j] = g->ps[j] / b;
        g->n_kernels *= g->n[j];
        g->V *= b;
        g->n_voxels *= s;
        g->n_padded *= g->ps[j];
    }
    return 0;
}

/* Reading R2: original index of padded index P along one dimension. */
static int64_t mirror(int64_t P, int64_t p0, int64_t s)
{
    int64_t x = P - p0;
    if (x < 0) x = -1 - x;
    if (x >= s) x = 2 * s - 1 - x;
    return x;
}

/* Geometry query: writes p, p0, p1, n (ndim entries each). */
int orc_geometry(int ndim, const int64_t *shape, const int64_t *ksize,
                 int64_t *p, int64_t *p0, int64_t *p1, int64_t *n)
{
    orc_geom g;
    if (geom_init(&g, ndim, shape, ksize)) return -1;
    for (int j = 0; j < ndim; ++j) {
        p[j] = g.p[j];
        p0[j] = g.p0[j];
        p1[j] = g.p1[j];
        n[j] = g.n[j];
    }
    return 0;
}

/* Algorithm 1, second step: symmetric padding of the whole volume (Sec. III.B,
 * reading R2).  padded has prod(s + p) entries, C order. */
static void pad_volume(const orc_geom *g, const float *in, float *padded)
{
    int D = g->ndim;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < g->n_padded; ++q) {
        int64_t rem = q, src = 0, stride = 1;
        int64_t P[ORC_MAXDIM];
        for (int j = D - 1; j >= 0; --j) {
            P[j] = rem % g->ps[j];
            rem /= g->ps[j];
        }
        for (int j = D - 1; j >= 0; --j) {
            src += mirror(P[j], g->p0[j], g->s[j]) * stride;
            stride *= g->s[j];
        }
        padded[q] = in[src];
    }
}

int orc_pad(int ndim, const int64_t *shape, const int64_t *ksize, const float *in, float *padded)
{
    orc_geom g;
    if (geom_init(&g, ndim, shape, ksize)) return -1;
    pad_volume(&g, in, padded);
    return 0;
}

/* Reading R4: fp32 scale of a histogram range. */
float orc_scale(float lo, float hi, int nb)
{
    volatile float width = hi - lo;  /* fp32, round to nearest */
    if (!(hi > lo)) return 0.0f;
    volatile float s = (float)nb / width;
    return s;
}

/* Reading R4: fp32 bin quantiser.  The two fp32 operations are kept apart
 * (volatile) so no compiler may fuse them into one rounding. */
int orc_bin(float x, float lo, float scale, int nb)
{
    volatile float diff = x - lo;
    volatile float y = diff * scale;
    if (!(y > 0.0f)) return 0;                  /* negatives and NaN */
    if (y >= (float)(nb - 1)) return nb - 1;
    return (int)floorf(y);
}

/* Reading R3: global range = [min, max] of the input. */
void orc_global_range(const float *x, int64_t count, float *lo, float *hi)
{
    float mn = x[0], mx = x[0];
    for (int64_t i = 1; i < count; ++i) {
        if (x[i] < mn) mn = x[i];
        if (x[i] > mx) mx = x[i];
    }
    *lo = mn;
    *hi = mx;
}

/* Offset (into the padded volume) of voxel v of kernel k, both flat C-order
 * indices over the kernel grid n and the kernel shape b (Algorithm 1, third
 * step: the padded volume split into adjoining kernels of size b). */
static int64_t kernel_voxel_offset(const orc_geom *g, int64_t k, int64_t v)
{
    int D = g->ndim;
    int64_t kk[ORC_MAXDIM], vv[ORC_MAXDIM];
    for (int j = D - 1; j >= 0; --j) {
        kk[j] = k % g->n[j];
        k /= g->n[j];
        vv[j] = v % g->b[j];
        v /= g->b[j];
    }
    int64_t off = 0;
    for (int j = 0; j < D; ++j) off = off * g->ps[j] + kk[j] * g->b[j] + vv[j];
    return off;
}

/* Sec. III.D (adaptive histogram range): per kernel, [min, max] of the
 * intensities of that kernel in the padded volume. */
static void kernel_ranges(const orc_geom *g, const float *padded, float *lo, float *hi)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t k = 0; k < g->n_kernels; ++k) {
        float mn = padded[kernel_voxel_offset(g, k, 0)], mx = mn;
        for (int64_t v = 1; v < g->V; ++v) {
            float x = padded[kernel_voxel_offset(g, k, v)];
            if (x < mn) mn = x;
            if (x > mx) mx = x;
        }
        lo[k] = mn;
        hi[k] = mx;
    }
}

/* Per-kernel histogram ranges: GHR (mode 0) one range for all kernels, from
 * range[] if given else the input's min/max (R3); AHR (mode 1) each kernel's
 * own min/max (Sec. III.D).  Writes lo_k[K], scale_k[K]. */
static void histogram_ranges(const orc_geom *g, int mode, int nb, const float *range,
                             const float *in, const float *padded, float *lo_k, float *scale_k)
{
    if (mode == 0) {
        float lo, hi;
        if (range) {
            lo = range[0];
            hi = range[1];
        } else {
            orc_global_range(in, g->n_voxels, &lo, &hi);
        }
        float sc = orc_scale(lo, hi, nb);
        for (int64_t k = 0; k < g->n_kernels; ++k) {
            lo_k[k] = lo;
            scale_k[k] = sc;
        }
    } else {
        float *hi_k = (float *)malloc(sizeof(float) * g->n_kernels);
        kernel_ranges(g, padded, lo_k, hi_k);
        for (int64_t k = 0; k < g->n_kernels; ++k) scale_k[k] = orc_scale(lo_k[k], hi_k[k], nb);
        free(hi_k);
    }
}

/* Algorithm 1, fourth and fifth steps: for every kernel of the padded volume,
 * the n_bins histogram of its V intensities (one count per padded voxel). */
static void histograms(const orc_geom *g, int nb, const float *padded,
                       const float *lo_k, const float *scale_k, uint64_t *hist)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t k = 0; k < g->n_kernels; ++k) {
        uint64_t *h = hist + k * nb;
        for (int i = 0; i < nb; ++i) h[i] = 0;
        for (int64_t v = 0; v < g->V; ++v) {
            float x = padded[kernel_voxel_offset(g, k, v)];
            h[orc_bin(x, lo_k[k], scale_k[k], nb)] += 1;
        }
    }
}

/* Algorithm 1, sixth to eighth steps, for one kernel: clip the histogram at
 * T = clip * V (R5), redistribute the excess equally over all bins (R6), take
 * the cumulative distribution and normalise it by its min and max (R8).
 * hclip (nullable) receives the clipped-and-redistributed histogram. */
void orc_clip_lut(const uint64_t *h, int nb, int64_t V, double clip, double *lut, double *hclip)
{
    double T = clip * (double)V;
    double excess = 0.0;
    for (int i = 0; i < nb; ++i)
        if ((double)h[i] > T) excess += (double)h[i] - T;
    double *hc = (double *)malloc(sizeof(double) * nb);
    for (int i = 0; i < nb; ++i) hc[i] = ((double)h[i] > T ? T : (double)h[i]) + excess / nb;
    double *cdf = (double *)malloc(sizeof(double) * nb);
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) {
        acc += hc[i];
        cdf[i] = acc;
    }
    double mn = cdf[0], mx = cdf[0];
    for (int i = 1; i < nb; ++i) {
        if (cdf[i] < mn) mn = cdf[i];
        if (cdf[i] > mx) mx = cdf[i];
    }
    for (int i = 0; i < nb; ++i) lut[i] = (mx > mn) ? (cdf[i] - mn) / (mx - mn) : 0.0;
    if (hclip)
        for (int i = 0; i < nb; ++i) hclip[i] = hc[i];
    free(cdf);
    free(hc);
}

/* Sec. III.C: the lower of the two nearest kernels along one dimension and the
 * distances d0 (to its centre) and d1 (to the next kernel's centre) of a voxel
 * at original index x (R7).  Kernel centres are half-integers k*b + (b-1)/2;
 * the lower neighbour is the largest k with centre <= x + p0. */
static void neighbours_1d(int64_t x, int64_t b, int64_t p0, int64_t *k0, double *d0, double *d1)
{
    int64_t P = x + p0;
    int64_t k = (2 * P - (b - 1)) / (2 * b);   /* 2P - (b-1) >= 0 since p0 >= (b-1)/2 */
    double centre = (double)k * (double)b + 0.5 * (double)(b - 1);
    *k0 = k;
    *d0 = (double)P - centre;
    *d1 = (double)b - *d0;                      /* next centre is b further on */
}

/* Sec. III.C, Eq. (12)-(13); Algorithm 1, the interpolation loop: every voxel
 * is mapped by each of its 2^D nearest kernels, m_i(I) = normalised CDF of
 * kernel i at the voxel's bin (Eq. (3)), and the results are combined with the
 * Lagrange coefficients c_i = prod_j (b_j - d_{j,i_j}) / b_j. */
static void map_voxels(const orc_geom *g, int nb, const float *in, const double *lut,
                       const float *lo_k, const float *scale_k, double *out)
{
    int D = g->ndim;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < g->n_voxels; ++q) {
        int64_t x[ORC_MAXDIM], k0[ORC_MAXDIM];
        double d[ORC_MAXDIM][2];
        int64_t rem = q;
        for (int j = D - 1; j >= 0; --j) {
            x[j] = rem % g->s[j];
            rem /= g->s[j];
        }
        for (int j = 0; j < D; ++j) neighbours_1d(x[j], g->b[j], g->p0[j], &k0[j], &d[j][0], &d[j][1]);
        double acc = 0.0;
        for (int i = 0; i < (1 << D); ++i) {       /* corner i = (i_0, ..., i_{D-1}) */
            double c = 1.0;
            int64_t k = 0;
            for (int j = 0; j < D; ++j) {
                int ij = (i >> (D - 1 - j)) & 1;
                c *= ((double)g->b[j] - d[j][ij]) / (double)g->b[j];
                k = k * g->n[j] + k0[j] + ij;
            }
            int bin = orc_bin(in[q], lo_k[k], scale_k[k], nb);
            acc += c * lut[k * nb + bin];
        }
        out[q] = acc;
    }
}

/* Map with caller-given mapping tables (used to check the interpolation on its
 * own).  lut: K * nb doubles; lo_k, scale_k: K floats. */
int orc_map(int ndim, const int64_t *shape, const int64_t *ksize, int nb, const float *in,
            const double *lut, const float *lo_k, const float *scale_k, double *out)
{
    orc_geom g;
    if (geom_init(&g, ndim, shape, ksize) || nb < 2) return -1;
    map_voxels(&g, nb, in, lut, lo_k, scale_k, out);
    return 0;
}

/* Histograms of all kernels (Algorithm 1, steps one to five).  hist: K * nb;
 * lo_k, scale_k: K floats each (outputs). */
int orc_histograms(int ndim, const int64_t *shape, const int64_t *ksize, int nb, int mode,
                   const float *range, const float *in, uint64_t *hist, float *lo_k, float *scale_k)
{
    orc_geom g;
    if (geom_init(&g, ndim, shape, ksize) || nb < 2 || (mode != 0 && mode != 1)) return -1;
    float *padded = (float *)malloc(sizeof(float) * g.n_padded);
    if (!padded) return -2;
    pad_volume(&g, in, padded);
    histogram_ranges(&g, mode, nb, range, in, padded, lo_k, scale_k);
    histograms(&g, nb, padded, lo_k, scale_k, hist);
    free(padded);
    return 0;
}

/* The whole of Algorithm 1.  out: prod(shape) doubles.  hist (K*nb), lut
 * (K*nb), lo_k and scale_k (K) are optional outputs (nullable). */
int orc_mclahe(int ndim, const int64_t *shape, const int64_t *ksize, int nb, double clip, int mode,
               const float *range, const float *in, double *out, uint64_t *hist_out,
               double *lut_out, float *lo_out, float *scale_out)
{
    orc_geom g;
    if (geom_init(&g, ndim, shape, ksize) || nb < 2 || (mode != 0 && mode != 1)) return -1;
    int64_t K = g.n_kernels;
    uint64_t *hist = hist_out ? hist_out : (uint64_t *)malloc(sizeof(uint64_t) * K * nb);
    double *lut = lut_out ? lut_out : (double *)malloc(sizeof(double) * K * nb);
    float *lo_k = lo_out ? lo_out : (float *)malloc(sizeof(float) * K);
    float *scale_k = scale_out ? scale_out : (float *)malloc(sizeof(float) * K);
    int rc = orc_histograms(ndim, shape, ksize, nb, mode, range, in, hist, lo_k, scale_k);
    if (rc == 0) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < K; ++k) orc_clip_lut(hist + k * nb, nb, g.V, clip, lut + k * nb, NULL);
        map_voxels(&g, nb, in, lut, lo_k, scale_k, out);
    }
    if (!hist_out) free(hist);
    if (!lut_out) free(lut);
    if (!lo_out) free(lo_k);
    if (!scale_out) free(scale_k);
    return rc;
}

/* Reverse mode of Algorithm 1's sixth to eighth steps for one kernel: given
 * dL/dlut (gl, nb entries) return dL/dT.  The steps are undone in reverse
 * order: normalisation (R8), cumulative sum, redistribution and clip (R5, R6).
 * At a kink (a count exactly equal to T) the clip indicator [h > T] is used. */
double orc_lut_backward(const uint64_t *h, int nb, int64_t V, double clip, const double *gl)
{
    double T = clip * (double)V;
    double excess = 0.0;
    int nclip = 0;
    for (int i = 0; i < nb; ++i)
        if ((double)h[i] > T) {
            excess += (double)h[i] - T;
            nclip += 1;
        }
    double *cdf = (double *)malloc(sizeof(double) * nb);
    double *gc = (double *)calloc(nb, sizeof(double));
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) {
        acc += ((double)h[i] > T ? T : (double)h[i]) + excess / nb;
        cdf[i] = acc;
    }
    double lo = cdf[0], span = cdf[nb - 1] - cdf[0];  /* the cdf is nondecreasing */
    double gT = 0.0;
    if (span > 0.0) {
        /* lut_j = (cdf_j - cdf_0) / (cdf_{nb-1} - cdf_0) */
        for (int j = 0; j < nb; ++j) {
            double num = cdf[j] - lo;
            gc[j] += gl[j] / span;
            gc[0] += gl[j] * (-1.0 / span + num / (span * span));
            gc[nb - 1] += -gl[j] * num / (span * span);
        }
        /* cdf_j = sum_{i<=j} h'_i  ->  dL/dh'_i = sum_{j>=i} dL/dcdf_j */
        double suffix = 0.0;
        for (int i = nb - 1; i >= 0; --i) {
            suffix += gc[i];
            /* h'_i = min(h_i, T) + E/nb, E = sum_{h>T} (h - T) */
            double dh_dT = ((double)h[i] > T ? 1.0 : 0.0) - (double)nclip / nb;
            gT += suffix * dh_dT;
        }
    }
    free(gc);
    free(cdf);
    return gT;
}

/* Gradient of L = sum_v g_v * out_v with respect to the mapping tables and the
 * clip limit.  The mapping step (Eq. (12)-(13)) is linear in the tables, so
 * dL/dlut[k][j] = sum over voxels v and corners i with k0(v)+i = k and
 * bin_k(v) = j of g_v * c_i(v); then dL/dclip = V * sum_k dL/dT_k.
 * grad_lut (K*nb, nullable), grad_clip (scalar). */
int orc_mclahe_backward(int ndim, const int64_t *shape, const int64_t *ksize, int nb, double clip,
                        int mode, const float *range, const float *in, const double *grad_out,
                        double *grad_lut_out, double *grad_clip)
{
    orc_geom g;
    if (geom_init(&g, ndim, shape, ksize) || nb < 2 || (mode != 0 && mode != 1)) return -1;
    int D = g.ndim;
    int64_t K = g.n_kernels;
    uint64_t *hist = (uint64_t *)malloc(sizeof(uint64_t) * K * nb);
    float *lo_k = (float *)malloc(sizeof(float) * K);
    float *scale_k = (float *)malloc(sizeof(float) * K);
    double *gl = (double *)calloc(K * nb, sizeof(double));
    int rc = orc_histograms(ndim, shape, ksize, nb, mode, range, in, hist, lo_k, scale_k);
    if (rc == 0) {
        for (int64_t q = 0; q < g.n_voxels; ++q) {      /* serial: fixed summation order */
            int64_t x[ORC_MAXDIM], k0[ORC_MAXDIM];
            double d[ORC_MAXDIM][2];
            int64_t rem = q;
            for (int j = D - 1; j >= 0; --j) {
                x[j] = rem % g.s[j];
                rem /= g.s[j];
            }
            for (int j = 0; j < D; ++j) neighbours_1d(x[j], g.b[j], g.p0[j], &k0[j], &d[j][0], &d[j][1]);
            for (int i = 0; i < (1 << D); ++i) {
                double c = 1.0;
                int64_t k = 0;
                for (int j = 0; j < D; ++j) {
                    int ij = (i >> (D - 1 - j)) & 1;
                    c *= ((double)g.b[j] - d[j][ij]) / (double)g.b[j];
                    k = k * g.n[j] + k0[j] + ij;
                }
                gl[k * nb + orc_bin(in[q], lo_k[k], scale_k[k], nb)] += grad_out[q] * c;
            }
        }
        double gclip = 0.0;
        for (int64_t k = 0; k < K; ++k)
            gclip += (double)g.V * orc_lut_backward(hist + k * nb, nb, g.V, clip, gl + k * nb);
        *grad_clip = gclip;
        if (grad_lut_out) memcpy(grad_lut_out, gl, sizeof(double) * K * nb);
    }
    free(gl);
    free(scale_k);
    free(lo_k);
    free(hist);
    return rc;
}
