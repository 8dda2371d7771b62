/*
 * mclahe.h -- C ABI of the GB300 (sm_103a) implementation of Multidimensional
 * Contrast Limited Adaptive Histogram Equalization (MCLAHE; Stimper, Bauer,
 * Ernstorfer, Schoelkopf, Xian, arXiv:1906.11355).
 *
 * The operation (Algorithm 1 of the paper):
 *   1. pad the D-dimensional volume symmetrically so that it splits into whole
 *      kernels of size b and every voxel has 2^D neighbouring kernels
 *      (Sec. III.B, Eq. (1)-(2));
 *   2. build one n_bins histogram per kernel, over a global or a per-kernel
 *      adaptive intensity range (Algorithm 1; Sec. III.D);
 *   3. clip each histogram at the clip limit, redistribute the excess equally,
 *      and turn its CDF, normalised by its min and max, into the kernel's
 *      mapping table (Algorithm 1);
 *   4. map every voxel by the multilinear (Lagrange) interpolation of its 2^D
 *      neighbouring kernels' tables at the voxel's bin (Sec. III.C,
 *      Eq. (12)-(13)).
 *
 * Conventions shared by every entry point
 *   - Volumes are float32, C order (dimension 0 slowest, D-1 contiguous),
 *     1 <= D <= 4, every extent >= 1, and the device pointers are 16-byte
 *     aligned.  Intensities must be finite.
 *   - The caller owns every device buffer and the stream.  The library owns
 *     only host-side plan objects; it never allocates device memory.
 *   - No entry point synchronises the stream unless it says so.  Argument
 *     errors are returned synchronously and leave the device untouched.
 *     A failed kernel launch returns MCLAHE_ERR_CUDA.  Errors found by device
 *     code are written to the status word at the start of the workspace and
 *     are read back by mclahe_sync_status(); a new workspace must start with
 *     that word zero (allocate it zeroed, or call mclahe_sync_status once).
 *   - Readings of points the paper leaves open:
 *       padding length p = 2b - 1 - ((s - 1) mod b) (Eq. (1); Algorithm 1's
 *         first step prints "+", which cannot make s + p a multiple of b);
 *       symmetric padding = edge-inclusive mirror, which needs b <= s;
 *       bin quantiser: scale = n_bins / (hi - lo) in fp32 (0 if hi <= lo),
 *         bin = clamp(floor((x - lo) * scale), 0, n_bins - 1), each operation
 *         rounded to nearest in fp32;
 *       global range = [min, max] of the input unless given;
 *       clip threshold T = clip_limit * V, V = prod(b) voxels per kernel;
 *       excess E = sum over bins of max(h - T, 0), added as E / n_bins to
 *         every bin (one pass);
 *       kernel centre along dim j = k * b_j + (b_j - 1) / 2 in padded
 *         coordinates; a voxel at original index x sits at x + p_j0;
 *       a kernel whose CDF is constant gets the all-zero table;
 *       the output lies in [0, 1] and is not rescaled to the input range.
 */
#ifndef MCLAHE_H
#define MCLAHE_H

#include <stddef.h>
#include <stdint.h>

#if defined(MCLAHE_BUILD) && defined(__GNUC__)
#define MCLAHE_API __attribute__((visibility("default")))
#else
#define MCLAHE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-compatible with cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *mclahe_stream_t;

/* Opaque host-side plan (geometry, parameters, launch shapes). */
typedef struct mclahe_plan_s *mclahe_plan_t;

typedef enum {
    MCLAHE_OK = 0,
    MCLAHE_ERR_INVALID_ARG = 1,   /* bad shape, kernel size, bins, clip, pointer */
    MCLAHE_ERR_UNSUPPORTED = 2,   /* valid in the paper, outside this build's limits */
    MCLAHE_ERR_WORKSPACE = 3,     /* workspace missing, too small or misaligned */
    MCLAHE_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
    MCLAHE_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    MCLAHE_ERR_NO_MEMORY = 6,     /* host allocation failed */
    MCLAHE_ERR_DEVICE = 7         /* device code recorded an internal error */
} mclahe_status;

typedef enum {
    MCLAHE_RANGE_GLOBAL = 0,      /* one histogram range for all kernels (GHR) */
    MCLAHE_RANGE_ADAPTIVE = 1     /* each kernel's own [min, max] (AHR, Sec. III.D) */
} mclahe_range_mode;

/* Geometry and workspace layout of a plan (filled by mclahe_plan_query). */
typedef struct {
    int32_t ndim;
    int32_t n_bins;
    int32_t mode;                 /* mclahe_range_mode */
    float clip_limit;
    int64_t shape[4];             /* s */
    int64_t kernel_size[4];       /* b */
    int64_t pad[4];               /* p, Eq. (1) */
    int64_t pad_before[4];        /* p0 = p // 2, Eq. (2) */
    int64_t pad_after[4];         /* p1 = (p + 1) // 2, Eq. (2) */
    int64_t n_kernels_dim[4];     /* n = (s + p) / b */
    int64_t n_kernels;            /* K = prod(n) */
    int64_t kernel_voxels;        /* V = prod(b) */
    int64_t n_voxels;             /* prod(s) */
    int64_t table_stride;         /* floats per mapping-table row in the workspace (>= n_bins;
                                     entries past n_bins - 1 repeat it) */
    /* byte offsets inside the workspace (all 256-byte aligned) */
    size_t ws_status;             /* uint32 status word */
    size_t ws_range_keys;         /* uint32 [2 + 2K] order-preserving min/max keys: the global
                                     range, then each kernel's adaptive range (flat pass) */
    size_t ws_hist;               /* uint32 [K][n_bins] kernel histograms */
    size_t ws_lo;                 /* float  [K] histogram range start per kernel */
    size_t ws_scale;              /* float  [K] histogram scale per kernel */
    size_t ws_lut;                /* float  [K][table_stride] mapping tables */
    size_t ws_scratch;            /* backward partials */
    size_t ws_bytes;              /* total workspace size */
    /* launch shapes (defaults, or those picked by mclahe_autotune) */
    int32_t hist_group;           /* kernels along the last dim per histogram work item */
    int32_t hist_cluster;         /* CTAs (a thread-block cluster) per histogram work item */
    int32_t hist_copies;          /* lane copies of the shared-memory histograms */
    int32_t map_chunks;           /* CTAs per inter-kernel cell in the mapping pass */
    int32_t bwd_chunks;           /* CTAs per inter-kernel cell in the backward pass */
    int32_t tuned;                /* 1 if the shapes come from mclahe_autotune, 2 if from
                                     mclahe_plan_set_shapes, else 0 */
    int32_t hist_shares;          /* > 0: the histogram pass is flat: every work item is cut
                                     into hist_shares equal shares of its rows, dealt out in
                                     order to a persistent grid (hist_cluster is then 1);
                                     0: one cluster per work item */
    int32_t hist_ctas;            /* CTAs of the flat histogram pass at its last launch (0 if
                                     not flat or not launched yet) */
    int32_t map_tma;              /* 1: the mapping pass streams its cells as TMA box tiles */
    int32_t hist_walk;            /* rows of the histogram pass: 0 cp.async ring, 1 TMA box
                                     tiles, 2 per-thread loads (least shared memory), 3 the
                                     kernel's footprint staged in the cluster's shared memory */
    int32_t hist_threads;         /* threads per histogram CTA (256; 512 allowed for 4-D) */
    int32_t map_flat;             /* 1: the mapping pass deals map_chunks shares per cell out to
                                     a persistent grid (per-thread walk only) */
    int32_t range_pass;           /* 1 (adaptive range, cluster form, walks 0-2): the per-kernel
                                     ranges come from a streaming sweep before the histogram
                                     pass (mclahe_plan_set_range_pass) */
} mclahe_plan_info;

/*
 * mclahe_plan -- validate parameters and build a plan (host only; no CUDA call).
 * Paper: Algorithm 1 (inputs data_in; parameters kernel_size, clip_limit in
 * [0, 1], n_bins), Sec. III.B (padding geometry), Sec. III.D (range mode).
 *   out          receives the plan; release it with mclahe_plan_destroy.
 *   ndim         D, 1..4.
 *   shape        D extents s_i >= 1.
 *   kernel_size  D kernel extents, 1 <= b_i <= s_i (the mirror padding of
 *                Sec. III.B reflects at most once).
 *   n_bins       2..4096.
 *   clip_limit   [0, 1]; the forward pass may override it per call.
 *   mode         MCLAHE_RANGE_GLOBAL or MCLAHE_RANGE_ADAPTIVE.
 *   global_range nullable {lo, hi}; GHR only.  NULL: the input's min and max,
 *                found on the device by every forward call.
 * Returns MCLAHE_OK, MCLAHE_ERR_INVALID_ARG, MCLAHE_ERR_UNSUPPORTED (volume or
 * kernel too large for 32-bit counters), MCLAHE_ERR_NO_MEMORY.
 */
MCLAHE_API mclahe_status mclahe_plan(mclahe_plan_t *out, int ndim, const int64_t *shape,
                          const int32_t *kernel_size, int32_t n_bins, float clip_limit,
                          mclahe_range_mode mode, const float *global_range);

/* Release a plan (NULL is ignored). */
MCLAHE_API void mclahe_plan_destroy(mclahe_plan_t plan);

/* Fill *info with the plan's geometry and workspace layout. */
MCLAHE_API mclahe_status mclahe_plan_query(mclahe_plan_t plan, mclahe_plan_info *info);

/* Bytes of device workspace one forward/backward call of this plan needs
 * (0 for a NULL plan).  The caller allocates it, 256-byte aligned. */
MCLAHE_API size_t mclahe_workspace_bytes(mclahe_plan_t plan);

/*
 * mclahe_forward -- the whole of Algorithm 1 on one volume, on `stream`.
 * Paper: Algorithm 1; Sec. III.B-III.D; Eq. (1)-(3), (12)-(13).
 *   d_in      device, prod(shape) float32, read only.
 *   d_out     device, prod(shape) float32, written; must not alias d_in.
 *   d_ws      device workspace of ws_bytes >= mclahe_workspace_bytes(plan).
 *             On return (in stream order) it holds the range, the kernel
 *             histograms and the mapping tables at the offsets of
 *             mclahe_plan_info; mclahe_backward reads them.
 *   d_clip    nullable device float: clip limit for this call (overrides the
 *             plan's; read on the device, so it can be a learnable parameter).
 *             Values outside [0, 1] are clamped.
 * Returns MCLAHE_OK, MCLAHE_ERR_INVALID_ARG (NULL or misaligned pointers),
 * MCLAHE_ERR_WORKSPACE, MCLAHE_ERR_CUDA.
 */
MCLAHE_API mclahe_status mclahe_forward(mclahe_plan_t plan, const float *d_in, float *d_out, void *d_ws,
                             size_t ws_bytes, const float *d_clip, mclahe_stream_t stream);

/*
 * mclahe_forward_graph -- mclahe_forward through a CUDA graph: the forward's
 * launches (the clear, range, histogram and mapping passes) are captured once
 * per (plan, d_in, d_out, d_ws, d_clip) and device into a graph the library
 * caches for the process, and replayed on `stream` by every call with the
 * same arguments (no counterpart in the paper).  For small volumes, whose
 * passes are a few microseconds each, this removes the per-launch costs.
 * Arguments and errors as for mclahe_forward; changing the plan's launch
 * shapes or destroying it drops its graphs.
 */
MCLAHE_API mclahe_status mclahe_forward_graph(mclahe_plan_t plan, const float *d_in, float *d_out,
                                              void *d_ws, size_t ws_bytes, const float *d_clip,
                                              mclahe_stream_t stream);

/* Element types of an input volume (mclahe_forward_typed). */
typedef enum {
    MCLAHE_F32 = 0,   /* float32 */
    MCLAHE_U16 = 1,   /* uint16: intensity = the integer (exact in fp32) */
    MCLAHE_U8 = 2     /* uint8: intensity = the integer */
} mclahe_dtype;

/*
 * mclahe_forward_typed -- mclahe_forward for a volume stored as float32,
 * uint16 or uint8 (Algorithm 1; Sec. III.B-III.D).  The paper's fluorescence
 * data are 8-bit (Sec. IV.B) and detectors commonly write 16-bit counts;
 * reading them as they are moves 2 or 1 bytes per voxel per pass instead of 4.
 * An integer voxel's intensity is the integer itself, converted to fp32
 * (exactly), so the output, histograms, ranges and tables equal those of
 * mclahe_forward on the float32 volume of the same values; a given global
 * range is in those units.  The output is float32 in [0, 1].
 *   dtype     MCLAHE_F32 (same as mclahe_forward), MCLAHE_U16 or MCLAHE_U8.
 *   d_in      device, prod(shape) elements of dtype, 16-byte aligned.
 *   others    as for mclahe_forward.
 * Integer volumes take the cluster form of the histogram pass (or the staged
 * walk) and the per-thread mapping walks, whatever the plan's shapes.
 * mclahe_backward and mclahe_batch take float32 volumes only.
 * Returns as mclahe_forward, and MCLAHE_ERR_INVALID_ARG for an unknown dtype.
 */
MCLAHE_API mclahe_status mclahe_forward_typed(mclahe_plan_t plan, mclahe_dtype dtype, const void *d_in,
                                              float *d_out, void *d_ws, size_t ws_bytes,
                                              const float *d_clip, mclahe_stream_t stream);

/*
 * mclahe_forward_chunked -- Algorithm 1 on a float32 volume held in HOST memory,
 * streamed through a device staging buffer in slabs along dimension 0, for
 * volumes larger than the device (no counterpart in the paper, which names
 * holding the whole dataset in memory as its main limitation, Sec. V).
 * Slabs are cut on kernel boundaries: a global-range sweep (global range not
 * given), a histogram sweep in which each slab holds the whole footprints of a
 * run of kernel rows (their histograms and tables complete in it), then a
 * mapping sweep over runs of cell rows whose output slabs are copied back.
 * The result equals mclahe_forward's (the same kernels, on slabs).
 *   h_in, h_out   host, prod(shape) float32 each (pinned memory lets the
 *                 copies run at full speed), distinct.
 *   d_ws          device workspace as for mclahe_forward (all K tables live in it).
 *   d_stage       device staging buffer of stage_bytes, 256-byte aligned; it
 *                 must hold two slabs of the widest kernel footprint along
 *                 dimension 0 (MCLAHE_ERR_WORKSPACE otherwise).
 *   d_clip        nullable device clip limit, as for mclahe_forward.
 * The histogram pass runs in its cluster form with the cp.async row ring and
 * the mapping pass on its per-cell grid.  2- to 4-D volumes.  Copies and
 * kernels run in order on `stream`; the call returns once all are enqueued
 * (h_out is complete when the stream is).
 * Returns MCLAHE_OK, MCLAHE_ERR_INVALID_ARG, MCLAHE_ERR_UNSUPPORTED (1-D),
 * MCLAHE_ERR_WORKSPACE, MCLAHE_ERR_CUDA.
 */
MCLAHE_API mclahe_status mclahe_forward_chunked(mclahe_plan_t plan, const float *h_in, float *h_out,
                                                void *d_ws, size_t ws_bytes, void *d_stage,
                                                size_t stage_bytes, const float *d_clip,
                                                mclahe_stream_t stream);

/* The passes of mclahe_forward, in the order it runs them. */
typedef enum {
    MCLAHE_PASS_CLEAR = 0,  /* zero what later passes accumulate with atomics (memset): the
                               global range keys; in the flat histogram form also the
                               per-kernel range keys, work-item tickets and histograms */
    MCLAHE_PASS_RANGE = 1,  /* global range, Sec. III.D (GHR without a given range), or each
                               kernel's adaptive range (AHR, flat histogram form) */
    MCLAHE_PASS_HIST = 2,   /* per-kernel histograms (with AHR in the cluster form also their
                               ranges), clip, redistribute, CDF and normalisation
                               (Algorithm 1): one cluster per group of kernels, or the flat
                               form (equal row shares over a persistent grid) */
    MCLAHE_PASS_LUT = 3,    /* no work: the tables are built by MCLAHE_PASS_HIST */
    MCLAHE_PASS_MAP = 4,    /* multilinear mapping, Sec. III.C, Eq. (12)-(13) */
    MCLAHE_N_PASSES = 5
} mclahe_pass;

/*
 * mclahe_forward_pass -- run one pass of mclahe_forward (same arguments and
 * errors).  Calling passes CLEAR..MAP in order on one stream is exactly
 * mclahe_forward; single passes let a caller time or reuse them (for example
 * re-run MAP with tables it has left in the workspace).  d_out may be NULL for
 * every pass but MAP.
 */
MCLAHE_API mclahe_status mclahe_forward_pass(mclahe_plan_t plan, mclahe_pass pass, const float *d_in,
                                             float *d_out, void *d_ws, size_t ws_bytes,
                                             const float *d_clip, mclahe_stream_t stream);

/* Number of this library's kernels a pass launches for this plan (0 for
 * CLEAR, which is a memset, and for RANGE with a caller-given global range). */
MCLAHE_API int mclahe_pass_launches(mclahe_plan_t plan, mclahe_pass pass);

/*
 * Slabs of one volume along dimension 0 (no counterpart in the paper; the
 * building blocks of mclahe_forward_chunked and of splitting one volume across
 * devices, partitioned in slabs with a one-row table halo).
 *
 * mclahe_slab_rows -- host only: the original rows [*first_row, *end_row) along
 * dimension 0 that a slab must hold for
 *   MCLAHE_PASS_RANGE  rows [row0, row1) themselves;
 *   MCLAHE_PASS_HIST   the kernel rows [row0, row1): the union of their
 *                      footprints (Sec. III.B, mirror images included);
 *   MCLAHE_PASS_MAP    the cell rows [row0, row1) (cell c lies between kernel
 *                      rows c and c + 1, Sec. III.C).
 *
 * mclahe_forward_slab -- one pass on a slab: d_slab holds the volume's elements
 * from slab_first on (a multiple of 4, at most first_row * row elements, 16-byte
 * aligned pointer), d_out_slab (MAP only) the output elements from slab_first on.
 *   RANGE  min/max of rows [row0, row1) added to the workspace's global range
 *          keys (global range not given; clear them first, and combine the
 *          keys of several devices by a maximum of each word);
 *   HIST   histograms and tables of the kernel rows [row0, row1) (a global
 *          range must already be in the keys);
 *   MAP    the cell rows [row0, row1), whose tables (kernel rows row0..row1,
 *          table rows, ranges lo and scale) must be in the workspace.
 * Kernel row k's tables are the contiguous workspace rows k K1 .. (k + 1) K1 - 1
 * of lut, lo and scale (K1 = K / n[0] kernels per row, mclahe_plan_info).
 * Returns MCLAHE_OK, MCLAHE_ERR_INVALID_ARG, MCLAHE_ERR_WORKSPACE, MCLAHE_ERR_CUDA.
 */
MCLAHE_API mclahe_status mclahe_slab_rows(mclahe_plan_t plan, mclahe_pass pass, int32_t row0,
                                          int32_t row1, int64_t *first_row, int64_t *end_row);
MCLAHE_API mclahe_status mclahe_forward_slab(mclahe_plan_t plan, mclahe_pass pass, const float *d_slab,
                                             int64_t slab_first, float *d_out_slab, void *d_ws,
                                             size_t ws_bytes, const float *d_clip, int32_t row0,
                                             int32_t row1, mclahe_stream_t stream);

/*
 * mclahe_backward -- adjoint of mclahe_forward (no counterpart in the paper,
 * which does not differentiate MCLAHE).  For the scalar L with upstream
 * gradient g = dL/d(out):
 *   dL/dlut[k][j] = sum over voxels v and corners i with neighbour k and
 *                   bin_k(v) = j of g_v * c_i(v)            (Eq. (12)-(13))
 *   dL/dclip      = V * sum_k dL/dT_k, through the normalisation, the
 *                   cumulative sum and the clip/redistribute step.
 * The output is piecewise constant in the intensities, so dL/d(in) = 0 almost
 * everywhere; no input gradient is produced.
 *   d_in, d_ws    as passed to the mclahe_forward call being differentiated
 *                 (the workspace must still hold that call's range and
 *                 histograms).
 *   d_grad_out    device, prod(shape) float32, finite.
 *   d_clip        the same clip pointer as the forward call (nullable).
 *   d_grad_lut    nullable device float [K][n_bins]: receives dL/dlut.
 *   d_grad_clip   device float scalar: receives dL/dclip_limit.
 * With d_grad_lut given, the per-voxel terms g_v * c_i(v) are summed as
 * fixed-point integers (each rounded at a scale set by max |g|, relative
 * resolution 2^-30 of it); the plan requires kernel_size[D-1] <= 65535.  With
 * d_grad_lut NULL only dL/dclip is formed, as a gather: the tables
 * d lut_kj / dT interpolated like the mapping pass and dotted with g
 * (compensated fp32 per thread, then double in a fixed order).  Both forms are
 * deterministic for a given plan.
 */
MCLAHE_API mclahe_status mclahe_backward(mclahe_plan_t plan, const float *d_in, const float *d_grad_out,
                              void *d_ws, size_t ws_bytes, const float *d_clip, float *d_grad_lut,
                              float *d_grad_clip, mclahe_stream_t stream);

/*
 * mclahe_forward_host -- mclahe_forward_typed on n_vol volumes of one plan
 * that live in host memory (no counterpart in the paper).  Volume v is copied
 * host -> device into slot v mod 2, mapped on `stream`, and its output copied
 * device -> host; the copies run on two library-owned streams, so the input
 * copy of volume v + 1 and the output copy of volume v - 1 overlap the mapping
 * of volume v.  The call returns once everything is enqueued; `stream` then
 * waits for the last output copy (the host outputs are complete when `stream`
 * is).
 *   dtype          element type of the inputs (the outputs are float32).
 *   h_in, h_out    host arrays of n_vol host pointers, prod(shape) elements
 *                  each; page-locked memory lets the copies overlap (pageable
 *                  memory works, serialised).  Outputs may repeat a pointer.
 *   d_in, d_out, d_ws   two-element host arrays of device pointers: the two
 *                  slots' input buffers (prod(shape) elements of dtype,
 *                  16-byte aligned), output buffers (float32) and workspaces
 *                  (ws_bytes each, zeroed once by the caller); all distinct.
 *   d_clip         nullable device float [n_vol] clip limits.
 * Argument errors return before anything is enqueued.  Calls from several host
 * threads are serialised on the host.
 */
MCLAHE_API mclahe_status mclahe_forward_host(mclahe_plan_t plan, mclahe_dtype dtype, int n_vol,
                                             const void *const *h_in, float *const *h_out,
                                             void *const *d_in, float *const *d_out, void *const *d_ws,
                                             size_t ws_bytes, const float *d_clip, mclahe_stream_t stream);

/*
 * mclahe_forward_batch -- mclahe_forward on n_vol volumes of one plan, each
 * with its own workspace (which then serves mclahe_backward or
 * mclahe_backward_batch), on `branches` (1..16) parallel branches forked from
 * `stream` and joined back into it, volumes dealt longest first to the least
 * loaded branch, so the passes of small volumes overlap.  Each output equals
 * mclahe_forward's bit for bit.  Nothing is cached between calls (the
 * pointers may change every call).  No counterpart in the paper.
 *   d_in, d_out, d_ws   host arrays of n_vol device pointers (outputs and
 *                 workspaces pairwise distinct, no output another volume's
 *                 input; workspaces of ws_bytes each).
 *   d_clip        nullable device float [n_vol] clip limits (NULL: the plan's).
 * Argument errors return before any launch.  The library's branch streams are
 * shared by the process: concurrent calls from several host threads are
 * serialised on the host.
 */
MCLAHE_API mclahe_status mclahe_forward_batch(mclahe_plan_t plan, int n_vol, const float *const *d_in,
                                              float *const *d_out, void *const *d_ws, size_t ws_bytes,
                                              const float *d_clip, mclahe_stream_t stream, int branches);

/*
 * mclahe_backward_batch -- dL/dclip_limit of n_vol forward calls of one plan
 * (the gather form of mclahe_backward, d_grad_lut NULL), in three launches
 * per 32 volumes instead of three per volume, so a batch of small volumes
 * fills the GPU.  Volume v's result equals mclahe_backward's for it bit for
 * bit.  No counterpart in the paper.
 *   d_in, d_grad_out, d_ws   host arrays of n_vol device pointers: each
 *                 volume's input, upstream gradient and the workspace of its
 *                 forward call (ws_bytes each, pairwise distinct).
 *   d_clip        nullable device float [n_vol]: the clip limits the forward
 *                 calls read (NULL: the plan's).
 *   d_grad_clip   device float [n_vol]: receives dL/dclip_limit per volume.
 * Argument errors (a null or misaligned pointer, a small workspace, a shared
 * workspace) return before any launch.
 */
MCLAHE_API mclahe_status mclahe_backward_batch(mclahe_plan_t plan, int n_vol, const float *const *d_in,
                                               const float *const *d_grad_out, void *const *d_ws,
                                               size_t ws_bytes, const float *d_clip,
                                               float *d_grad_clip, mclahe_stream_t stream);

/*
 * mclahe_batch -- Algorithm 1 on n_vol independent volumes of possibly
 * different shapes, dimensionalities and parameters (no counterpart in the
 * paper).  Each phase runs as one persistent launch over a work list that
 * spans all volumes.  With use_graph != 0 the launches are captured once into
 * a CUDA graph, cached by the library per (plans, pointers) for the process,
 * and replayed on later calls with the same plans and pointers; destroying
 * any of the plans drops the graphs that use it.
 *   plans     n_vol plans.
 *   d_in      host array of n_vol device input pointers.
 *   d_out     host array of n_vol device output pointers.
 *   d_ws      device workspace of ws_bytes >= mclahe_batch_workspace_bytes().
 *   d_clip    nullable device float [n_vol] clip limits.
 */
MCLAHE_API mclahe_status mclahe_batch(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                           float *const *d_out, void *d_ws, size_t ws_bytes, const float *d_clip,
                           mclahe_stream_t stream, int use_graph);

/* Workspace bytes mclahe_batch needs for these plans. */
MCLAHE_API size_t mclahe_batch_workspace_bytes(int n_vol, const mclahe_plan_t *plans);

/*
 * mclahe_batch_concurrent -- the same batch as mclahe_batch (same arguments and
 * workspace), run as every volume's own forward pass -- its plan's launch
 * shapes and walks, so each output equals mclahe_forward's bit for bit -- on
 * `branches` (1..16) parallel branches forked from `stream` and joined back
 * into it, the volumes dealt longest first to the least loaded branch.  Small
 * volumes and the tails of passes then overlap instead of running one after
 * another.  With use_graph != 0 the whole fork-join is captured once per
 * (plans, pointers, branches) into a cached CUDA graph and replayed.  No
 * counterpart in the paper.  Returns as mclahe_batch.
 */
MCLAHE_API mclahe_status mclahe_batch_concurrent(int n_vol, const mclahe_plan_t *plans,
                                                 const float *const *d_in, float *const *d_out,
                                                 void *d_ws, size_t ws_bytes, const float *d_clip,
                                                 mclahe_stream_t stream, int branches, int use_graph);

/*
 * mclahe_batch_set_wait -- the bounded waits of mclahe_batch's persistent
 * launches (no counterpart in the paper; failure detection).  A tile that
 * depends on another phase of its volume polls that volume's ready counter;
 * after max_polls polls (with a growing back-off of up to about 1 us each) it
 * gives up, records MCLAHE_ERR_TIMEOUT in the batch status word (read back by
 * mclahe_sync_status on the batch workspace) and every later wait of the
 * launch returns at once, so the launch always ends.  The results of a launch
 * that gave up are undefined.
 *   max_polls    polls before a wait gives up; 0 restores the default (2^22).
 *   unreachable  0 in normal use.  Non-zero raises every wait's target above
 *                any value the counter can reach, so that the first wait gives
 *                up after max_polls polls: this tests the timeout path without
 *                faulting or hanging the device.
 * Host-side setting for the process, applied to mclahe_batch calls made after
 * it (a cached batch graph records the setting it was captured with).  Always
 * returns MCLAHE_OK.
 */
MCLAHE_API mclahe_status mclahe_batch_set_wait(uint32_t max_polls, int unreachable);

/*
 * mclahe_autotune -- time the candidate launch shapes of the plan's passes on
 * the given buffers (which it overwrites) and keep the fastest in the plan.
 * Results are cached per (D, kernel size, n_bins, range mode) for the process.
 * Synchronises the stream.
 */
MCLAHE_API mclahe_status mclahe_autotune(mclahe_plan_t plan, const float *d_in, float *d_out, void *d_ws,
                              size_t ws_bytes, mclahe_stream_t stream);

/*
 * mclahe_plan_set_shapes -- set the plan's launch shapes explicitly (host
 * only; no CUDA call), e.g. shapes a previous process's mclahe_autotune picked
 * (read back with mclahe_plan_query).  No counterpart in the paper: shapes
 * change how the work is split, never the result.
 *   hist_group    kernels along the last dim per histogram work item, 1..n_last.
 *   hist_cluster  CTAs per work item (a cluster): 1, 2, 4 or 8; 1 if hist_shares > 0.
 *   hist_copies   lane copies of the shared-memory histograms: 1, 2, 4, ..., 32.
 *   hist_shares   0: cluster form; 1..4096: flat form with that many shares per item.
 *   hist_walk     0: per-thread cp.async row ring; 1: TMA box tiles (2- to 4-D volumes
 *                 whose last extent is a multiple of 4, footprint rows of at most 256
 *                 elements per tile); 2: per-thread loads into registers (no row buffer
 *                 in shared memory); 3: the kernel's footprint staged whole in the
 *                 shared memory of its cluster (hist_group 1, hist_shares 0, 256
 *                 threads, where it fits).
 *   hist_threads  threads per histogram CTA: 256, or 512 for 4-D volumes.
 *   map_chunks    CTAs per inter-kernel cell in the mapping pass, 1..64.
 *   map_tma       0: per-thread loads and stores; 1: TMA box tiles (3- and 4-D volumes
 *                 whose last dim and cell rows start on 16-byte boundaries only).
 *   map_flat      0: one CTA per chunk of a cell; 1: map_chunks row shares per cell dealt
 *                 out in order to a persistent grid (map_tma = 0 only).
 * Returns MCLAHE_ERR_INVALID_ARG (plan unchanged) for values outside these
 * ranges, a histogram CTA above 220 KiB of shared memory, or hist_walk = 1 or
 * map_tma = 1 on a geometry that does not allow it.  Sets tuned = 2.
 */
MCLAHE_API mclahe_status mclahe_plan_set_shapes(mclahe_plan_t plan, int32_t hist_group,
                                                int32_t hist_cluster, int32_t hist_copies,
                                                int32_t hist_shares, int32_t hist_walk,
                                                int32_t hist_threads, int32_t map_chunks,
                                                int32_t map_tma, int32_t map_flat);

/*
 * mclahe_plan_set_range_pass -- where an adaptive plan's per-kernel ranges
 * (Sec. III.D) are taken (host only; no counterpart in the paper).
 *   separate  1: one streaming sweep over the volume in memory order
 *             (MCLAHE_PASS_RANGE) leaves every kernel's min and max, and the
 *             histogram pass reads them (the cluster form with walks 0-2; the
 *             volume is then read from L2 by the histogram pass when it fits
 *             there); 0: each histogram work item sweeps its footprint for its
 *             range before binning it.
 * The result is the same either way.  Returns MCLAHE_ERR_INVALID_ARG for a
 * value other than 0 or 1, and MCLAHE_ERR_UNSUPPORTED for 1 on a plan whose
 * range is global, whose last extent is not a multiple of 4, or whose keys (8
 * bytes per kernel) and quad table (4 bytes per 4 elements of the last extent)
 * exceed 48 KiB.  Sets tuned = 2.
 */
MCLAHE_API mclahe_status mclahe_plan_set_range_pass(mclahe_plan_t plan, int32_t separate);

/* Size of the library's built-in scratch array used by mclahe_forward_noalloc. */
#define MCLAHE_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * mclahe_forward_noalloc -- mclahe_forward for callers that cannot allocate
 * device memory.  The paper has no counterpart; it exists because some callers
 * cannot provide the workspace mclahe_forward needs: plugin or custom-operator
 * interfaces that pass only input and output buffers, code running where an
 * allocation is forbidden or would break a fixed memory budget, and foreign
 * callers without a CUDA allocator.
 *   d_in, d_out, d_clip, stream   as for mclahe_forward.
 * The workspace comes from one array of MCLAHE_NOALLOC_SCRATCH_BYTES built into
 * the library, which every GPU that uses the library keeps until the process
 * exits.  This call allocates nothing.  Every call looks up the array's device
 * address on the current device (a host-side lookup, so a reset device context
 * is picked up); the first call on a device may load the library's device code,
 * so make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (the parts that must start at zero are
 * cleared by every call), so calls that overlap on the GPU race with each other;
 * run them on one stream or otherwise one after another.
 * Errors found by device code (a bounded wait that gave up) are recorded in the
 * status word of the built-in array, like mclahe_forward's in its workspace;
 * read and clear it with mclahe_noalloc_sync_status.
 * Returns MCLAHE_ERR_UNSUPPORTED when the plan's forward workspace (the offset
 * ws_scratch of mclahe_plan_info) exceeds MCLAHE_NOALLOC_SCRATCH_BYTES,
 * MCLAHE_ERR_INVALID_ARG for NULL, aliased or misaligned pointers, and
 * MCLAHE_ERR_CUDA if the address lookup or a launch fails.
 */
MCLAHE_API mclahe_status mclahe_forward_noalloc(mclahe_plan_t plan, const float *d_in, float *d_out,
                                                const float *d_clip, mclahe_stream_t stream);

/* mclahe_noalloc_sync_status -- mclahe_sync_status for the built-in array of
 * mclahe_forward_noalloc on the current device (no counterpart in the paper):
 * synchronise `stream`, then read and clear the array's status word.  Allocates
 * nothing.  Returns MCLAHE_OK, the error device code recorded, or
 * MCLAHE_ERR_CUDA if the lookup or the copy fails. */
MCLAHE_API mclahe_status mclahe_noalloc_sync_status(mclahe_stream_t stream);

/*
 * mclahe_metrics -- the contrast metrics the paper reports for its results
 * (Sec. II; Tables I and II of Sec. IV), on the device.  The paper does not
 * print their formulas; this library's readings:
 *   every volume is normalised to [0, 1] by its own min and max (a constant
 *   volume becomes 0);
 *   d_out[0] = mean, d_out[1] = standard deviation (population, 1/n) of x;
 *   d_out[2] = Shannon entropy in bits of x's 256-bin grey-level histogram
 *              over its own [min, max] (bins by the fp32 quantiser of the
 *              histogram pass);
 *   d_out[3] = MSE = mean((x^ - ref^)^2), d_out[4] = PSNR = 10 log10(peak^2 /
 *              MSE) dB with peak = 2^23, the peak that every (MSE, PSNR) pair
 *              of Tables I-II implies (NaN for both when d_ref is NULL).
 *   d_x, d_ref  device float32 volumes of n elements (d_ref nullable), 16-byte
 *               aligned, distinct.
 *   d_ws        device workspace of ws_bytes >= mclahe_metrics_workspace_bytes(n),
 *               256-byte aligned (cleared by the call).
 *   d_out       device double[5], 8-byte aligned.
 * Sums are compensated fp32 per thread and fp64 across threads in a fixed
 * order, so the result depends only on the inputs.  Does not synchronise.
 * Returns MCLAHE_OK, MCLAHE_ERR_INVALID_ARG, MCLAHE_ERR_WORKSPACE, MCLAHE_ERR_CUDA.
 */
MCLAHE_API mclahe_status mclahe_metrics(const float *d_x, const float *d_ref, int64_t n, void *d_ws,
                                        size_t ws_bytes, double *d_out, mclahe_stream_t stream);

/* Workspace bytes of mclahe_metrics for n elements (0 for n < 1). */
MCLAHE_API size_t mclahe_metrics_workspace_bytes(int64_t n);

/*
 * Pre-filters the paper applies before MCLAHE: a Gaussian (Sec. IV.A, the
 * photoemission data, standard deviations 0.7, 0.9 and 1.3 along momenta,
 * energy and time) and a median filter (Sec. IV.B, the fluorescence data,
 * window (2, 2, 2, 1)).  The paper leaves boundary, truncation and the median
 * of an even window open; readings (scipy.ndimage's conventions): the
 * edge-inclusive mirror boundary of MCLAHE's padding (Sec. III.B), reflected
 * as often as needed; Gaussian radius r = floor(4 sigma + 0.5).
 * Volumes: device float32, C order, 1 <= ndim <= 4, every extent >= 1.
 *
 * mclahe_gaussian_weights -- host only (no CUDA call): the 2r + 1 fp32 weights
 * of one dimension, exp(-k^2 / (2 sigma^2)) for k = -r..r normalised in double
 * and rounded to fp32, into w[capacity]; *radius = r.  MCLAHE_ERR_UNSUPPORTED
 * for r > 64.
 *
 * mclahe_filter_gaussian -- separable Gaussian of d_in into d_out, dimension 0
 * first; sigma[ndim] >= 0 (0 leaves a dimension as it is).  Each output is the
 * fp32 sum over the taps k = -r..r, in that order, of fp32(w_k * x) with every
 * product and sum rounded to nearest, so the result is one exact function of
 * the input.  d_tmp (device, n floats) is needed when two or more dimensions
 * are filtered; no buffer may alias another.
 *
 * mclahe_filter_median -- median filter of d_in into d_out: window
 * [x - floor(k/2), x - floor(k/2) + k - 1] along each dimension (size[ndim],
 * at most 32 voxels in all), the value of rank floor(n/2) (0-based) of the
 * window's n values (the upper median when n is even).
 *
 * None synchronises; argument errors return MCLAHE_ERR_INVALID_ARG without
 * touching the device, a failed launch MCLAHE_ERR_CUDA.
 */
MCLAHE_API mclahe_status mclahe_gaussian_weights(float sigma, float *w, int capacity, int *radius);
MCLAHE_API mclahe_status mclahe_filter_gaussian(const float *d_in, float *d_out, float *d_tmp, int ndim,
                                                const int64_t *shape, const float *sigma,
                                                mclahe_stream_t stream);
MCLAHE_API mclahe_status mclahe_filter_median(const float *d_in, float *d_out, int ndim, const int64_t *shape,
                                              const int32_t *size, mclahe_stream_t stream);

/* Synchronise `stream`, then read and clear the device status word of the
 * workspace.  Returns MCLAHE_OK or the error device code recorded. */
MCLAHE_API mclahe_status mclahe_sync_status(void *d_ws, mclahe_stream_t stream);

/* Static description of a status code. */
MCLAHE_API const char *mclahe_status_string(mclahe_status status);

/* Library version, MAJOR * 10000 + MINOR * 100 + PATCH. */
MCLAHE_API int mclahe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MCLAHE_H */
