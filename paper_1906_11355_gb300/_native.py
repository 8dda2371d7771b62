"""ctypes binding of libmclahe.so (the C ABI declared in include/mclahe.h).

Argument marshalling only: every step of MCLAHE runs in the library's CUDA
kernels.  The functions keep the C names; tensors may be passed wherever the C
function takes a device pointer (their ``data_ptr()`` is used), and streams
may be torch streams or raw handles.  There is no CPU fallback: if the library
is missing, loading fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libmclahe.so")

MCLAHE_OK = 0
MCLAHE_ERR_INVALID_ARG = 1
MCLAHE_ERR_UNSUPPORTED = 2
MCLAHE_ERR_WORKSPACE = 3
MCLAHE_ERR_CUDA = 4
MCLAHE_ERR_TIMEOUT = 5
MCLAHE_ERR_NO_MEMORY = 6
MCLAHE_ERR_DEVICE = 7

MCLAHE_RANGE_GLOBAL = 0
MCLAHE_RANGE_ADAPTIVE = 1

# every symbol include/mclahe.h declares
EXPORTS = (
    "mclahe_plan", "mclahe_plan_destroy", "mclahe_plan_query", "mclahe_workspace_bytes",
    "mclahe_forward", "mclahe_backward", "mclahe_backward_batch", "mclahe_forward_batch",
    "mclahe_forward_host", "mclahe_batch", "mclahe_batch_workspace_bytes",
    "mclahe_autotune", "mclahe_sync_status", "mclahe_status_string", "mclahe_version",
    "mclahe_forward_pass", "mclahe_pass_launches", "mclahe_forward_noalloc",
    "mclahe_plan_set_shapes", "mclahe_plan_set_range_pass", "mclahe_forward_graph",
    "mclahe_noalloc_sync_status",
    "mclahe_batch_set_wait", "mclahe_forward_typed", "mclahe_metrics",
    "mclahe_metrics_workspace_bytes", "mclahe_gaussian_weights", "mclahe_filter_gaussian",
    "mclahe_filter_median", "mclahe_forward_chunked", "mclahe_slab_rows", "mclahe_forward_slab",
    "mclahe_batch_concurrent",
)

MCLAHE_F32, MCLAHE_U16, MCLAHE_U8 = 0, 1, 2

MCLAHE_NOALLOC_SCRATCH_BYTES = 8 << 20

MCLAHE_PASS_CLEAR, MCLAHE_PASS_RANGE, MCLAHE_PASS_HIST, MCLAHE_PASS_LUT, MCLAHE_PASS_MAP = range(5)
MCLAHE_N_PASSES = 5
PASS_NAMES = ("clear", "range", "hist", "lut", "map")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("clip_limit", ctypes.c_float),
        ("shape", ctypes.c_int64 * 4), ("kernel_size", ctypes.c_int64 * 4),
        ("pad", ctypes.c_int64 * 4), ("pad_before", ctypes.c_int64 * 4),
        ("pad_after", ctypes.c_int64 * 4), ("n_kernels_dim", ctypes.c_int64 * 4),
        ("n_kernels", ctypes.c_int64), ("kernel_voxels", ctypes.c_int64),
        ("n_voxels", ctypes.c_int64), ("table_stride", ctypes.c_int64),
        ("ws_status", ctypes.c_size_t), ("ws_range_keys", ctypes.c_size_t),
        ("ws_hist", ctypes.c_size_t), ("ws_lo", ctypes.c_size_t), ("ws_scale", ctypes.c_size_t),
        ("ws_lut", ctypes.c_size_t), ("ws_scratch", ctypes.c_size_t), ("ws_bytes", ctypes.c_size_t),
        ("hist_group", ctypes.c_int32), ("hist_cluster", ctypes.c_int32),
        ("hist_copies", ctypes.c_int32), ("map_chunks", ctypes.c_int32),
        ("bwd_chunks", ctypes.c_int32), ("tuned", ctypes.c_int32),
        ("hist_shares", ctypes.c_int32), ("hist_ctas", ctypes.c_int32),
        ("map_tma", ctypes.c_int32), ("hist_walk", ctypes.c_int32),
        ("hist_threads", ctypes.c_int32), ("map_flat", ctypes.c_int32),
        ("range_pass", ctypes.c_int32),
    ]

    def as_dict(self):
        d = self.ndim
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v)[:d] if isinstance(v, ctypes.Array) else v
        return out


class MclaheError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libmclahe.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"libmclahe.so not found at {path}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        vp, sz, i32, f32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_float
        lib.mclahe_plan.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(i32), i32, f32, ctypes.c_int, vp]
        lib.mclahe_plan.restype = ctypes.c_int
        lib.mclahe_plan_destroy.argtypes = [vp]
        lib.mclahe_plan_destroy.restype = None
        lib.mclahe_plan_query.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        lib.mclahe_plan_query.restype = ctypes.c_int
        lib.mclahe_workspace_bytes.argtypes = [vp]
        lib.mclahe_workspace_bytes.restype = sz
        lib.mclahe_forward.argtypes = [vp, vp, vp, vp, sz, vp, vp]
        lib.mclahe_forward.restype = ctypes.c_int
        lib.mclahe_forward_graph.argtypes = [vp, vp, vp, vp, sz, vp, vp]
        lib.mclahe_forward_graph.restype = ctypes.c_int
        lib.mclahe_backward.argtypes = [vp, vp, vp, vp, sz, vp, vp, vp, vp]
        lib.mclahe_backward.restype = ctypes.c_int
        lib.mclahe_backward_batch.argtypes = [vp, ctypes.c_int, vp, vp, vp, sz, vp, vp, vp]
        lib.mclahe_backward_batch.restype = ctypes.c_int
        lib.mclahe_forward_batch.argtypes = [vp, ctypes.c_int, vp, vp, vp, sz, vp, vp, ctypes.c_int]
        lib.mclahe_forward_batch.restype = ctypes.c_int
        lib.mclahe_forward_host.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, sz, vp, vp]
        lib.mclahe_forward_host.restype = ctypes.c_int
        lib.mclahe_batch.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp), vp, sz, vp, vp, ctypes.c_int]
        lib.mclahe_batch.restype = ctypes.c_int
        lib.mclahe_batch_concurrent.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                ctypes.POINTER(vp), vp, sz, vp, vp, ctypes.c_int, ctypes.c_int]
        lib.mclahe_batch_concurrent.restype = ctypes.c_int
        lib.mclahe_batch_workspace_bytes.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
        lib.mclahe_batch_workspace_bytes.restype = sz
        lib.mclahe_autotune.argtypes = [vp, vp, vp, vp, sz, vp]
        lib.mclahe_autotune.restype = ctypes.c_int
        lib.mclahe_sync_status.argtypes = [vp, vp]
        lib.mclahe_sync_status.restype = ctypes.c_int
        lib.mclahe_status_string.argtypes = [ctypes.c_int]
        lib.mclahe_status_string.restype = ctypes.c_char_p
        lib.mclahe_forward_pass.argtypes = [vp, ctypes.c_int, vp, vp, vp, sz, vp, vp]
        lib.mclahe_forward_pass.restype = ctypes.c_int
        lib.mclahe_pass_launches.argtypes = [vp, ctypes.c_int]
        lib.mclahe_pass_launches.restype = ctypes.c_int
        lib.mclahe_forward_noalloc.argtypes = [vp, vp, vp, vp, vp]
        lib.mclahe_forward_noalloc.restype = ctypes.c_int
        lib.mclahe_slab_rows.argtypes = [vp, ctypes.c_int, i32, i32, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64)]
        lib.mclahe_slab_rows.restype = ctypes.c_int
        lib.mclahe_forward_slab.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, vp, vp, sz, vp, i32, i32, vp]
        lib.mclahe_forward_slab.restype = ctypes.c_int
        lib.mclahe_forward_chunked.argtypes = [vp, vp, vp, vp, sz, vp, sz, vp, vp]
        lib.mclahe_forward_chunked.restype = ctypes.c_int
        lib.mclahe_gaussian_weights.argtypes = [f32, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.mclahe_gaussian_weights.restype = ctypes.c_int
        lib.mclahe_filter_gaussian.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(f32), vp]
        lib.mclahe_filter_gaussian.restype = ctypes.c_int
        lib.mclahe_filter_median.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(i32), vp]
        lib.mclahe_filter_median.restype = ctypes.c_int
        lib.mclahe_metrics.argtypes = [vp, vp, ctypes.c_int64, vp, sz, vp, vp]
        lib.mclahe_metrics.restype = ctypes.c_int
        lib.mclahe_metrics_workspace_bytes.argtypes = [ctypes.c_int64]
        lib.mclahe_metrics_workspace_bytes.restype = sz
        lib.mclahe_forward_typed.argtypes = [vp, ctypes.c_int, vp, vp, vp, sz, vp, vp]
        lib.mclahe_forward_typed.restype = ctypes.c_int
        lib.mclahe_noalloc_sync_status.argtypes = [vp]
        lib.mclahe_noalloc_sync_status.restype = ctypes.c_int
        lib.mclahe_batch_set_wait.argtypes = [ctypes.c_uint32, ctypes.c_int]
        lib.mclahe_batch_set_wait.restype = ctypes.c_int
        lib.mclahe_plan_set_shapes.argtypes = [vp] + [ctypes.c_int32] * 9
        lib.mclahe_plan_set_shapes.restype = ctypes.c_int
        lib.mclahe_plan_set_range_pass.argtypes = [vp, ctypes.c_int32]
        lib.mclahe_plan_set_range_pass.restype = ctypes.c_int
        lib.mclahe_version.argtypes = []
        lib.mclahe_version.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(x):
    """Device (or host) address of a tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status, where):
    if status != MCLAHE_OK:
        raise MclaheError(status, where)


def status_string(status: int) -> str:
    return load().mclahe_status_string(int(status)).decode()


def mclahe_status_string(status: int) -> str:
    return status_string(status)


def mclahe_version() -> int:
    return int(load().mclahe_version())


class Plan:
    """Owns an mclahe_plan_t; destroyed with the object."""

    def __init__(self, handle, lib):
        self.handle = handle
        self._lib = lib

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            self._lib.mclahe_plan_destroy(h)

    @property
    def _as_parameter_(self):
        return self.handle


def mclahe_plan(shape, kernel_size, n_bins, clip_limit, mode=MCLAHE_RANGE_GLOBAL,
                global_range=None) -> Plan:
    """mclahe_plan: validate parameters and build a host-side plan."""
    lib = load()
    d = len(shape)
    h = ctypes.c_void_p()
    sh = (ctypes.c_int64 * d)(*[int(v) for v in shape])
    ks = (ctypes.c_int32 * len(kernel_size))(*[int(v) for v in kernel_size])
    if len(kernel_size) != d:
        raise MclaheError(MCLAHE_ERR_INVALID_ARG, "mclahe_plan")
    rng = None if global_range is None else (ctypes.c_float * 2)(*[float(v) for v in global_range])
    st = lib.mclahe_plan(ctypes.byref(h), d, sh, ks, int(n_bins), float(clip_limit), int(mode),
                         ctypes.cast(rng, ctypes.c_void_p) if rng is not None else None)
    _check(st, "mclahe_plan")
    return Plan(h.value, lib)


def mclahe_plan_query(plan) -> dict:
    info = PlanInfo()
    _check(load().mclahe_plan_query(plan.handle, ctypes.byref(info)), "mclahe_plan_query")
    return info.as_dict()


def mclahe_plan_set_shapes(plan, hist_group, hist_cluster, hist_copies, hist_shares, map_chunks,
                           map_tma=0, hist_walk=0, hist_threads=256, map_flat=0):
    _check(load().mclahe_plan_set_shapes(plan.handle, int(hist_group), int(hist_cluster),
                                         int(hist_copies), int(hist_shares), int(hist_walk),
                                         int(hist_threads), int(map_chunks), int(map_tma),
                                         int(map_flat)),
           "mclahe_plan_set_shapes")


def mclahe_plan_set_range_pass(plan, separate):
    _check(load().mclahe_plan_set_range_pass(plan.handle, int(separate)), "mclahe_plan_set_range_pass")


def mclahe_workspace_bytes(plan) -> int:
    return int(load().mclahe_workspace_bytes(plan.handle))


def mclahe_forward(plan, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None):
    st = load().mclahe_forward(plan.handle, _ptr(d_in), _ptr(d_out), _ptr(d_ws), int(ws_bytes),
                               _ptr(d_clip), _stream(stream))
    _check(st, "mclahe_forward")


def mclahe_forward_graph(plan, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None):
    st = load().mclahe_forward_graph(plan.handle, _ptr(d_in), _ptr(d_out), _ptr(d_ws), int(ws_bytes),
                                     _ptr(d_clip), _stream(stream))
    _check(st, "mclahe_forward_graph")


def dtype_code(t) -> int:
    """mclahe_dtype of a torch tensor (float32, uint16 or uint8)."""
    import torch

    codes = {torch.float32: MCLAHE_F32, torch.uint8: MCLAHE_U8}
    if hasattr(torch, "uint16"):
        codes[torch.uint16] = MCLAHE_U16
    if t.dtype not in codes:
        raise MclaheError(MCLAHE_ERR_INVALID_ARG, f"unsupported input dtype {t.dtype}")
    return codes[t.dtype]


def mclahe_forward_typed(plan, dtype, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None):
    """Forward pass of a float32, uint16 or uint8 volume (dtype: MCLAHE_F32/U16/U8)."""
    st = load().mclahe_forward_typed(plan.handle, int(dtype), _ptr(d_in), _ptr(d_out), _ptr(d_ws),
                                     int(ws_bytes), _ptr(d_clip), _stream(stream))
    _check(st, "mclahe_forward_typed")


def mclahe_metrics_workspace_bytes(n) -> int:
    return int(load().mclahe_metrics_workspace_bytes(int(n)))


def mclahe_metrics(d_x, d_ref, n, d_ws, ws_bytes, d_out, stream=None):
    """Contrast metrics of x (and MSE/PSNR against ref) into device double[5]."""
    st = load().mclahe_metrics(_ptr(d_x), _ptr(d_ref), int(n), _ptr(d_ws), int(ws_bytes), _ptr(d_out),
                               _stream(stream))
    _check(st, "mclahe_metrics")


def mclahe_filter_gaussian(d_in, d_out, d_tmp, shape, sigma, stream=None):
    """Separable Gaussian pre-filter (device float32 volumes)."""
    d = len(shape)
    sh = (ctypes.c_int64 * d)(*[int(v) for v in shape])
    sg = (ctypes.c_float * d)(*[float(v) for v in sigma])
    _check(load().mclahe_filter_gaussian(_ptr(d_in), _ptr(d_out), _ptr(d_tmp), d, sh, sg, _stream(stream)),
           "mclahe_filter_gaussian")


def mclahe_filter_median(d_in, d_out, shape, size, stream=None):
    """Median pre-filter (device float32 volumes)."""
    d = len(shape)
    sh = (ctypes.c_int64 * d)(*[int(v) for v in shape])
    sz = (ctypes.c_int32 * d)(*[int(v) for v in size])
    _check(load().mclahe_filter_median(_ptr(d_in), _ptr(d_out), d, sh, sz, _stream(stream)),
           "mclahe_filter_median")


def mclahe_slab_rows(plan, pass_, row0, row1):
    """Original rows (first, end) along dimension 0 a slab needs for a pass."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().mclahe_slab_rows(plan.handle, int(pass_), int(row0), int(row1), ctypes.byref(a),
                                   ctypes.byref(b)), "mclahe_slab_rows")
    return int(a.value), int(b.value)


def mclahe_forward_slab(plan, pass_, d_slab, slab_first, d_out_slab, d_ws, ws_bytes, row0, row1,
                        d_clip=None, stream=None):
    """One pass (RANGE, HIST or MAP) on a slab of the volume along dimension 0."""
    st = load().mclahe_forward_slab(plan.handle, int(pass_), _ptr(d_slab), int(slab_first), _ptr(d_out_slab),
                                    _ptr(d_ws), int(ws_bytes), _ptr(d_clip), int(row0), int(row1),
                                    _stream(stream))
    _check(st, "mclahe_forward_slab")


def mclahe_forward_chunked(plan, h_in, h_out, d_ws, ws_bytes, d_stage, stage_bytes, d_clip=None,
                           stream=None):
    """Forward pass of a host-resident float32 volume streamed through d_stage."""
    st = load().mclahe_forward_chunked(plan.handle, _ptr(h_in), _ptr(h_out), _ptr(d_ws), int(ws_bytes),
                                       _ptr(d_stage), int(stage_bytes), _ptr(d_clip), _stream(stream))
    _check(st, "mclahe_forward_chunked")


def mclahe_forward_noalloc(plan, d_in, d_out, d_clip=None, stream=None):
    """Forward pass using the library's built-in scratch array (allocates nothing)."""
    st = load().mclahe_forward_noalloc(plan.handle, _ptr(d_in), _ptr(d_out), _ptr(d_clip),
                                       _stream(stream))
    _check(st, "mclahe_forward_noalloc")


def mclahe_noalloc_sync_status(stream=None) -> int:
    """Read and clear the status word of the built-in array of mclahe_forward_noalloc."""
    return int(load().mclahe_noalloc_sync_status(_stream(stream)))


def mclahe_forward_pass(plan, pass_, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None):
    st = load().mclahe_forward_pass(plan.handle, int(pass_), _ptr(d_in), _ptr(d_out), _ptr(d_ws),
                                    int(ws_bytes), _ptr(d_clip), _stream(stream))
    _check(st, "mclahe_forward_pass")


def mclahe_pass_launches(plan, pass_) -> int:
    return int(load().mclahe_pass_launches(plan.handle, int(pass_)))


def mclahe_backward(plan, d_in, d_grad_out, d_ws, ws_bytes, d_clip, d_grad_lut, d_grad_clip,
                    stream=None):
    st = load().mclahe_backward(plan.handle, _ptr(d_in), _ptr(d_grad_out), _ptr(d_ws),
                                int(ws_bytes), _ptr(d_clip), _ptr(d_grad_lut), _ptr(d_grad_clip),
                                _stream(stream))
    _check(st, "mclahe_backward")


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))(*[_ptr(x) for x in items])
    return arr


def mclahe_forward_host(plan, dtype, h_in, h_out, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None):
    """mclahe_forward_typed on len(h_in) host-resident volumes through two
    device slots (d_in, d_out, d_ws: two buffers each), copies overlapping."""
    n = len(h_in)
    if len(h_out) != n or len(d_in) != 2 or len(d_out) != 2 or len(d_ws) != 2:
        raise ValueError("h_in and h_out of equal length; two device slots")
    st = load().mclahe_forward_host(plan.handle, int(dtype), n, _ptr_array(h_in), _ptr_array(h_out),
                                    _ptr_array(d_in), _ptr_array(d_out), _ptr_array(d_ws), int(ws_bytes),
                                    _ptr(d_clip), _stream(stream))
    _check(st, "mclahe_forward_host")


def mclahe_forward_batch(plan, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None, branches=8):
    """mclahe_forward on len(d_in) volumes of one plan on parallel branches
    (lists of tensors or pointers; d_clip: n_vol clip limits or None)."""
    n = len(d_in)
    if len(d_out) != n or len(d_ws) != n:
        raise ValueError("d_in, d_out and d_ws must have the same length")
    st = load().mclahe_forward_batch(plan.handle, n, _ptr_array(d_in), _ptr_array(d_out), _ptr_array(d_ws),
                                     int(ws_bytes), _ptr(d_clip), _stream(stream), int(branches))
    _check(st, "mclahe_forward_batch")


def mclahe_backward_batch(plan, d_in, d_grad_out, d_ws, ws_bytes, d_clip, d_grad_clip, stream=None):
    """dL/dclip of len(d_in) forward calls of one plan (lists of tensors or
    pointers; d_clip: n_vol clip limits or None; d_grad_clip: n_vol floats)."""
    n = len(d_in)
    if len(d_grad_out) != n or len(d_ws) != n:
        raise ValueError("d_in, d_grad_out and d_ws must have the same length")
    st = load().mclahe_backward_batch(plan.handle, n, _ptr_array(d_in), _ptr_array(d_grad_out),
                                      _ptr_array(d_ws), int(ws_bytes), _ptr(d_clip), _ptr(d_grad_clip),
                                      _stream(stream))
    _check(st, "mclahe_backward_batch")


def mclahe_batch_workspace_bytes(plans) -> int:
    hs = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    return int(load().mclahe_batch_workspace_bytes(len(plans), hs))


def mclahe_batch(plans, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None, use_graph=True):
    n = len(plans)
    hs = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    st = load().mclahe_batch(n, hs, _ptr_array(d_in), _ptr_array(d_out), _ptr(d_ws), int(ws_bytes),
                             _ptr(d_clip), _stream(stream), 1 if use_graph else 0)
    _check(st, "mclahe_batch")


def mclahe_batch_set_wait(max_polls=0, unreachable=False):
    """Polls before a batch wait gives up (0: default); unreachable=True raises every
    wait target out of reach (tests of the timeout path only)."""
    _check(load().mclahe_batch_set_wait(int(max_polls), 1 if unreachable else 0),
           "mclahe_batch_set_wait")


def mclahe_batch_concurrent(plans, d_in, d_out, d_ws, ws_bytes, d_clip=None, stream=None, branches=8,
                            use_graph=True):
    n = len(plans)
    hs = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    st = load().mclahe_batch_concurrent(n, hs, _ptr_array(d_in), _ptr_array(d_out), _ptr(d_ws),
                                        int(ws_bytes), _ptr(d_clip), _stream(stream), int(branches),
                                        1 if use_graph else 0)
    _check(st, "mclahe_batch_concurrent")


def mclahe_autotune(plan, d_in, d_out, d_ws, ws_bytes, stream=None):
    st = load().mclahe_autotune(plan.handle, _ptr(d_in), _ptr(d_out), _ptr(d_ws), int(ws_bytes),
                                _stream(stream))
    _check(st, "mclahe_autotune")


def mclahe_sync_status(d_ws, stream=None) -> int:
    return int(load().mclahe_sync_status(_ptr(d_ws), _stream(stream)))
