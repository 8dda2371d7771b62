"""CPU oracle of Multidimensional CLAHE (arXiv:1906.11355), FP64.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import this package.  It shares
no code with the CUDA path: the arithmetic lives in ``mclahe_oracle.c`` (plain
C, compiled with gcc), and this module only marshals numpy arrays to it.

Each wrapper names the passage of the paper it follows; the C source carries
the readings of the points the paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mclahe_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmclahe_oracle.so")
_lock = threading.Lock()
_lib = None

GLOBAL = 0    # global histogram range (GHR), Sec. III.D
ADAPTIVE = 1  # adaptive histogram range (AHR), Sec. III.D


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march=native, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        lib.orc_geometry.argtypes = [ctypes.c_int, i64p, i64p, i64p, i64p, i64p, i64p]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        lib.orc_pad.argtypes = [ctypes.c_int, i64p, i64p, vp, vp]
        lib.orc_scale.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int]
        lib.orc_scale.restype = ctypes.c_float
        lib.orc_bin.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int]
        lib.orc_global_range.argtypes = [vp, ctypes.c_int64, vp, vp]
        lib.orc_clip_lut.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_double, vp, vp]
        lib.orc_map.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, vp, vp, vp, vp, vp]
        lib.orc_histograms.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_int,
                                       vp, vp, vp, vp, vp]
        lib.orc_mclahe.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_lut_backward.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_double, vp]
        lib.orc_lut_backward.restype = ctypes.c_double
        lib.orc_mclahe_backward.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, vp, vp, vp, vp, vp]
        _lib = lib
        return lib


def _i64(seq):
    arr = (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])
    return arr


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _range_arg(range_):
    if range_ is None:
        return None
    return np.asarray(range_, dtype=np.float32).reshape(2).copy()


def geometry(shape, ksize):
    """Sec. III.B, Eq. (1)-(2): padding p, p0, p1 and kernels per dim n."""
    lib = _load()
    d = len(shape)
    p, p0, p1, n = (_i64([0] * d) for _ in range(4))
    if lib.orc_geometry(d, _i64(shape), _i64(ksize), p, p0, p1, n):
        raise ValueError("invalid shape/kernel size")
    return dict(p=list(p), p0=list(p0), p1=list(p1), n=list(n))


def pad(x, ksize):
    """Algorithm 1, first two steps: symmetric padding (Sec. III.B)."""
    lib = _load()
    x = _f32(x)
    g = geometry(x.shape, ksize)
    out = np.empty([s + p for s, p in zip(x.shape, g["p"])], dtype=np.float32)
    if lib.orc_pad(x.ndim, _i64(x.shape), _i64(ksize), _ptr(x), _ptr(out)):
        raise ValueError("invalid shape/kernel size")
    return out


def scale(lo, hi, n_bins):
    """fp32 scale n_bins / (hi - lo) of a histogram range (0 if hi <= lo)."""
    return float(_load().orc_scale(lo, hi, n_bins))


def bin_index(x, lo, scale_, n_bins):
    """fp32 bin quantiser of the histogram of Algorithm 1."""
    return int(_load().orc_bin(x, lo, scale_, n_bins))


def histograms(x, ksize, n_bins, mode=GLOBAL, range_=None):
    """Per-kernel histograms of the padded volume (Algorithm 1, steps 1-5).

    Returns (hist[K, nb] uint64, lo[K] f32, scale[K] f32, n[ndim])."""
    lib = _load()
    x = _f32(x)
    g = geometry(x.shape, ksize)
    K = int(np.prod(g["n"]))
    hist = np.zeros((K, n_bins), dtype=np.uint64)
    lo = np.zeros(K, dtype=np.float32)
    sc = np.zeros(K, dtype=np.float32)
    rc = lib.orc_histograms(x.ndim, _i64(x.shape), _i64(ksize), n_bins, mode,
                            _ptr(_range_arg(range_)), _ptr(x), _ptr(hist), _ptr(lo), _ptr(sc))
    if rc:
        raise ValueError(f"orc_histograms failed ({rc})")
    return hist, lo, sc, g["n"]


def clip_lut(hist_row, V, clip_limit, with_clipped=False):
    """Algorithm 1, steps 6-8 for one kernel: clip, redistribute, CDF, normalise."""
    lib = _load()
    h = np.ascontiguousarray(hist_row, dtype=np.uint64)
    nb = h.shape[0]
    lut = np.zeros(nb, dtype=np.float64)
    hc = np.zeros(nb, dtype=np.float64)
    lib.orc_clip_lut(_ptr(h), nb, int(V), float(clip_limit), _ptr(lut), _ptr(hc))
    return (lut, hc) if with_clipped else lut


def map_volume(x, ksize, lut, lo, scale_):
    """Sec. III.C, Eq. (12)-(13): multilinear interpolation of given tables."""
    lib = _load()
    x = _f32(x)
    lut = np.ascontiguousarray(lut, dtype=np.float64)
    lo = _f32(lo)
    sc = _f32(scale_)
    out = np.empty(x.shape, dtype=np.float64)
    rc = lib.orc_map(x.ndim, _i64(x.shape), _i64(ksize), lut.shape[1], _ptr(x), _ptr(lut),
                     _ptr(lo), _ptr(sc), _ptr(out))
    if rc:
        raise ValueError("orc_map failed")
    return out


def set_threads(n):
    """Threads of the oracle's OpenMP loops (n < 1: all processors); timing only."""
    _load().orc_set_threads(int(n))


def mclahe(x, ksize, n_bins, clip_limit, mode=GLOBAL, range_=None, full=False):
    """Algorithm 1 end to end.  Returns the FP64 output (and, with full=True,
    a dict with hist, lut, lo, scale)."""
    lib = _load()
    x = _f32(x)
    g = geometry(x.shape, ksize)
    K = int(np.prod(g["n"]))
    out = np.empty(x.shape, dtype=np.float64)
    hist = np.zeros((K, n_bins), dtype=np.uint64)
    lut = np.zeros((K, n_bins), dtype=np.float64)
    lo = np.zeros(K, dtype=np.float32)
    sc = np.zeros(K, dtype=np.float32)
    rc = lib.orc_mclahe(x.ndim, _i64(x.shape), _i64(ksize), n_bins, float(clip_limit), mode,
                        _ptr(_range_arg(range_)), _ptr(x), _ptr(out), _ptr(hist), _ptr(lut),
                        _ptr(lo), _ptr(sc))
    if rc:
        raise ValueError(f"orc_mclahe failed ({rc})")
    if full:
        return out, dict(hist=hist, lut=lut, lo=lo, scale=sc, n=g["n"])
    return out


def lut_backward(hist_row, V, clip_limit, grad_lut_row):
    """Reverse mode of Algorithm 1, steps 6-8, for one kernel: dL/dT."""
    lib = _load()
    h = np.ascontiguousarray(hist_row, dtype=np.uint64)
    gl = np.ascontiguousarray(grad_lut_row, dtype=np.float64)
    return float(lib.orc_lut_backward(_ptr(h), h.shape[0], int(V), float(clip_limit), _ptr(gl)))


def mclahe_backward(x, ksize, n_bins, clip_limit, grad_out, mode=GLOBAL, range_=None):
    """Gradient of sum(grad_out * mclahe(x)) w.r.t. the tables and clip_limit.

    Returns (grad_lut[K, nb] f64, grad_clip float).  The input gradient is 0
    almost everywhere (the output is piecewise constant in the intensities)."""
    lib = _load()
    x = _f32(x)
    g = geometry(x.shape, ksize)
    K = int(np.prod(g["n"]))
    go = np.ascontiguousarray(grad_out, dtype=np.float64)
    gl = np.zeros((K, n_bins), dtype=np.float64)
    gc = np.zeros(1, dtype=np.float64)
    rc = lib.orc_mclahe_backward(x.ndim, _i64(x.shape), _i64(ksize), n_bins, float(clip_limit),
                                 mode, _ptr(_range_arg(range_)), _ptr(x), _ptr(go), _ptr(gl),
                                 _ptr(gc))
    if rc:
        raise ValueError(f"orc_mclahe_backward failed ({rc})")
    return gl, float(gc[0])
