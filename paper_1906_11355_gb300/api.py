"""High-level PyTorch front end of the MCLAHE library.

``MCLAHE`` holds a plan and its device workspace and runs the forward pass on
CUDA tensors through the C ABI; ``mclahe`` is the one-call form.  PyTorch
provides device memory and streams only.
"""
from __future__ import annotations

import torch

from . import _native as nat


class MCLAHE:
    """Plan + workspace for one volume shape (Algorithm 1 of arXiv:1906.11355).

    shape, kernel_size: per-dimension extents (1..4 dims, 1 <= b <= s).
    n_bins: histogram bins (2..4096).  clip_limit: [0, 1], T = clip_limit * V.
    adaptive: per-kernel histogram range (Sec. III.D) instead of a global one.
    global_range: optional (lo, hi) for the global range (else the data's).
    """

    def __init__(self, shape, kernel_size, n_bins=256, clip_limit=0.01, adaptive=False,
                 global_range=None, device="cuda"):
        self.shape = tuple(int(s) for s in shape)
        self.kernel_size = tuple(int(b) for b in kernel_size)
        self.n_bins = int(n_bins)
        self.clip_limit = float(clip_limit)
        self.adaptive = bool(adaptive)
        mode = nat.MCLAHE_RANGE_ADAPTIVE if adaptive else nat.MCLAHE_RANGE_GLOBAL
        self.plan = nat.mclahe_plan(self.shape, self.kernel_size, self.n_bins, self.clip_limit,
                                    mode, global_range)
        self.info = nat.mclahe_plan_query(self.plan)
        self.device = torch.device(device)
        self.ws_bytes = nat.mclahe_workspace_bytes(self.plan)
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=self.device)

    @property
    def n_kernels(self):
        return int(self.info["n_kernels"])

    def _check_volume(self, x, integers=False):
        ok = (torch.float32,) + ((torch.uint8,) + ((torch.uint16,) if hasattr(torch, "uint16") else ())
                                 if integers else ())
        if x.device.type != "cuda" or x.dtype not in ok or not x.is_contiguous():
            raise ValueError("expected a contiguous " + ("float32, uint16 or uint8" if integers else "float32")
                             + " CUDA tensor")
        if tuple(x.shape) != self.shape:
            raise ValueError(f"expected shape {self.shape}, got {tuple(x.shape)}")

    def forward(self, x, out=None, clip=None, stream=None, graph=False):
        """Run Algorithm 1 on x; returns out (float32, allocated if not given).

        x: float32, or uint16 / uint8 (intensities are the integers; mclahe_forward_typed).
        clip: optional 1-element float32 CUDA tensor overriding the clip limit.
        graph: replay a CUDA graph cached per (x, out, clip) (mclahe_forward_graph;
        float32 volumes)."""
        self._check_volume(x, integers=True)
        if out is None:
            out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        if x.dtype != torch.float32:
            nat.mclahe_forward_typed(self.plan, nat.dtype_code(x), x, out, self.ws, self.ws_bytes, clip,
                                     stream)
            return out
        fwd = nat.mclahe_forward_graph if graph else nat.mclahe_forward
        fwd(self.plan, x, out, self.ws, self.ws_bytes, clip, stream)
        return out

    __call__ = forward

    def forward_host(self, xs, outs=None, clip=None, stream=None):
        """Run Algorithm 1 on volumes held in host memory (mclahe_forward_host):
        xs is a list of CPU tensors of the plan's shape (float32, uint16 or
        uint8, all the same dtype; page-locked memory lets the copies overlap
        the kernels).  Returns the float32 CPU outputs (`outs`, or new
        page-locked tensors); they are complete once `stream` (default: the
        current stream) has reached this call's end.  Two device slots are kept
        on the object for later calls."""
        if not xs:
            return [] if outs is None else outs
        dt = xs[0].dtype
        for x in xs:
            if x.device.type != "cpu" or x.dtype != dt or not x.is_contiguous() or tuple(x.shape) != self.shape:
                raise ValueError("expected contiguous CPU tensors of one dtype and the plan's shape")
        if outs is None:
            outs = [torch.empty(self.shape, dtype=torch.float32).pin_memory() for _ in xs]
        if len(outs) != len(xs) or any(o.device.type != "cpu" or o.dtype != torch.float32 or
                                       not o.is_contiguous() or tuple(o.shape) != self.shape for o in outs):
            raise ValueError("outs: contiguous float32 CPU tensors of the plan's shape, one per input")
        key = (dt, str(self.device))
        slots = getattr(self, "_host_slots", None)
        if slots is None or slots[0] != key:
            d_in = [torch.empty(self.shape, dtype=dt, device=self.device) for _ in range(2)]
            d_out = [torch.empty(self.shape, dtype=torch.float32, device=self.device) for _ in range(2)]
            d_ws = [torch.zeros(self.ws_bytes, dtype=torch.uint8, device=self.device) for _ in range(2)]
            slots = (key, d_in, d_out, d_ws)
            self._host_slots = slots
        _, d_in, d_out, d_ws = slots
        nat.mclahe_forward_host(self.plan, nat.dtype_code(xs[0]), xs, outs, d_in, d_out, d_ws, self.ws_bytes,
                                clip, stream)
        return outs

    def autotune(self, x, out=None, stream=None):
        """Pick launch shapes by timing candidates on x (overwrites out)."""
        self._check_volume(x)
        if out is None:
            out = torch.empty_like(x)
        nat.mclahe_autotune(self.plan, x, out, self.ws, self.ws_bytes, stream)

    def shapes(self):
        """The plan's launch shapes (to reuse them with set_shapes)."""
        info = nat.mclahe_plan_query(self.plan)
        return {k: int(info[k]) for k in ("hist_group", "hist_cluster", "hist_copies",
                                          "hist_shares", "hist_walk", "hist_threads", "map_chunks",
                                          "map_tma", "map_flat", "range_pass")}

    def set_shapes(self, hist_group, hist_cluster, hist_copies, hist_shares, map_chunks,
                   map_tma=0, hist_walk=0, hist_threads=256, map_flat=0, range_pass=None):
        """Set launch shapes explicitly (e.g. from another process's autotune);
        range_pass (adaptive plans): 1 the separate streaming range sweep, 0 the
        sweep inside the histogram pass, None leaves it as it is."""
        nat.mclahe_plan_set_shapes(self.plan, hist_group, hist_cluster, hist_copies, hist_shares,
                                   map_chunks, map_tma, hist_walk, hist_threads, map_flat)
        if range_pass is not None and (range_pass or self.adaptive):
            nat.mclahe_plan_set_range_pass(self.plan, range_pass)

    # views into the workspace left by the last forward call
    def _view(self, key, count, dtype):
        off = int(self.info[key])
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype)

    def histograms(self):
        """uint32 [K, n_bins] kernel histograms (as int64 for convenience)."""
        h = self._view("ws_hist", self.n_kernels * self.n_bins, torch.int32)
        return h.view(self.n_kernels, self.n_bins).to(torch.int64) & 0xFFFFFFFF

    def tables(self):
        """float32 [K, n_bins] mapping tables (rows of table_stride floats in
        the workspace, padded past n_bins with the last entry)."""
        ls = int(self.info["table_stride"])
        return self._view("ws_lut", self.n_kernels * ls, torch.float32).view(
            self.n_kernels, ls)[:, :self.n_bins]

    def ranges(self):
        """(lo[K], scale[K]) histogram ranges of the kernels."""
        K = self.n_kernels
        return (self._view("ws_lo", K, torch.float32), self._view("ws_scale", K, torch.float32))


_cache = {}


def mclahe(x, kernel_size, n_bins=256, clip_limit=0.01, adaptive=False, global_range=None):
    """One-call MCLAHE of a contiguous float32 CUDA tensor (plan cached)."""
    key = (tuple(x.shape), tuple(kernel_size), int(n_bins), float(clip_limit), bool(adaptive),
           None if global_range is None else tuple(float(v) for v in global_range), x.device)
    op = _cache.get(key)
    if op is None:
        op = MCLAHE(x.shape, kernel_size, n_bins, clip_limit, adaptive, global_range, x.device)
        _cache[key] = op
    return op.forward(x)


class MCLAHEBatch:
    """Many volumes of possibly different shapes, dimensionalities and
    parameters in one call (mclahe_batch: one persistent launch per kind of
    volume, optionally replayed from a captured CUDA graph).

    specs: list of dicts with keys shape, kernel (kernel size), n_bins,
    clip_limit, adaptive, and optionally global_range."""

    def __init__(self, specs, device="cuda"):
        self.specs = [dict(s) for s in specs]
        self.plans = []
        for s in self.specs:
            mode = nat.MCLAHE_RANGE_ADAPTIVE if s.get("adaptive", False) else nat.MCLAHE_RANGE_GLOBAL
            self.plans.append(nat.mclahe_plan(s["shape"], s["kernel"], s.get("n_bins", 256),
                                              s.get("clip_limit", 0.01), mode, s.get("global_range")))
        self.device = torch.device(device)
        self.ws_bytes = nat.mclahe_batch_workspace_bytes(self.plans)
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def forward(self, xs, outs=None, clip=None, stream=None, use_graph=True, concurrent=0):
        """Run MCLAHE on every volume of xs (contiguous float32 CUDA tensors);
        returns outs.  clip: optional float32 CUDA tensor of one clip limit per
        volume.  With use_graph, calls with the same tensors replay one graph.
        concurrent > 0: every volume's own forward pass on that many parallel
        graph branches (mclahe_batch_concurrent) instead of the persistent
        work-list launches (mclahe_batch)."""
        if len(xs) != len(self.plans):
            raise ValueError("one input per plan expected")
        for x, s in zip(xs, self.specs):
            if x.device.type != "cuda" or x.dtype != torch.float32 or not x.is_contiguous():
                raise ValueError("expected contiguous float32 CUDA tensors")
            if tuple(x.shape) != tuple(s["shape"]):
                raise ValueError(f"expected shape {tuple(s['shape'])}, got {tuple(x.shape)}")
        if outs is None:
            outs = [torch.empty_like(x) for x in xs]
        if concurrent:
            nat.mclahe_batch_concurrent(self.plans, xs, outs, self.ws, self.ws_bytes, clip, stream, concurrent,
                                        use_graph)
        else:
            nat.mclahe_batch(self.plans, xs, outs, self.ws, self.ws_bytes, clip, stream, use_graph)
        return outs

    __call__ = forward


METRIC_NAMES = ("mean", "std", "entropy", "mse", "psnr")


def contrast_metrics(x, ref=None, stream=None):
    """Contrast metrics of a float32 CUDA volume (mclahe_metrics): mean, std,
    entropy (bits, 256 grey levels) of x normalised to [0, 1], and with ref
    the MSE and PSNR (peak 2^23) of x against ref, each normalised the same
    way.  Returns a dict of floats (synchronises)."""
    if x.dtype != torch.float32 or not x.is_contiguous() or x.device.type != "cuda":
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if ref is not None and (ref.shape != x.shape or ref.dtype != torch.float32 or not ref.is_contiguous()):
        raise ValueError("ref must be a contiguous float32 tensor of x's shape")
    n = x.numel()
    ws = torch.empty(nat.mclahe_metrics_workspace_bytes(n), dtype=torch.uint8, device=x.device)
    out = torch.empty(5, dtype=torch.float64, device=x.device)
    nat.mclahe_metrics(x, ref, n, ws, ws.numel(), out, stream)
    vals = out.cpu().tolist()
    res = dict(zip(METRIC_NAMES, vals))
    if ref is None:
        del res["mse"], res["psnr"]
    return res


def compare_frames_vs_volume(x, kernel_size, n_bins=256, clip_limit=0.02, adaptive=False, use_graph=True):
    """The paper's comparison (Sec. IV): D-dimensional CLAHE of the whole volume
    against (D-1)-dimensional CLAHE of every frame along dimension 0, with
    kernel_size[1:] for the frames (the same kernel in the frame dimensions).
    x: contiguous float32 CUDA tensor, frames along dim 0 (contiguous views; the
    frames run as one mclahe_batch call).  Returns (out_volume, out_frames,
    metrics) where metrics holds contrast_metrics of both results against x."""
    if x.dim() < 3:
        raise ValueError("need at least 3 dimensions (frames along dimension 0)")
    ks = tuple(int(b) for b in kernel_size)
    vol = MCLAHE(x.shape, ks, n_bins, clip_limit, adaptive, device=x.device)
    out_v = vol.forward(x)
    spec = dict(shape=tuple(x.shape[1:]), kernel=ks[1:], n_bins=n_bins, clip_limit=clip_limit,
                adaptive=adaptive)
    frames = MCLAHEBatch([spec] * int(x.shape[0]), device=x.device)
    out_f = torch.empty_like(x)
    frames.forward([x[t] for t in range(x.shape[0])], outs=[out_f[t] for t in range(x.shape[0])],
                   use_graph=use_graph)
    return out_v, out_f, {"volume": contrast_metrics(out_v, x), "frames": contrast_metrics(out_f, x),
                          "input": contrast_metrics(x)}


def gaussian_filter(x, sigma, out=None, stream=None):
    """Separable Gaussian pre-filter of a float32 CUDA volume (mclahe_filter_gaussian;
    one sigma per dimension, mirror boundary, radius floor(4 sigma + 0.5))."""
    if x.dtype != torch.float32 or not x.is_contiguous() or x.device.type != "cuda":
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if len(sigma) != x.dim():
        raise ValueError("one sigma per dimension")
    out = torch.empty_like(x) if out is None else out
    tmp = torch.empty_like(x) if sum(1 for s in sigma if s > 0) >= 2 else None
    nat.mclahe_filter_gaussian(x, out, tmp, tuple(x.shape), sigma, stream)
    return out


def median_filter(x, size, out=None, stream=None):
    """Median pre-filter of a float32 CUDA volume (mclahe_filter_median; window
    [x - k//2, x - k//2 + k - 1] per dimension, mirror boundary, upper median)."""
    if x.dtype != torch.float32 or not x.is_contiguous() or x.device.type != "cuda":
        raise ValueError("expected a contiguous float32 CUDA tensor")
    out = torch.empty_like(x) if out is None else out
    nat.mclahe_filter_median(x, out, tuple(x.shape), size, stream)
    return out
