#!/usr/bin/env python3
"""Throughput of the MCLAHE hot path on GB300 (one JSON line on stdout).

A step is one full forward pass (range, histograms, tables, mapping) over one
synthetic volume already resident in HBM.  The default workload (the headline)
is the largest one-GPU configuration, the 4-D photoemission-like volume
128x128x256x32 (kernel 32x32x32x8, 512 bins, clip 0.01, global range found on
the device); the 3-D fluorescence-like stack 64x512x512 (kernel 16x64x64, 256
bins, clip 0.02, adaptive range) and the 2-D image 512x512 are measured the
same way and reported beside it.  L2 is flushed (a 256 MiB write) between
timed steps, outside the step's events.  Each pass is timed with CUDA events on
the stream that launches it; the step time is the first-to-last event span.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on this host

Under torchrun (N > 1) each rank processes its own volume (different seed) with
no data exchange (weak scaling); rank 0 prints the whole-job throughput from
the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MCLAHE Gvoxel/s & % HBM roofline; batched and fwd+bwd vs plain fwd"
DEFAULT_WORKLOAD = "4d-photoemission-128x128x256x32"
EXTRA_WORKLOADS = ("3d-fluorescence-64x512x512", "2d-smooth-512x512")
L2_FLUSH_BYTES = 256 << 20
PEAK_FALLBACK_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (context for the measured peak)

def pass_kernel(pass_name, info):
    """Kernel launched by a pass (for the roofline and the ncu launch list)."""
    flat = info["hist_shares"] > 0
    if pass_name == "range":
        if info["mode"] == 1:
            return "k_hist_flat" if flat else "k_range_kernels"
        return "k_range_global"
    mapk = "k_map_tma" if info["map_tma"] else ("k_map_flat" if info["map_flat"] else "k_map")
    histk = "k_hist_flat" if flat else ("k_hist_staged" if info["hist_walk"] == 3 else "k_hist")
    return {"hist": histk, "map": mapk}[pass_name]



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default launch shapes (mclahe_autotune is skipped)")
    ap.add_argument("--shapes", default=None,
                    help="launch shapes as JSON (the keys of MCLAHE.set_shapes) instead of autotuning")
    ap.add_argument("--no-graph", action="store_true",
                    help="time mclahe_forward instead of the graph-replayed mclahe_forward_graph")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and forward+backward forms")
    ap.add_argument("--form-steps", type=int, default=20)
    ap.add_argument("--no-extra", action="store_true",
                    help="measure only the selected workload (not the other configurations)")
    return ap.parse_args()


def dist_env():
    from paper_1906_11355_gb300.dist import dist_env as env

    return env()


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region (nvidia-smi sampled in the background)
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        def parse(line):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                return None
            try:
                return dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                            hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8])
            except ValueError:
                return None

        inside = [parse(l) for t, l in self.samples if t0 <= t <= t1]
        inside = [s for s in inside if s]
        window = "timed"
        if not inside:   # region shorter than the sampling period
            inside = [s for s in (parse(l) for _, l in self.samples) if s]
            window = "warmup+timed"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sms = sorted(s["sm"] for s in inside)
        reasons = set()
        for s in inside:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if s[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": max(s["smax"] for s in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window,
                "power_w_max": max(s["power"] for s in inside)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of each pass (HBM roofline)
# ---------------------------------------------------------------------------
def algorithmic_bytes(info, adaptive, has_range):
    """Bytes each pass must move at least: the range pass reads the input once
    (a global range not given by the caller); the histogram pass reads the
    input once and writes the histograms, tables and ranges; the mapping pass
    reads the input and writes the output (4 B per voxel each).  With the
    adaptive range the flat histogram form, and the cluster form with the
    separate streaming range sweep, have a range pass of their own, which
    reads the input once and writes every kernel's min/max keys."""
    N = info["n_voxels"]
    K = info["n_kernels"]
    nb = info["n_bins"]
    ls = info["table_stride"]
    if adaptive:
        own = info["hist_shares"] > 0 or (info.get("range_pass", 0) and info["hist_walk"] != 3)
        rng = 4 * N + 8 * K if own else 0
    else:
        rng = 0 if has_range else 4 * N
    return {
        "range": rng,
        "hist": 4 * N + 4 * K * nb + 4 * K * ls + 8 * K,
        "lut": 0,
        "map": 8 * N,
    }


def kernel_source_hash(pass_name):
    """Hash of the sources a pass's kernel is compiled from (the recorded ncu
    traffic is only reported while this matches)."""
    hist = ("k_hist.cu", "k_hist_tma.cu", "k_hist_lsu.cu", "k_hist_staged.cu", "k_hist_impl.cuh",
            "hist_impl.cuh", "hist_staged.cuh", "tma.cuh")
    files = {"range": ("k_range.cu",) + hist, "hist": hist,
             "map": ("k_map.cu", "k_map_impl.cuh", "map_impl.cuh", "tma.cuh")}[pass_name]
    h = hashlib.sha256()
    for f in files + ("mclahe_internal.cuh",):
        with open(os.path.join(ROOT, "paper_1906_11355_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# launch shapes that select the kernel variant of a pass
VARIANT_KEYS = {
    "range": ("hist_shares", "hist_walk", "hist_threads", "range_pass"),
    "hist": ("hist_group", "hist_cluster", "hist_copies", "hist_shares", "hist_walk", "hist_threads"),
    "map": ("map_chunks", "map_tma", "map_flat"),
}


def pass_variant(pass_name, info):
    return {k: int(info[k]) for k in VARIANT_KEYS[pass_name]}


def recorded_traffic(workload, pass_name, info):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source, the same kernel and the same launch shapes (else
    None)."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)[workload][pass_name]
    except Exception:
        return None
    if rec.get("source_sha") != kernel_source_hash(pass_name):
        return None
    if rec.get("kernel", "").split("<")[0] != pass_kernel(pass_name, info):
        return None
    if rec.get("shapes") != pass_variant(pass_name, info):
        return None
    return rec.get("bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on this host's cores
# ---------------------------------------------------------------------------
def oracle_rate(x, w, min_seconds=10.0):
    import numpy as np

    import oracle

    oracle.build()
    clip = float(np.float32(w["clip_limit"]))
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.mclahe(x, w["kernel"], w["n_bins"], clip, mode=int(w["adaptive"]))
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # the same oracle on one thread (a bounded sample: at least one volume, about 3 s)
    oracle.set_threads(1)
    reps1, t1 = 0, time.perf_counter()
    while True:
        oracle.mclahe(x, w["kernel"], w["n_bins"], clip, mode=int(w["adaptive"]))
        reps1 += 1
        el1 = time.perf_counter() - t1
        if el1 >= 3.0:
            break
    oracle.set_threads(0)
    single = {"value": x.size * reps1 / el1 / 1e9, "cores": 1,
              "sample": f"whole volume x{reps1} ({el1:.1f} s, FP64, one thread)"}
    return x.size * reps / el / 1e9, reps, el, cores, single


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1906_11355_gb300 import synth

    w = synth.WORKLOADS[args.workload]
    x = synth.make_volume(w["gen"], w["shape"], w["seed"])
    import numpy as np

    import oracle

    oracle.build()
    clip = float(np.float32(w["clip_limit"]))
    # bound the whole run to about two minutes: shrink the volume to a leading
    # block of whole kernels (dim 0 first, then dim 1, ...) when K full-volume
    # steps would take longer
    t0 = time.perf_counter()
    oracle.mclahe(x, w["kernel"], w["n_bins"], clip, mode=int(w["adaptive"]))
    t_full = time.perf_counter() - t0
    sample = f"the whole {args.workload} volume per step"
    budget = 120.0 / max(args.steps + args.warmup, 1)
    if t_full > budget:
        ext = list(w["shape"])
        for d in range(len(ext)):
            b = w["kernel"][d]
            frac = budget / (t_full * np.prod(ext) / np.prod(w["shape"]))
            ext[d] = max(b, int(ext[d] * frac) // b * b)
            if t_full * np.prod(ext) / np.prod(w["shape"]) <= budget:
                break
        x = np.ascontiguousarray(x[tuple(slice(0, e) for e in ext)])
        sample = (f"leading {'x'.join(str(e) for e in ext)} block (whole kernels) of the "
                  f"{args.workload} volume per step")
    for _ in range(max(args.warmup, 0)):
        oracle.mclahe(x, w["kernel"], w["n_bins"], clip, mode=int(w["adaptive"]))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.mclahe(x, w["kernel"], w["n_bins"], clip, mode=int(w["adaptive"]))
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = x.size / (ms * 1e-3) / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gvoxel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "shape": list(w["shape"]), "kernel": list(w["kernel"]),
                   "n_bins": w["n_bins"], "clip_limit": w["clip_limit"],
                   "range": "adaptive" if w["adaptive"] else "global"},
        "cpu_baseline": {"value": value, "unit": "Gvoxel/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gvoxel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# the batched and forward+backward forms, each against the plain forward
# ---------------------------------------------------------------------------
def _time_steps(fn, steps, warmup, stream, flush=None):
    """Mean ms of fn() over `steps` calls timed with CUDA events on `stream`
    (after `warmup` calls); flush() runs between steps, outside the events."""
    import torch

    for _ in range(warmup):
        if flush is not None:
            flush()
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def measure_batched(dev, steps, warmup):
    """48 volumes of uneven shape (16 2-D, 24 3-D, 8 4-D; kernel 1/8 of each
    extent, 256 or 512 bins) in one mclahe_batch call replayed from a CUDA
    graph, against the same volumes run one mclahe_forward after another."""
    import numpy as np
    import torch

    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE, MCLAHEBatch

    specs = synth.batch_specs()
    for s in specs:
        s["clip_limit"] = float(np.float32(s["clip_limit"]))
    xs = [synth.batch_volume_t(s, device=dev) for s in specs]
    outs = [torch.empty_like(x) for x in xs]
    voxels = sum(int(x.numel()) for x in xs)
    stream = torch.cuda.current_stream(dev)
    batch = MCLAHEBatch(specs, device=dev)
    ms_batch = _time_steps(lambda: batch.forward(xs, outs=outs, use_graph=True), steps, warmup, stream)
    ops = [MCLAHE(s["shape"], s["kernel"], s["n_bins"], s["clip_limit"], s["adaptive"], device=dev)
           for s in specs]

    def plain():
        for op, x, o in zip(ops, xs, outs):
            op.forward(x, out=o)

    ms_plain = _time_steps(plain, steps, warmup, stream)
    ms_conc = _time_steps(lambda: batch.forward(xs, outs=outs, use_graph=True, concurrent=8), steps, warmup,
                          stream)
    launches = {"plain": 0}
    from paper_1906_11355_gb300 import _native as nat

    for op in ops:
        launches["plain"] += sum(nat.mclahe_pass_launches(op.plan, p) for p in range(nat.MCLAHE_N_PASSES))
    groups = len({(len(s["shape"]), bool(s["adaptive"])) for s in specs})
    del xs, outs, batch, ops
    torch.cuda.empty_cache()
    return {"workload": "batch-48-uneven-2d3d4d", "volumes": len(specs), "voxels": voxels,
            "value": voxels / (ms_batch * 1e-3) / 1e9, "unit": "Gvoxel/s", "ms_per_step": ms_batch,
            "plain_forward_ms": ms_plain, "plain_forward_value": voxels / (ms_plain * 1e-3) / 1e9,
            "speedup_vs_plain_forward": ms_plain / ms_batch,
            "concurrent": {"call": "mclahe_batch_concurrent (8 graph branches, each volume's own forward)",
                           "ms_per_step": ms_conc, "value": voxels / (ms_conc * 1e-3) / 1e9,
                           "speedup_vs_plain_forward": ms_plain / ms_conc},
            "launches": {"batched": groups, "plain_forward": launches["plain"]},
            "data": "synthetic, drawn on the device (torch generators, seeds 1000+v)"}


def measure_fwd_bwd(dev, steps, warmup):
    """Forward + backward of 8 volumes 64x256x256 (fluorescence-like; kernel
    16x64x64, 256 bins, adaptive range) with one learnable clip limit per
    volume (U[0.005, 0.05]) and loss = mean squared error to a seeded target;
    against the forward alone.  The step is what MCLAHEBatchFunction runs: one
    mclahe_forward_batch call (the eight forwards on parallel branches), dL/dout
    of the loss (two elementwise launches over the batch), one
    mclahe_backward_batch call; the per-volume calls are timed beside it."""
    import torch

    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE

    B, shape, ks, nb = 8, (64, 256, 256), (16, 64, 64), 256
    xs = torch.stack([synth.fluorescence_t(shape, seed=2000 + v, device=dev) for v in range(B)])
    tgt = torch.stack([synth.fluorescence_t(shape, seed=3000 + v, device=dev) for v in range(B)])
    tgt /= tgt.amax(dim=(1, 2, 3), keepdim=True)
    g = torch.Generator(device="cpu")
    g.manual_seed(4)
    clips = (0.005 + 0.045 * torch.rand(B, generator=g)).to(dev)
    op = MCLAHE(shape, ks, nb, 0.02, adaptive=True, device=dev)
    wss = [torch.zeros(op.ws_bytes, dtype=torch.uint8, device=dev) for _ in range(B)]
    outs = torch.empty_like(xs)
    gouts = torch.empty_like(xs)
    gclip = torch.empty(B, dtype=torch.float32, device=dev)
    n = float(xs.numel())
    stream = torch.cuda.current_stream(dev)
    xl, ol, gl = list(xs), list(outs), list(gouts)

    def fwd():
        nat.mclahe_forward_batch(op.plan, xl, ol, wss, op.ws_bytes, clips, stream)

    def bwd():
        nat.mclahe_backward_batch(op.plan, xl, gl, wss, op.ws_bytes, clips, gclip, stream)

    def fwd_bwd():
        fwd()
        torch.sub(outs, tgt, out=gouts).mul_(2.0 / n)   # dL/d(out) of the MSE
        bwd()

    def fwd_pv():
        for v in range(B):
            nat.mclahe_forward(op.plan, xl[v], ol[v], wss[v], op.ws_bytes, clips[v:v + 1], stream)

    def bwd_pv():
        for v in range(B):
            nat.mclahe_backward(op.plan, xl[v], gl[v], wss[v], op.ws_bytes, clips[v:v + 1], None,
                                gclip[v:v + 1], stream)

    ms_fwd = _time_steps(fwd, steps, warmup, stream)
    ms_fb = _time_steps(fwd_bwd, steps, warmup, stream)
    ms_bwd = _time_steps(bwd, steps, warmup, stream)
    ms_fwd_pv = _time_steps(fwd_pv, steps, warmup, stream)
    ms_bwd_pv = _time_steps(bwd_pv, steps, warmup, stream)
    voxels = int(n)
    peak, peak_kind = measured_peak_gbs()
    bwd_bytes = 8 * voxels   # reads of the input and the upstream gradient

    def roof(ms):
        ach = bwd_bytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "algorithmic_bytes": bwd_bytes, "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "peak_kind": peak_kind}

    out = {"workload": "fwd+bwd-8x64x256x256-learnable-clip", "voxels": voxels,
           "value": voxels / (ms_fb * 1e-3) / 1e9, "unit": "Gvoxel/s", "ms_per_step": ms_fb,
           "forward_ms": ms_fwd, "forward_value": voxels / (ms_fwd * 1e-3) / 1e9,
           "fwd_bwd_over_fwd": ms_fb / ms_fwd,
           "backward_ms": ms_bwd,
           "backward_roofline": dict(roof(ms_bwd), note="one mclahe_backward_batch call (k_dtab, "
                                     "k_mapdot, k_clipsum over the 8 volumes), 8 B per voxel"),
           "per_volume_calls": {"forward_ms": ms_fwd_pv, "backward_ms": ms_bwd_pv,
                                "backward_frac": roof(ms_bwd_pv)["frac"]},
           "grad_clip_finite": bool(torch.isfinite(gclip).all().item()),
           "data": "synthetic, drawn on the device (torch generators, seeds 2000+v, targets 3000+v)"}
    del xs, tgt, wss, outs, gouts
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
SHAPE_KEYS = ("hist_group", "hist_cluster", "hist_shares", "hist_copies", "hist_walk", "hist_threads",
              "map_flat", "map_chunks", "map_tma", "range_pass", "tuned")


class Workload:
    """One workload on the device: its plan (autotuned or given shapes), input,
    output, and the step and per-pass timings."""

    def __init__(self, name, args, dev, rank, given_range=False):
        import numpy as np
        import torch

        from paper_1906_11355_gb300 import synth
        from paper_1906_11355_gb300.api import MCLAHE
        from paper_1906_11355_gb300.dist import rank_seed

        self.name = name
        self.w = w = synth.WORKLOADS[name]
        self.x_host = synth.make_volume(w["gen"], w["shape"], rank_seed(w["seed"], rank))
        rng = None
        if given_range:   # the data's own range, given to the plan (no range pass)
            rng = (float(self.x_host.min()), float(self.x_host.max()))
        self.given_range = rng
        self.op = MCLAHE(w["shape"], w["kernel"], w["n_bins"], float(np.float32(w["clip_limit"])),
                         adaptive=w["adaptive"], global_range=rng, device=dev)
        self.x = torch.from_numpy(self.x_host).to(dev)
        self.out = torch.empty_like(self.x)
        self.voxels = int(np.prod(w["shape"]))
        self.dev = dev

    def tune(self, args):
        import json as _json

        from paper_1906_11355_gb300 import _native as nat

        if args.shapes and self.name == args.workload:
            self.op.set_shapes(**_json.loads(args.shapes))
        elif not args.no_autotune:
            self.op.autotune(self.x, self.out)   # timed on this volume, outside the timed region
        self.info = nat.mclahe_plan_query(self.op.plan)
        self.shapes = {k: v for k, v in self.info.items() if k in SHAPE_KEYS}
        self.launches = {p: nat.mclahe_pass_launches(self.op.plan, p) for p in range(nat.MCLAHE_N_PASSES)}

    def step_fn(self, args, stream):
        from paper_1906_11355_gb300 import _native as nat

        fwd = nat.mclahe_forward if args.no_graph else nat.mclahe_forward_graph
        op, x, out = self.op, self.x, self.out

        def step(e0, e1):
            e0.record(stream)
            fwd(op.plan, x, out, op.ws, op.ws_bytes, None, stream)
            e1.record(stream)

        return step

    def time_passes(self, flush, stream, n):
        """Mean time of each pass (an event between passes; L2 flushed first)."""
        import torch

        from paper_1906_11355_gb300 import _native as nat

        passes = list(range(nat.MCLAHE_N_PASSES))
        bd = [[torch.cuda.Event(enable_timing=True) for _ in range(len(passes) + 1)] for _ in range(n)]
        op = self.op
        for i in range(n):
            flush.fill_(i & 0xFF)
            bd[i][0].record(stream)
            for p in passes:
                nat.mclahe_forward_pass(op.plan, p, self.x, self.out, op.ws, op.ws_bytes, None, stream)
                bd[i][p + 1].record(stream)
        torch.cuda.synchronize(self.dev)
        return {nat.PASS_NAMES[p]: sum(ev[p].elapsed_time(ev[p + 1]) for ev in bd) / n for p in passes}

    def roofline(self, pass_ms):
        from paper_1906_11355_gb300 import _native as nat

        peak, peak_kind = measured_peak_gbs()
        w = self.w
        algo = algorithmic_bytes(self.info, w["adaptive"], self.given_range is not None)
        kern = {k: v for k, v in pass_ms.items()
                if k in ("range", "hist", "map") and self.launches[nat.PASS_NAMES.index(k)] > 0}
        per_pass = {}
        for k in kern:
            ach = algo[k] / (pass_ms[k] * 1e-3) / 1e9
            per_pass[k] = {"kernel": pass_kernel(k, self.info), "variant": pass_variant(k, self.info),
                           "ms": pass_ms[k], "algorithmic_bytes": algo[k], "achieved": ach,
                           "frac": ach / peak, "traffic": recorded_traffic(self.name, k, self.info)}
        dom = max(kern, key=kern.get)
        d = per_pass[dom]
        return {"bound": "hbm", "kernel": d["kernel"], "variant": d["variant"],
                "achieved": d["achieved"], "peak": peak, "unit": "GB/s", "frac": d["frac"],
                "traffic": d["traffic"], "peak_kind": peak_kind, "algorithmic_bytes": d["algorithmic_bytes"],
                "frac_of_nominal": d["achieved"] / NOMINAL_HBM_GBS}, per_pass

    def config(self, args):
        w = self.w
        c = {"workload": self.name, "shape": list(w["shape"]), "kernel": list(w["kernel"]),
             "n_bins": w["n_bins"], "clip_limit": w["clip_limit"],
             "range": "adaptive" if w["adaptive"] else "global",
             "l2": "flushed between steps (256 MiB write outside the step events)",
             "launch_shapes": self.shapes,
             "call": "mclahe_forward" if args.no_graph else "mclahe_forward_graph",
             "voxels_per_gpu": self.voxels}
        if self.given_range is not None:
            c["range"] = "global, given to the plan (the data's own min and max; no range pass)"
        return c

    def release(self):
        import torch

        del self.x, self.out, self.op
        torch.cuda.empty_cache()


def measure_simple(wl, args, stream, flush, steps):
    """A workload beside the headline: step time (events, L2 flushed between
    steps), per-pass times and rooflines."""
    import torch

    step = wl.step_fn(args, stream)
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        step(*ev[i])
    torch.cuda.synchronize(wl.dev)
    ms_l = [a.elapsed_time(b) for a, b in ev]
    ms = sum(ms_l) / steps
    pass_ms = wl.time_passes(flush, stream, min(steps, 50))
    roof, per_pass = wl.roofline(pass_ms)
    return {"value": wl.voxels / (ms * 1e-3) / 1e9, "unit": "Gvoxel/s", "ms_per_step": ms,
            "ms_per_step_median": float(sorted(ms_l)[len(ms_l) // 2]), "steps": steps,
            "hbm_roofline_frac_whole_step": 12 * wl.voxels / (ms * 1e-3) / 1e9 / roof["peak"],
            "config": wl.config(args), "passes_ms": pass_ms, "roofline": roof,
            "roofline_per_pass": per_pass}


TYPED_WORKLOADS = (("3d-fluorescence-64x512x512", "u16"), ("4d-photoemission-128x128x256x32", "u8"))


def measure_typed(name, dtype, args, dev, stream, flush, steps):
    """A workload read in its native integer type (mclahe_forward_typed): uint16
    fluorescence counts, uint8 photoemission counts.  Launch shapes are tuned on
    the float32 volume of the same values; bytes per voxel: the element size for
    each input read (range pass under a global range, histogram, mapping) plus
    4 for the output."""
    import numpy as np
    import torch

    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE

    w = synth.WORKLOADS[name]
    if dtype == "u16":
        xi = synth.fluorescence_u16(w["shape"], seed=w["seed"])
        xd = torch.from_numpy(xi.view(np.int16)).to(dev)
        code, esize = nat.MCLAHE_U16, 2
    else:
        xf = synth.make_volume(w["gen"], w["shape"], w["seed"])
        assert xf.min() >= 0 and xf.max() <= 255 and np.array_equal(xf, np.round(xf))
        xi = xf.astype(np.uint8)
        xd = torch.from_numpy(xi).to(dev)
        code, esize = nat.MCLAHE_U8, 1
    op = MCLAHE(w["shape"], w["kernel"], w["n_bins"], float(np.float32(w["clip_limit"])),
                adaptive=w["adaptive"], device=dev)
    out = torch.empty(w["shape"], dtype=torch.float32, device=dev)
    if not args.no_autotune:
        xfl = torch.from_numpy(xi.astype(np.float32)).to(dev)
        op.autotune(xfl, out)
        del xfl
    voxels = int(np.prod(w["shape"]))

    def step(e0, e1):
        e0.record(stream)
        nat.mclahe_forward_typed(op.plan, code, xd, out, op.ws, op.ws_bytes, None, stream)
        e1.record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        step(*ev[i])
    torch.cuda.synchronize(dev)
    ms_l = [a.elapsed_time(b) for a, b in ev]
    ms = sum(ms_l) / steps
    reads = 3 if not w["adaptive"] else 2
    step_bytes = voxels * (reads * esize + 4)
    peak, peak_kind = measured_peak_gbs()
    ach = step_bytes / (ms * 1e-3) / 1e9
    res = {"value": voxels / (ms * 1e-3) / 1e9, "unit": "Gvoxel/s", "ms_per_step": ms,
           "ms_per_step_median": float(sorted(ms_l)[len(ms_l) // 2]), "steps": steps,
           "dtype": dtype, "call": "mclahe_forward_typed",
           "config": {"workload": f"{name}-{dtype}", "shape": list(w["shape"]), "kernel": list(w["kernel"]),
                      "n_bins": w["n_bins"], "clip_limit": w["clip_limit"],
                      "range": "adaptive" if w["adaptive"] else "global", "input": dtype,
                      "launch_shapes": {k: v for k, v in nat.mclahe_plan_query(op.plan).items()
                                        if k in SHAPE_KEYS}},
           "roofline_whole_step": {"bound": "hbm", "bytes_per_voxel": reads * esize + 4,
                                   "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                   "peak_kind": peak_kind}}
    del xd, out, op
    torch.cuda.empty_cache()
    return res


def run_native(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import build as nbuild
    from paper_1906_11355_gb300.dist import max_over_ranks

    nbuild.build()
    nat.load()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    wl = Workload(args.workload, args, dev, rank)
    wl.tune(args)
    op, x, out = wl.op, wl.x, wl.out
    step = wl.step_fn(args, stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize(dev)

    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.time()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                 # evict the previous step's lines from L2
        step(*events[i])
    torch.cuda.synchronize(dev)
    t1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    sampler.stop()

    step_ms = [a.elapsed_time(b) for a, b in events]
    pass_ms = wl.time_passes(flush, stream, min(args.steps, 50))
    ms = sum(step_ms) / args.steps
    ms_median = float(sorted(step_ms)[len(step_ms) // 2])
    ms = max_over_ranks(ms, device=dev)   # the slowest rank sets the whole-job time
    voxels = wl.voxels
    value = voxels * world / (ms * 1e-3) / 1e9

    # end to end through the public API: every step copies its volume from
    # pinned host memory to the device, maps it and copies the result back
    # (MCLAHE.forward_host: two device slots, so the copies of neighbouring
    # steps overlap each other and the kernels)
    e2e = None
    if rank == 0 or world > 1:
        h_in = torch.from_numpy(wl.x_host).pin_memory()
        h_out = torch.empty(h_in.shape, dtype=torch.float32).pin_memory()
        op.forward_host([h_in] * 3, [h_out] * 3, stream=stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        op.forward_host([h_in] * args.e2e_steps, [h_out] * args.e2e_steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
        e2e = {"value": voxels * world / (e2e_ms * 1e-3) / 1e9, "unit": "Gvoxel/s",
               "h2d_bytes_per_step": int(h_in.numel() * 4), "d2h_bytes_per_step": int(h_out.numel() * 4),
               "ms_per_step": e2e_ms, "call": "MCLAHE.forward_host (mclahe_forward_host)"}
        del h_in, h_out

    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    roofline, per_pass = wl.roofline(pass_ms)
    whole = 12 * voxels / (ms * 1e-3) / 1e9    # 2 input reads + 1 output write
    config = wl.config(args)
    x_host = wl.x_host
    wname = wl.w
    gpu_launches = int(sum(wl.launches.values()) * args.steps)
    wl.release()

    # the other configurations, and the headline volume with its range given
    extra = None
    if not args.no_extra and world == 1:
        extra = {}
        if not wname["adaptive"]:
            g = Workload(args.workload, args, dev, rank, given_range=True)
            g.tune(args)
            extra[args.workload + "+given-range"] = measure_simple(g, args, stream, flush,
                                                                   min(args.steps, 2000))
            g.release()
        for name in EXTRA_WORKLOADS:
            if name == args.workload:
                continue
            e = Workload(name, args, dev, rank)
            e.tune(args)
            extra[name] = measure_simple(e, args, stream, flush, min(args.steps, 2000))
            e.release()
        for name, dt in TYPED_WORKLOADS:
            extra[f"{name}-{dt}"] = measure_typed(name, dt, args, dev, stream, flush, min(args.steps, 2000))

    cpu = None
    if not args.no_cpu_baseline:
        rate, reps, el, cores, single = oracle_rate(x_host, wname)
        cpu = {"value": rate, "unit": "Gvoxel/s", "cores": cores, "kind": "oracle",
               "sample": f"whole {args.workload} volume x{reps} ({el:.1f} s, FP64, OpenMP)",
               "single_thread": single}

    forms = None
    if not args.no_forms and world == 1:
        forms = {"batched": measure_batched(dev, args.form_steps, 3),
                 "fwd_bwd": measure_fwd_bwd(dev, args.form_steps, 3)}

    line = {
        "metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "hbm_roofline_frac_whole_step": whole / roofline["peak"],
        "ms_per_step_median": ms_median,
        "passes_ms": pass_ms,
        "roofline": roofline,
        "roofline_per_pass": per_pass,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": sampler.summary(t0, t1),
        "workloads": extra,
        "forms": forms,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
