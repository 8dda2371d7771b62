"""The benchmark's output contract, on the CPU: the reference arm (the FP64
oracle timed on the host cores) prints one JSON line with the contract's keys,
the GPU arm fails loudly where there is no GPU instead of falling back, and the
roofline's byte counts and recorded DRAM traffic belong to the kernel timed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "Gvoxel/s" and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 3)
    assert d["config"]["workload"] == "4d-photoemission-128x128x256x32"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the no-GPU behaviour")
def test_gpu_arm_fails_without_a_gpu():
    r = run_bench("--steps", "1", "--warmup", "3", timeout=200)
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def _bench():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_recorded_traffic_is_keyed_on_kernel_shapes_and_source():
    """The DRAM bytes the bench reports come from the committed ncu summary only
    for the kernel, launch shapes and kernel sources that it was taken on."""
    import json

    b = _bench()
    wl = "4d-photoemission-128x128x256x32"
    with open(os.path.join(ROOT, "profiles", f"dram_traffic_{wl}.json")) as f:
        rec = json.load(f)[wl]
    info = dict(rec["map"]["shapes"])
    info.update(rec["hist"]["shapes"])
    info.update(rec["range"]["shapes"])
    info["mode"] = 0
    for p in ("range", "hist", "map"):
        assert b.pass_kernel(p, info) == rec[p]["kernel"].split("<")[0]
        assert b.recorded_traffic(wl, p, info) == rec[p]["bytes_per_launch"], p
    other = dict(info, map_chunks=info["map_chunks"] * 2)   # another mapping variant: no figure
    assert b.recorded_traffic(wl, "map", other) is None
    assert b.recorded_traffic(wl, "hist", dict(info, hist_copies=info["hist_copies"] // 2)) is None


def test_algorithmic_bytes_and_kernels_of_the_range_forms():
    b = _bench()
    base = {"n_voxels": 1000, "n_kernels": 10, "n_bins": 64, "table_stride": 68, "hist_shares": 0,
            "hist_walk": 0, "range_pass": 0, "map_tma": 0, "map_flat": 0}
    # adaptive, in-pass sweep: no range pass; separate sweep or flat form: one read of the input
    assert b.algorithmic_bytes(base, True, False)["range"] == 0
    assert b.algorithmic_bytes(dict(base, range_pass=1), True, False)["range"] == 4 * 1000 + 8 * 10
    assert b.algorithmic_bytes(dict(base, hist_shares=4), True, False)["range"] == 4 * 1000 + 8 * 10
    # global range: one read unless given
    assert b.algorithmic_bytes(base, False, False)["range"] == 4000
    assert b.algorithmic_bytes(base, False, True)["range"] == 0
    assert b.algorithmic_bytes(base, False, False)["map"] == 8000
    assert b.pass_kernel("range", dict(base, mode=1, range_pass=1)) == "k_range_kernels"
    assert b.pass_kernel("range", dict(base, mode=1, hist_shares=2)) == "k_hist_flat"
    assert b.pass_kernel("range", dict(base, mode=0)) == "k_range_global"
    assert b.pass_kernel("hist", dict(base, mode=1, hist_walk=3)) == "k_hist_staged"
    assert b.pass_kernel("map", dict(base, mode=0, map_tma=1)) == "k_map_tma"
    assert b.pass_kernel("map", dict(base, mode=0, map_flat=1)) == "k_map_flat"
