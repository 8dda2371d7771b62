"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every symbol include/mclahe.h declares, validates arguments, and its
plan geometry matches the oracle's (Sec. III.B, Eq. (1)-(2))."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "mclahe.h")).read()
    return sorted(set(re.findall(r"MCLAHE_API\s+[\w\s\*]*?\b(mclahe_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(nat):
    declared = _declared_symbols()
    assert len(declared) >= 12
    lib = nat.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(nat.EXPORTS) == declared


def test_status_strings_and_version(nat):
    assert nat.status_string(0) == "ok"
    for s in range(1, 8):
        assert nat.status_string(s) not in ("ok", "unknown status")
    assert nat.status_string(99) == "unknown status"
    assert nat.mclahe_version() >= 100


@pytest.mark.parametrize("shape,ks", [((512, 512), (64, 64)), ((64, 512, 512), (16, 64, 64)),
                                      ((128, 128, 256, 32), (32, 32, 32, 8)), ((37,), (6,)),
                                      ((5, 4, 7), (2, 3, 7)), ((9, 1, 11, 3), (4, 1, 5, 2))])
def test_plan_geometry_matches_oracle(nat, orc, shape, ks):
    plan = nat.mclahe_plan(shape, ks, 256, 0.01, nat.MCLAHE_RANGE_ADAPTIVE)
    info = nat.mclahe_plan_query(plan)
    g = orc.geometry(shape, ks)
    assert info["pad"] == g["p"] and info["pad_before"] == g["p0"]
    assert info["pad_after"] == g["p1"] and info["n_kernels_dim"] == g["n"]
    assert info["n_kernels"] == int(np.prod(g["n"]))
    assert info["kernel_voxels"] == int(np.prod(ks))
    assert info["n_voxels"] == int(np.prod(shape))
    offs = [info[k] for k in ("ws_status", "ws_range_keys", "ws_hist", "ws_lo", "ws_scale",
                              "ws_lut", "ws_scratch", "ws_bytes")]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    assert nat.mclahe_workspace_bytes(plan) == info["ws_bytes"]
    K, nb = info["n_kernels"], 256
    assert info["ws_lut"] - info["ws_hist"] >= 4 * K * nb + 8 * K


@pytest.mark.parametrize("kw", [
    dict(shape=(8, 8), ks=(9, 2)),            # kernel larger than the volume
    dict(shape=(0, 8), ks=(1, 2)),            # empty volume
    dict(shape=(8, 0), ks=(2, 1)),
    dict(shape=(8, 8), ks=(0, 2)),
    dict(shape=(8, 8), ks=(2,)),              # rank mismatch
    dict(shape=(8, 8, 8, 8, 8), ks=(2,) * 5),  # five dims
    dict(shape=(8, 8), ks=(2, 2), nb=1),
    dict(shape=(8, 8), ks=(2, 2), nb=4097),
    dict(shape=(8, 8), ks=(2, 2), clip=-0.1),
    dict(shape=(8, 8), ks=(2, 2), clip=1.5),
    dict(shape=(8, 8), ks=(2, 2), clip=float("nan")),
    dict(shape=(8, 8), ks=(2, 2), mode=7),
    dict(shape=(8, 8), ks=(2, 2), rng=(1.0, 0.0)),
    dict(shape=(8, 8), ks=(2, 2), rng=(0.0, float("inf"))),
    dict(shape=(8, 8), ks=(2, 2), mode=1, rng=(0.0, 1.0)),  # range only with GHR
])
def test_plan_rejects_invalid_arguments(nat, kw):
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_plan(kw["shape"], kw["ks"], kw.get("nb", 16), kw.get("clip", 0.1),
                        kw.get("mode", 0), kw.get("rng"))
    assert e.value.status == nat.MCLAHE_ERR_INVALID_ARG


def test_plan_rejects_unsupported_table_size(nat):
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_plan((64, 64, 64, 64), (8, 8, 8, 8), 4096, 0.1)
    assert e.value.status == nat.MCLAHE_ERR_UNSUPPORTED


def test_forward_rejects_bad_pointers_without_touching_the_device(nat):
    plan = nat.mclahe_plan((64, 64), (16, 16), 64, 0.1)
    ws = nat.mclahe_workspace_bytes(plan)
    lib = nat.load()
    # NULL input, misaligned output, workspace too small / misaligned: all host checks
    assert lib.mclahe_forward(plan.handle, None, 4096, 8192, ws, None, None) == nat.MCLAHE_ERR_INVALID_ARG
    assert lib.mclahe_forward(plan.handle, 4096, 4100, 8192, ws, None, None) == nat.MCLAHE_ERR_INVALID_ARG
    assert lib.mclahe_forward(plan.handle, 4096, 4096, 8192, ws, None, None) == nat.MCLAHE_ERR_INVALID_ARG
    assert lib.mclahe_forward(plan.handle, 4096, 8192, 16384, ws - 1, None, None) == nat.MCLAHE_ERR_WORKSPACE
    assert lib.mclahe_forward(plan.handle, 4096, 8192, 16400, ws, None, None) == nat.MCLAHE_ERR_WORKSPACE
    assert lib.mclahe_forward(None, 4096, 8192, 16384, ws, None, None) == nat.MCLAHE_ERR_INVALID_ARG


def test_set_shapes_validates_and_round_trips(nat):
    plan = nat.mclahe_plan((64, 512, 512), (16, 64, 64), 256, 0.02, nat.MCLAHE_RANGE_ADAPTIVE)
    n_last = nat.mclahe_plan_query(plan)["n_kernels_dim"][-1]
    nat.mclahe_plan_set_shapes(plan, 2, 1, 8, 24, 3)
    info = nat.mclahe_plan_query(plan)
    assert (info["hist_group"], info["hist_cluster"], info["hist_copies"], info["hist_shares"],
            info["map_chunks"], info["tuned"]) == (2, 1, 8, 24, 3, 2)
    # the adaptive range gets a flat range pass of its own in the flat form
    assert nat.mclahe_pass_launches(plan, nat.MCLAHE_PASS_RANGE) == 1
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1)
    assert nat.mclahe_plan_query(plan)["hist_shares"] == 0
    # the cluster form: the sweep inside the histogram pass (the default), or
    # the separate streaming range sweep
    assert nat.mclahe_plan_query(plan)["range_pass"] == 0
    assert nat.mclahe_pass_launches(plan, nat.MCLAHE_PASS_RANGE) == 0
    nat.mclahe_plan_set_range_pass(plan, 1)
    assert nat.mclahe_plan_query(plan)["range_pass"] == 1
    assert nat.mclahe_pass_launches(plan, nat.MCLAHE_PASS_RANGE) == 1
    nat.mclahe_plan_set_range_pass(plan, 0)
    assert nat.mclahe_plan_query(plan)["range_pass"] == 0
    assert nat.mclahe_pass_launches(plan, nat.MCLAHE_PASS_RANGE) == 0
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_plan_set_range_pass(plan, 2)
    assert e.value.status == nat.MCLAHE_ERR_INVALID_ARG
    glob = nat.mclahe_plan((64, 64), (16, 16), 64, 0.1)   # a global range has no per-kernel ranges
    assert nat.mclahe_plan_query(glob)["range_pass"] == 0
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_plan_set_range_pass(glob, 1)
    assert e.value.status == nat.MCLAHE_ERR_UNSUPPORTED
    odd_last = nat.mclahe_plan((16, 30), (4, 6), 64, 0.1, nat.MCLAHE_RANGE_ADAPTIVE)   # 30 % 4 != 0
    assert nat.mclahe_plan_query(odd_last)["range_pass"] == 0
    bad = [(0, 1, 8, 0, 1), (n_last + 1, 1, 8, 0, 1), (1, 3, 8, 0, 1), (1, 16, 8, 0, 1),
           (1, 1, 12, 0, 1), (1, 1, 64, 0, 1), (1, 2, 8, 4, 1), (1, 1, 8, -1, 1),
           (1, 1, 8, 4097, 1), (1, 1, 8, 0, 0), (1, 1, 8, 0, 65)]
    for args in bad:
        with pytest.raises(nat.MclaheError) as e:
            nat.mclahe_plan_set_shapes(plan, *args)
        assert e.value.status == nat.MCLAHE_ERR_INVALID_ARG, args
    # TMA tiles: this geometry's cell rows start on 16-byte boundaries
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 1)
    assert nat.mclahe_plan_query(plan)["map_tma"] == 1
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0)
    with pytest.raises(nat.MclaheError):
        nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 2)
    odd = nat.mclahe_plan((19, 23, 29), (5, 4, 7), 100, 0.02)
    with pytest.raises(nat.MclaheError):
        nat.mclahe_plan_set_shapes(odd, 1, 1, 8, 0, 1, 1)
    # histogram row walks: 0 ring, 1 TMA tiles (aligned rows only), 2 per-thread loads
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, hist_walk=2)
    assert nat.mclahe_plan_query(plan)["hist_walk"] == 2
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, hist_walk=1)
    assert nat.mclahe_plan_query(plan)["hist_walk"] == 1
    for bad_walk in (-1, 4):
        with pytest.raises(nat.MclaheError):
            nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, hist_walk=bad_walk)
    nat.mclahe_plan_set_shapes(odd, 1, 1, 8, 0, 1, 0, hist_walk=2)
    with pytest.raises(nat.MclaheError):
        nat.mclahe_plan_set_shapes(odd, 1, 1, 8, 0, 1, 0, hist_walk=1)
    # staged footprints (3): one kernel per cluster, 256-thread CTAs, aligned rows,
    # and the cluster's share of the footprint within the shared memory
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, hist_walk=3)
    assert nat.mclahe_plan_query(plan)["hist_walk"] == 3
    for args in ((2, 4, 16, 0), (1, 1, 16, 0), (1, 1, 8, 4)):   # G = 2; 256 KiB in one CTA; flat
        with pytest.raises(nat.MclaheError):
            nat.mclahe_plan_set_shapes(plan, *args, 1, 0, hist_walk=3)
    with pytest.raises(nat.MclaheError):
        nat.mclahe_plan_set_shapes(odd, 1, 1, 8, 0, 1, 0, hist_walk=3)
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, hist_walk=0)
    # 512-thread histogram CTAs only for 4-D volumes
    with pytest.raises(nat.MclaheError):
        nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, hist_threads=512)
    p4 = nat.mclahe_plan((16, 16, 24, 8), (4, 4, 6, 2), 256, 0.01)
    nat.mclahe_plan_set_shapes(p4, 1, 1, 8, 0, 1, 0, hist_threads=512)
    assert nat.mclahe_plan_query(p4)["hist_threads"] == 512
    with pytest.raises(nat.MclaheError):
        nat.mclahe_plan_set_shapes(p4, 1, 1, 8, 0, 1, 0, hist_threads=384)
    # flat mapping grid: 0 or 1, and not together with TMA tiles
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 8, 0, map_flat=1)
    assert (nat.mclahe_plan_query(plan)["map_flat"], nat.mclahe_plan_query(plan)["map_chunks"]) == (1, 8)
    for tma, flat in ((0, 2), (0, -1), (1, 1)):
        with pytest.raises(nat.MclaheError):
            nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 8, tma, map_flat=flat)
    assert nat.mclahe_plan_query(plan)["map_flat"] == 1
    nat.mclahe_plan_set_shapes(plan, 1, 4, 16, 0, 1, 0, map_flat=0)
    info = nat.mclahe_plan_query(plan)   # unchanged by the rejected calls
    assert (info["hist_group"], info["hist_cluster"], info["hist_copies"], info["hist_shares"],
            info["map_chunks"], info["map_flat"]) == (1, 4, 16, 0, 1, 0)
