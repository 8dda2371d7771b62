"""Parity of the CUDA forward path (through the C ABI) with the FP64 oracle.

Histograms and ranges must match bit for bit, mapping tables to 1e-6 and the
output to 1e-5 max-abs (the output lies in [0, 1]).  Small cases span several
kernels and ragged tails in 1-4 dimensions.  The workload cases run the full
synthetic volumes after mclahe_autotune has picked the launch shapes, which is
what the benchmark does before it times them, and then under every mapping
walk (per-cell grid, flat persistent grid, TMA tiles) with one and several
CTAs per cell."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OUT_TOL = 1e-5
LUT_TOL = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_11355_gb300 import build

    build.build()
    return torch


def f32(c):
    return float(np.float32(c))


def run_case(torch, orc, x, ks, nb, clip, adaptive=False, global_range=None, shapes=None):
    from paper_1906_11355_gb300.api import MCLAHE

    clip = f32(clip)
    op = MCLAHE(x.shape, ks, n_bins=nb, clip_limit=clip, adaptive=adaptive,
                global_range=global_range)
    if shapes is not None:
        op.set_shapes(**shapes)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = op.forward(xd)
    torch.cuda.synchronize()
    want, aux = orc.mclahe(x, ks, nb, clip, mode=int(adaptive), range_=global_range, full=True)
    hist = op.histograms().cpu().numpy()
    np.testing.assert_array_equal(hist, aux["hist"].astype(np.int64))
    lo, sc = (t.cpu().numpy() for t in op.ranges())
    np.testing.assert_array_equal(lo, aux["lo"])
    np.testing.assert_array_equal(sc, aux["scale"])
    lut = op.tables().cpu().numpy().astype(np.float64)
    assert np.abs(lut - aux["lut"]).max() <= LUT_TOL
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - want).max()
    assert err <= OUT_TOL, f"max abs error {err}"
    return op, out, got


CASES = [
    # (shape, kernel, n_bins, clip, adaptive)
    ((37,), (6,), 16, 0.05, False),
    ((1000,), (7,), 64, 0.02, True),
    ((53, 47), (8, 7), 64, 0.01, False),
    ((53, 47), (8, 7), 64, 0.01, True),
    ((64, 64), (16, 16), 256, 0.0, False),
    ((64, 64), (16, 16), 256, 1.0, True),
    ((30, 41), (30, 41), 32, 0.1, False),        # b = s
    ((33, 18), (1, 5), 8, 0.3, True),            # unit kernel along dim 0
    ((130, 97), (13, 24), 4096, 0.002, False),   # many bins, odd rows
    ((19, 23, 29), (5, 4, 7), 100, 0.02, False),
    ((19, 23, 29), (5, 4, 7), 100, 0.02, True),
    ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
    ((11, 9, 13, 10), (3, 4, 5, 2), 50, 0.03, False),
    ((11, 9, 13, 10), (3, 4, 5, 2), 50, 0.03, True),
    ((8, 8, 16, 12), (4, 4, 8, 3), 512, 0.01, False),
    ((4, 3, 5, 3), (4, 3, 5, 3), 7, 0.5, True),
]


@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) + ("A" if c[4] else "G") for c in CASES])
def test_forward_matches_oracle(torch_cuda, orc, case):
    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    run_case(torch_cuda, orc, x, ks, nb, clip, adaptive)


# both histogram forms with explicit launch shapes: clusters of 1-8 CTAs, and
# the flat form with 1 share per item up to more shares than an item has rows
FORM_CASES = [
    ((53, 47), (8, 7), 64, 0.01, False),
    ((19, 23, 29), (5, 4, 7), 100, 0.02, True),
    ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
    ((11, 9, 13, 10), (3, 4, 5, 2), 50, 0.03, False),
    ((11, 9, 13, 10), (3, 4, 5, 2), 50, 0.03, True),
]
FORMS = [dict(hist_group=1, hist_cluster=4, hist_copies=4, hist_shares=0, map_chunks=2),
         dict(hist_group=2, hist_cluster=2, hist_copies=8, hist_shares=0, map_chunks=1,
              hist_threads=512),
         dict(hist_group=1, hist_cluster=1, hist_copies=8, hist_shares=1, map_chunks=1),
         dict(hist_group=2, hist_cluster=1, hist_copies=2, hist_shares=7, map_chunks=1),
         dict(hist_group=1, hist_cluster=1, hist_copies=16, hist_shares=300, map_chunks=3),
         dict(hist_group=1, hist_cluster=2, hist_copies=8, hist_shares=0, map_chunks=5,
              map_flat=1)]


@pytest.mark.parametrize("form", range(len(FORMS)))
@pytest.mark.parametrize("case", FORM_CASES,
                         ids=[str(c[0]) + ("A" if c[4] else "G") for c in FORM_CASES])
def test_histogram_forms_match_oracle(torch_cuda, orc, case, form):
    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, form)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    shapes = dict(FORMS[form])
    # clusters of whole kernels: at most the kernels along the last dimension
    from paper_1906_11355_gb300 import _native as nat

    n_last = nat.mclahe_plan_query(nat.mclahe_plan(shape, ks, nb, f32(clip), int(adaptive)))[
        "n_kernels_dim"][-1]
    shapes["hist_group"] = min(shapes["hist_group"], n_last)
    if shapes.get("hist_threads", 256) == 512 and len(shape) < 4:
        pytest.skip("512-thread histogram CTAs are for 4-D volumes")
    op, _, _ = run_case(torch_cuda, orc, x, ks, nb, clip, adaptive, shapes=shapes)
    assert {k: v for k, v in op.shapes().items() if k in shapes} == shapes
    # a second call on the same workspace (the flat form's accumulators are cleared)
    x2 = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    xd = torch_cuda.from_numpy(x2).cuda()
    got = op.forward(xd).cpu().numpy().astype(np.float64)
    want = orc.mclahe(x2, ks, nb, f32(clip), mode=int(adaptive))
    assert np.abs(got - want).max() <= OUT_TOL


# the mapping pass on TMA box tiles: 3- and 4-D, both range modes, cells cut
# into whole tiles and edge cells with partial tiles (per-element stores)
TMA_CASES = [
    ((12, 40, 64), (4, 8, 8), 64, 0.02, False),
    ((20, 24, 48), (5, 6, 12), 128, 0.01, True),
    ((6, 10, 12, 16), (3, 5, 4, 8), 512, 0.01, False),
    ((8, 8, 16, 24), (4, 4, 8, 8), 100, 0.03, True),
    ((13, 37, 36), (4, 6, 12), 256, 0.02, False),
    ((9, 11, 14, 20), (3, 4, 5, 4), 50, 0.05, True),
]


@pytest.mark.parametrize("chunks", [1, 3])
@pytest.mark.parametrize("case", TMA_CASES, ids=[str(c[0]) + ("A" if c[4] else "G") for c in TMA_CASES])
def test_tma_mapping_matches_oracle(torch_cuda, orc, case, chunks):
    from paper_1906_11355_gb300 import _native as nat

    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, chunks)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    x[rng.random(size=shape) < 0.3] = 0.0   # many voxels in bin 0 (global range)
    plan = nat.mclahe_plan(shape, ks, nb, f32(clip), int(adaptive))
    shapes = {k: v for k, v in nat.mclahe_plan_query(plan).items()
              if k in ("hist_group", "hist_cluster", "hist_copies", "hist_shares")}
    shapes.update(map_chunks=chunks, map_tma=1)
    op, out, _ = run_case(torch_cuda, orc, x, ks, nb, clip, adaptive, shapes=shapes)
    assert op.shapes()["map_tma"] == 1
    assert nat.mclahe_sync_status(op.ws) == 0


# the histogram pass on TMA box tiles and on per-thread loads (the ring walk is
# the default of every other test): 2- to 4-D, both range modes, cluster and
# flat forms, mirror pieces that start off a 16-byte boundary
TMA_HIST_CASES = [
    ((64, 64), (16, 16), 256, 0.02, False),
    ((40, 56), (5, 7), 64, 0.03, True),
    ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
    ((13, 37, 36), (4, 6, 12), 256, 0.02, False),
    ((6, 10, 12, 16), (3, 5, 4, 8), 512, 0.01, False),
    ((9, 11, 14, 20), (3, 4, 5, 4), 50, 0.05, True),
]
TMA_HIST_FORMS = [dict(hist_group=1, hist_cluster=2, hist_copies=4, hist_shares=0),
                  dict(hist_group=2, hist_cluster=1, hist_copies=8, hist_shares=7),
                  dict(hist_group=1, hist_cluster=1, hist_copies=16, hist_shares=300)]


@pytest.mark.parametrize("walk", [1, 2], ids=["tma", "loads"])
@pytest.mark.parametrize("form", range(len(TMA_HIST_FORMS)))
@pytest.mark.parametrize("case", TMA_HIST_CASES,
                         ids=[str(c[0]) + ("A" if c[4] else "G") for c in TMA_HIST_CASES])
def test_histogram_walks_match_oracle(torch_cuda, orc, case, form, walk):
    from paper_1906_11355_gb300 import _native as nat

    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, form, 7)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    shapes = dict(TMA_HIST_FORMS[form], map_chunks=1, hist_walk=walk)
    op, _, _ = run_case(torch_cuda, orc, x, ks, nb, clip, adaptive, shapes=shapes)
    assert op.shapes()["hist_walk"] == walk
    assert nat.mclahe_sync_status(op.ws) == 0


def test_tma_mapping_rejected_where_rows_are_unaligned(torch_cuda):
    from paper_1906_11355_gb300.api import MCLAHE
    from paper_1906_11355_gb300 import _native as nat

    op = MCLAHE((19, 23, 29), (5, 4, 7), n_bins=100, clip_limit=0.02)
    sh = op.shapes()
    sh["map_tma"] = 1
    with pytest.raises(nat.MclaheError):
        op.set_shapes(**sh)


@pytest.mark.parametrize("case", [((512, 512), (64, 64), 256, 0.01, False),
                                  ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
                                  ((6, 10, 12, 16), (3, 5, 4, 8), 512, 0.01, False)],
                         ids=["2dG", "3dA", "4dG"])
def test_graph_forward_equals_forward(torch_cuda, orc, case):
    """mclahe_forward_graph replays the same launches: bit-equal to mclahe_forward, on
    repeated calls and new contents of the same buffers, and after a shape change."""
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(5)
    op = MCLAHE(shape, ks, nb, f32(clip), adaptive)
    x = torch.empty(shape, device="cuda")
    a, b = torch.empty_like(x), torch.empty_like(x)
    for rep in range(3):
        x.copy_(torch.from_numpy(rng.gamma(2.0, 1.0, size=shape).astype(np.float32)))
        op.forward(x, out=a)
        op.forward(x, out=b, graph=True)
        torch.cuda.synchronize()
        assert torch.equal(a, b), rep
        if rep == 1:   # new launch shapes: the cached graph is dropped and recaptured
            sh = op.shapes()
            sh["map_chunks"] = 2 if sh["map_chunks"] == 1 else 1
            op.set_shapes(**sh)
    want = orc.mclahe(x.cpu().numpy(), ks, nb, f32(clip), mode=int(adaptive))
    assert np.abs(b.cpu().numpy().astype(np.float64) - want).max() <= OUT_TOL


def test_given_global_range_and_out_of_range_values(torch_cuda, orc):
    rng = np.random.default_rng(5)
    x = rng.normal(0.5, 0.4, size=(40, 50)).astype(np.float32)
    run_case(torch_cuda, orc, x, (8, 10), 64, 0.02, False, global_range=(0.0, 1.0))


@pytest.mark.parametrize("adaptive", [False, True])
def test_constant_and_two_level_images(torch_cuda, orc, adaptive):
    x = np.full((24, 36), 0.7, np.float32)
    _, _, got = run_case(torch_cuda, orc, x, (8, 9), 32, 0.02, adaptive)
    assert np.all(got == 0.0)
    x = np.zeros((20, 20, 8), np.float32)
    x[:, :10] = 1.0
    run_case(torch_cuda, orc, x, (5, 5, 4), 16, 0.05, adaptive)


def test_integer_valued_data_with_ties(torch_cuda, orc):
    rng = np.random.default_rng(8)
    x = rng.poisson(1.5, size=(24, 20, 16, 8)).astype(np.float32)
    run_case(torch_cuda, orc, x, (8, 5, 8, 4), 512, 0.01, False)
    run_case(torch_cuda, orc, x, (8, 5, 8, 4), 256, 0.01, True)


def test_device_clip_overrides_plan_and_is_deterministic(torch_cuda, orc):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE

    rng = np.random.default_rng(9)
    x = rng.random((48, 40), dtype=np.float32)
    xd = torch.from_numpy(x).cuda()
    op = MCLAHE(x.shape, (12, 10), 64, clip_limit=0.5)
    clip = torch.tensor([f32(0.015)], device="cuda")
    a = op.forward(xd, clip=clip)
    b = op.forward(xd, clip=clip)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    want = orc.mclahe(x, (12, 10), 64, f32(0.015))
    assert np.abs(a.cpu().numpy() - want).max() <= OUT_TOL
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = op.forward(xd, clip=clip, stream=s)
    s.synchronize()
    assert torch.equal(a, c)


WORKLOADS = ["2d-smooth-512x512", "3d-fluorescence-64x512x512", "4d-photoemission-128x128x256x32"]


@pytest.fixture(scope="module")
def workload_cache(orc):
    """Each full-size workload volume and its oracle result, computed once."""
    from paper_1906_11355_gb300 import synth

    cache = {}

    def get(name):
        if name not in cache:
            w = synth.WORKLOADS[name]
            x = synth.make_volume(w["gen"], w["shape"], w["seed"])
            want, aux = orc.mclahe(x, w["kernel"], w["n_bins"], f32(w["clip_limit"]),
                                   mode=int(w["adaptive"]), full=True)
            cache.clear()   # one full-size volume held at a time
            cache[name] = (w, x, want, aux)
        return cache[name]

    return get


def check_full(torch, op, xd, want, aux, out=None, graph=False):
    out = op.forward(xd, out=out, graph=graph)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(op.histograms().cpu().numpy(), aux["hist"].astype(np.int64))
    lo, sc = (t.cpu().numpy() for t in op.ranges())
    np.testing.assert_array_equal(lo, aux["lo"])
    np.testing.assert_array_equal(sc, aux["scale"])
    assert np.abs(op.tables().cpu().numpy().astype(np.float64) - aux["lut"]).max() <= LUT_TOL
    err = np.abs(out.cpu().numpy().astype(np.float64) - want).max()
    assert err <= OUT_TOL, f"max abs error {err} with shapes {op.shapes()}"
    return out


@pytest.mark.parametrize("name", WORKLOADS)
def test_workload_full_size_autotuned(torch_cuda, workload_cache, name):
    """The full volume with the launch shapes mclahe_autotune picks (the benchmark's
    configuration), through mclahe_forward and the graph-replayed mclahe_forward_graph."""
    from paper_1906_11355_gb300.api import MCLAHE

    w, x, want, aux = workload_cache(name)
    op = MCLAHE(x.shape, w["kernel"], w["n_bins"], f32(w["clip_limit"]), w["adaptive"])
    xd = torch_cuda.from_numpy(x).cuda()
    out = torch_cuda.empty_like(xd)
    op.autotune(xd, out)
    check_full(torch_cuda, op, xd, want, aux, out=out)
    out.fill_(-1.0)
    check_full(torch_cuda, op, xd, want, aux, out=out, graph=True)


def _map_walks(name, tuned):
    walks = [dict(map_flat=0, map_tma=0, map_chunks=1), dict(map_flat=1, map_tma=0, map_chunks=1),
             dict(map_flat=0, map_tma=0, map_chunks=4), dict(map_flat=1, map_tma=0, map_chunks=32)]
    if name != "2d-smooth-512x512":
        walks += [dict(map_flat=0, map_tma=1, map_chunks=1), dict(map_flat=0, map_tma=1, map_chunks=4)]
    if tuned not in walks:
        walks.append(tuned)
    return walks


@pytest.mark.parametrize("name", WORKLOADS)
def test_workload_full_size_every_mapping_walk(torch_cuda, workload_cache, name):
    """The full volume under every mapping walk, with the autotuned histogram shapes."""
    from paper_1906_11355_gb300.api import MCLAHE

    w, x, want, aux = workload_cache(name)
    op = MCLAHE(x.shape, w["kernel"], w["n_bins"], f32(w["clip_limit"]), w["adaptive"])
    xd = torch_cuda.from_numpy(x).cuda()
    out = torch_cuda.empty_like(xd)
    op.autotune(xd, out)
    tuned = op.shapes()
    for walk in _map_walks(name, {k: tuned[k] for k in ("map_flat", "map_tma", "map_chunks")}):
        op.set_shapes(**{**tuned, **walk})
        out.fill_(-1.0)
        check_full(torch_cuda, op, xd, want, aux, out=out)


# the staged histogram walk (hist_walk = 3): every kernel's footprint copied into
# the shared memory of its cluster once; 2- to 4-D, both range modes, edge
# kernels with mirror multiplicities 2 and 3 (b not dividing s), clusters of 1-8
STAGED_CASES = [
    ((64, 64), (16, 16), 256, 0.02, False),
    ((40, 56), (5, 7), 64, 0.03, True),
    ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
    ((13, 37, 36), (4, 6, 12), 256, 0.02, False),
    ((19, 23, 28), (5, 4, 7), 100, 0.02, True),
    ((6, 10, 12, 16), (3, 5, 4, 8), 512, 0.01, False),
    ((9, 11, 14, 20), (3, 4, 5, 4), 50, 0.05, True),
]


@pytest.mark.parametrize("cluster,copies", [(1, 32), (2, 8), (4, 16), (8, 2)])
@pytest.mark.parametrize("case", STAGED_CASES,
                         ids=[str(c[0]) + ("A" if c[4] else "G") for c in STAGED_CASES])
def test_staged_histogram_walk_matches_oracle(torch_cuda, orc, case, cluster, copies):
    from paper_1906_11355_gb300 import _native as nat

    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, cluster, 3)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    x[rng.random(size=shape) < 0.2] = 0.0
    shapes = dict(hist_group=1, hist_cluster=cluster, hist_copies=copies, hist_shares=0,
                  map_chunks=1, hist_walk=3)
    op, _, _ = run_case(torch_cuda, orc, x, ks, nb, clip, adaptive, shapes=shapes)
    assert op.shapes()["hist_walk"] == 3
    assert nat.mclahe_sync_status(op.ws) == 0
