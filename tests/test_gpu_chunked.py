"""Out-of-core processing (mclahe_forward_chunked): a host-resident volume
streamed through a small device staging buffer in slabs along dimension 0.

The slabs run the same kernels as the in-core forward pass (cluster-form
histograms with the row ring, per-cell mapping), so with those shapes the
output must equal mclahe_forward's bit for bit, and the oracle's within 1e-5
(histograms exact).  Staging buffers just large enough for one kernel row's
footprint force a slab per kernel row; geometries with b not dividing s give
edge kernels whose footprints reach across several mirror images."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_11355_gb300 import build

    build.build()
    return torch


def f32(c):
    return float(np.float32(c))


def footprint_rows(shape, ks):
    """The widest footprint along dimension 0 (rows), from the oracle's geometry."""
    import oracle

    g = oracle.geometry(shape, ks)
    b, p0, s = ks[0], g["p0"][0], shape[0]
    widest = 0
    for k in range(g["n"][0]):
        rows = set()
        for P in range(k * b, k * b + b):
            j = P - p0
            while j < 0 or j >= s:
                j = -1 - j if j < 0 else 2 * s - 1 - j
            rows.add(j)
        widest = max(widest, max(rows) - min(rows) + 1)
    return max(widest, b)


def run_chunked(torch, orc, x, ks, nb, clip, adaptive, stage_rows_factor=1.0, global_range=None):
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    clip = f32(clip)
    op = MCLAHE(x.shape, ks, nb, clip, adaptive, global_range=global_range)
    sh = op.shapes()
    sh.update(hist_shares=0, hist_walk=0, map_tma=0, map_flat=0)
    op.set_shapes(**sh)
    row = int(np.prod(x.shape[1:]))
    rows = int(footprint_rows(x.shape, ks) * stage_rows_factor)
    stage_bytes = 2 * (rows * row + 8) * 4 + 256
    stage = torch.empty(stage_bytes, dtype=torch.uint8, device="cuda")
    h_in = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    h_out = torch.full(x.shape, -1.0, dtype=torch.float32).pin_memory()
    nat.mclahe_forward_chunked(op.plan, h_in, h_out, op.ws, op.ws_bytes, stage, stage_bytes)
    torch.cuda.synchronize()
    got = h_out.numpy().copy()
    hist = op.histograms().cpu().numpy()
    # in core, the same walks
    ref = op.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(got, ref)
    want, aux = orc.mclahe(x, ks, nb, clip, mode=int(adaptive), range_=global_range, full=True)
    np.testing.assert_array_equal(hist, aux["hist"].astype(np.int64))
    assert np.abs(got.astype(np.float64) - want).max() <= 1e-5
    return op


CASES = [
    ((40, 56), (8, 7), 64, 0.02, False),
    ((37, 20, 24), (6, 5, 8), 100, 0.02, True),
    ((19, 23, 28), (5, 4, 7), 128, 0.03, False),
    ((13, 9, 11, 8), (3, 4, 5, 4), 50, 0.03, True),
    ((12, 8, 16, 12), (4, 4, 8, 3), 512, 0.01, False),
]


@pytest.mark.parametrize("factor", [1.0, 2.5])
@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) + ("A" if c[4] else "G") for c in CASES])
def test_chunked_equals_in_core_and_oracle(torch_cuda, orc, case, factor):
    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, 5)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    run_chunked(torch_cuda, orc, x, ks, nb, clip, adaptive, stage_rows_factor=factor)


def test_chunked_fluorescence_stack(torch_cuda, orc):
    """The 3-D fluorescence workload (64x512x512, kernel 16x64x64, adaptive range)
    through a staging buffer of about 24 MiB: five slabs per sweep."""
    from paper_1906_11355_gb300 import synth

    x = synth.fluorescence((64, 512, 512), seed=1)
    run_chunked(torch_cuda, orc, x, (16, 64, 64), 256, 0.02, True, stage_rows_factor=1.5)


def test_chunked_rejects_a_staging_buffer_too_small(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE((32, 16, 16), (8, 4, 4), 64, 0.02)
    stage = torch.empty(4096, dtype=torch.uint8, device="cuda")
    h = torch.zeros((32, 16, 16)).pin_memory()
    o = torch.zeros((32, 16, 16)).pin_memory()
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_forward_chunked(op.plan, h, o, op.ws, op.ws_bytes, stage, 4096)
    assert e.value.status == nat.MCLAHE_ERR_WORKSPACE


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", [((40, 12, 16), (8, 4, 8), 64, 0.02, True),
                                  ((30, 9, 10, 12), (6, 3, 5, 4), 128, 0.01, False),
                                  ((64, 512, 512), (16, 64, 64), 256, 0.02, True)],
                         ids=["3dA", "4dG", "fluorescence"])
def test_one_volume_split_across_ranks_in_one_process(torch_cuda, orc, case, world):
    """The split-volume path (dist.SlabRank, mclahe_forward_slab) with `world`
    ranks emulated one after another on one GPU, phase by phase: each rank its
    own workspace and input slab; the range keys combined by a maximum; the
    one-row table halo copied from rank r + 1 to rank r; each rank's output rows
    assembled into the volume.  Equal to the oracle (histograms exact)."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import dist as md
    from paper_1906_11355_gb300 import synth

    shape, ks, nb, clip, adaptive = case
    if shape == (64, 512, 512):
        x = synth.fluorescence(shape, seed=1)
    else:
        x = np.random.default_rng(sum(shape)).gamma(2.0, size=shape).astype(np.float32)
    clip = f32(clip)
    mode = nat.MCLAHE_RANGE_ADAPTIVE if adaptive else nat.MCLAHE_RANGE_GLOBAL
    plan = nat.mclahe_plan(shape, ks, nb, clip, mode)
    flat = torch.from_numpy(x).cuda().reshape(-1)
    ranks = [md.SlabRank(plan, r, world) for r in range(world)]
    slabs = []
    for p in ranks:
        a, b = p.slab_bounds()
        slabs.append((flat[a:b].clone(), torch.full((b - a,), -1.0, device="cuda")))
    if not adaptive:
        for p, (s, _) in zip(ranks, slabs):
            p.range(s)
        keys = torch.stack([p.keys().to(torch.int64) & 0xFFFFFFFF for p in ranks]).max(0).values
        for p in ranks:
            p.set_keys(keys.where(keys < 2 ** 31, keys - 2 ** 32).to(torch.int32))
    for p, (s, _) in zip(ranks, slabs):
        p.hist(s)
    for r, p in enumerate(ranks):
        k = p.needs_row()
        if k is not None:
            p.put_row_tables(k, ranks[r + 1].first_row_tables())
    out = torch.full_like(flat, -2.0)
    row = int(np.prod(shape[1:]))
    for p, (s, o) in zip(ranks, slabs):
        p.map(s, o)
        a, b = p.out_rows()
        first = p.slab_bounds()[0]
        out[a * row:b * row] = o[a * row - first:b * row - first]
    torch.cuda.synchronize()
    want = orc.mclahe(x, ks, nb, clip, mode=int(adaptive))
    got = out.reshape(shape).cpu().numpy()
    assert np.abs(got.astype(np.float64) - want).max() <= 1e-5
