"""The adaptive range's separate streaming sweep (k_range_kernels,
mclahe_plan_set_range_pass): the per-kernel ranges it leaves must equal those
the histogram pass finds by sweeping each footprint itself, so ranges,
histograms, tables and outputs are equal bit for bit between the two forms,
and the oracle's within the usual bounds.  Geometries with b not dividing s
give footprints that overlap through the mirror images (a voxel in up to three
kernels per dimension); rows whose quad count is not a multiple of 32 leave
lanes idle in the last group."""
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


CASES = [
    ((40, 56), (8, 7), 64),
    ((12, 300), (5, 37), 128),            # wide rows, b not dividing s
    ((37, 20, 24), (6, 5, 8), 100),
    ((19, 23, 28), (5, 4, 7), 128),
    ((64, 96, 128), (16, 24, 32), 256),
    ((13, 9, 11, 8), (3, 4, 5, 4), 50),
    ((10, 12, 16, 20), (4, 5, 6, 7), 512),
]


@pytest.mark.parametrize("walk", [0, 1, 2])
@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) for c in CASES])
def test_separate_range_sweep_equals_in_pass_sweep(torch_cuda, orc, case, walk):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb = case
    rng = np.random.default_rng(hash((shape, ks, 17)) % 2**32)
    x = (rng.gamma(2.0, size=shape) * rng.uniform(0.5, 3.0)).astype(np.float32)
    clip = float(np.float32(0.02))
    xd = torch.from_numpy(x).cuda()
    res = []
    for rp in (1, 0):
        op = MCLAHE(shape, ks, n_bins=nb, clip_limit=clip, adaptive=True)
        sh = op.shapes()
        if walk == 1:
            sh.update(hist_walk=1)
            try:
                op.set_shapes(**sh)
            except nat.MclaheError:
                pytest.skip("no TMA row tiles for this geometry")
        else:
            sh.update(hist_walk=walk)
            op.set_shapes(**sh)
        if (shape[-1] % 4) == 0:
            nat.mclahe_plan_set_range_pass(op.plan, rp)
        elif rp == 1:
            continue
        assert nat.mclahe_pass_launches(op.plan, nat.MCLAHE_PASS_RANGE) == rp
        out = op.forward(xd)
        torch.cuda.synchronize()
        info = nat.mclahe_plan_query(op.plan)
        a, b = info["ws_hist"], info["ws_scratch"]
        res.append((out.cpu().numpy(), op.ws[a:b].cpu().numpy(), op.histograms().cpu().numpy()))
    if len(res) == 2:
        assert np.array_equal(res[0][0], res[1][0])
        assert np.array_equal(res[0][1], res[1][1])   # histograms, ranges and tables
    want, aux = orc.mclahe(x, ks, nb, clip, mode=1, full=True)
    np.testing.assert_array_equal(res[0][2], aux["hist"].astype(np.int64))
    assert np.abs(res[0][0].astype(np.float64) - want).max() <= 1e-5


def test_separate_range_sweep_on_the_fluorescence_stack(torch_cuda, orc):
    """The 3-D fluorescence workload (64x512x512, kernel 16x64x64, 256 bins):
    both forms, and the oracle, on the full volume."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE

    x = synth.fluorescence((64, 512, 512), seed=1)
    ks, nb, clip = (16, 64, 64), 256, float(np.float32(0.02))
    xd = torch.from_numpy(x).cuda()
    outs = []
    for rp in (1, 0):
        op = MCLAHE(x.shape, ks, n_bins=nb, clip_limit=clip, adaptive=True)
        nat.mclahe_plan_set_range_pass(op.plan, rp)
        outs.append(op.forward(xd).cpu().numpy())
        if rp == 1:
            hist = op.histograms().cpu().numpy()
    assert np.array_equal(outs[0], outs[1])
    want, aux = orc.mclahe(x, ks, nb, clip, mode=1, full=True)
    np.testing.assert_array_equal(hist, aux["hist"].astype(np.int64))
    assert np.abs(outs[0].astype(np.float64) - want).max() <= 1e-5
