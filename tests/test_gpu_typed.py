"""Native integer inputs (mclahe_forward_typed): uint16 and uint8 volumes.

An integer voxel's intensity is the integer itself, so the oracle is run on the
float32 volume of the same values (an exact conversion).  Histograms and ranges
must match bit for bit and the output within 1e-5; with the same walks the
integer forms must also equal mclahe_forward on that float32 volume bit for
bit.  The full-size cases are the 3-D fluorescence stack as its uint16 counts
and the 4-D photoemission counts as uint8."""
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


def device_ints(torch, x):
    """x (uint16 or uint8 numpy) on the device, and its dtype code (int16 / uint8 storage)."""
    from paper_1906_11355_gb300 import _native as nat

    if x.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int16)).cuda(), nat.MCLAHE_U16
    return torch.from_numpy(np.ascontiguousarray(x)).cuda(), nat.MCLAHE_U8


def run_typed(torch, orc, x, ks, nb, clip, adaptive, shapes=None, global_range=None):
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    clip = f32(clip)
    op = MCLAHE(x.shape, ks, n_bins=nb, clip_limit=clip, adaptive=adaptive, global_range=global_range)
    if shapes is not None:
        op.set_shapes(**shapes)
    xd, code = device_ints(torch, x)
    out = torch.full(x.shape, -1.0, dtype=torch.float32, device="cuda")
    nat.mclahe_forward_typed(op.plan, code, xd, out, op.ws, op.ws_bytes)
    torch.cuda.synchronize()
    xf = x.astype(np.float32)
    want, aux = orc.mclahe(xf, ks, nb, clip, mode=int(adaptive), range_=global_range, full=True)
    np.testing.assert_array_equal(op.histograms().cpu().numpy(), aux["hist"].astype(np.int64))
    lo, sc = (t.cpu().numpy() for t in op.ranges())
    np.testing.assert_array_equal(lo, aux["lo"])
    np.testing.assert_array_equal(sc, aux["scale"])
    assert np.abs(op.tables().cpu().numpy().astype(np.float64) - aux["lut"]).max() <= LUT_TOL
    err = np.abs(out.cpu().numpy().astype(np.float64) - want).max()
    assert err <= OUT_TOL, f"max abs error {err}"
    return op, out, xf


CASES = [
    # (shape, kernel, n_bins, clip, adaptive)
    ((37,), (6,), 16, 0.05, False),
    ((53, 47), (8, 7), 64, 0.01, False),
    ((64, 64), (16, 16), 256, 0.02, True),
    ((19, 23, 29), (5, 4, 7), 100, 0.02, True),
    ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
    ((11, 9, 13, 10), (3, 4, 5, 2), 50, 0.03, False),
    ((8, 8, 16, 12), (4, 4, 8, 3), 512, 0.01, True),
]


@pytest.mark.parametrize("dtype", ["u16", "u8"])
@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) + ("A" if c[4] else "G") for c in CASES])
def test_integer_input_matches_oracle_and_float_path(torch_cuda, orc, case, dtype):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, dtype)) % 2**32)
    if dtype == "u16":
        x = rng.poisson(rng.uniform(50, 3000, size=shape)).clip(0, 65535).astype(np.uint16)
    else:
        x = rng.poisson(rng.uniform(0.3, 60, size=shape)).clip(0, 255).astype(np.uint8)
    # the same walks for both forms: cluster histograms with the ring, per-thread mapping
    plan_shapes = MCLAHE(shape, ks, nb, f32(clip), adaptive).shapes()
    plan_shapes.update(hist_shares=0, hist_walk=0, map_tma=0, map_flat=0)
    if plan_shapes["hist_cluster"] < 1:
        plan_shapes["hist_cluster"] = 1
    op, out, xf = run_typed(torch, orc, x, ks, nb, clip, adaptive, shapes=plan_shapes)
    ref = op.forward(torch.from_numpy(xf).cuda())
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("walk", [0, 2, 3])
def test_integer_input_under_other_plan_shapes(torch_cuda, orc, walk):
    """Plans tuned for float32 volumes (flat histograms, TMA or flat mapping, the
    per-thread or staged histogram walks) still give exact results for integers."""
    shape, ks, nb = (16, 40, 48), (4, 8, 12), 128
    rng = np.random.default_rng(walk)
    x = rng.poisson(rng.uniform(1, 40, size=shape)).clip(0, 255).astype(np.uint8)
    shapes = dict(hist_group=1, hist_cluster=2 if walk == 3 else 1, hist_copies=8,
                  hist_shares=0 if walk == 3 else 5, map_chunks=2, map_tma=1 if walk == 0 else 0,
                  hist_walk=walk, map_flat=1 if walk == 2 else 0)
    run_typed(torch_cuda, orc, x, ks, nb, 0.02, True, shapes=shapes)
    run_typed(torch_cuda, orc, x.astype(np.uint16) * 7, ks, nb, 0.02, False, shapes=shapes)


def test_integer_input_given_global_range(torch_cuda, orc):
    rng = np.random.default_rng(3)
    x = rng.integers(0, 4096, size=(40, 56), dtype=np.uint16)
    run_typed(torch_cuda, orc, x, (8, 8), 64, 0.02, False, global_range=(0.0, 4095.0))


def test_fluorescence_stack_as_uint16_full_size(torch_cuda, orc):
    """The 3-D fluorescence workload read as its uint16 counts (64x512x512,
    kernel 16x64x64, 256 bins, clip 0.02, adaptive range), autotuned shapes."""
    from paper_1906_11355_gb300 import synth

    x = synth.fluorescence_u16((64, 512, 512), seed=1)
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE(x.shape, (16, 64, 64), 256, f32(0.02), True)
    xf = torch_cuda.from_numpy(x.astype(np.float32)).cuda()
    op.autotune(xf)
    run_typed(torch_cuda, orc, x, (16, 64, 64), 256, 0.02, True, shapes=op.shapes())


def test_photoemission_counts_as_uint8_full_size(torch_cuda, orc):
    """The 4-D photoemission workload's counts (at most 74) read as uint8
    (128x128x256x32, kernel 32x32x32x8, 512 bins, clip 0.01, global range)."""
    from paper_1906_11355_gb300 import synth

    xf = synth.photoemission((128, 128, 256, 32), seed=2)
    assert xf.max() <= 255
    run_typed(torch_cuda, orc, xf.astype(np.uint8), (32, 32, 32, 8), 512, 0.01, False)


def test_typed_entry_rejects_unknown_dtype(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE((16, 16), (4, 4), 16, 0.02)
    x = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_forward_typed(op.plan, 7, x, out, op.ws, op.ws_bytes)
    assert e.value.status == nat.MCLAHE_ERR_INVALID_ARG
