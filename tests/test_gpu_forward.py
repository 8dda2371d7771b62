"""Parity of the CUDA forward path (through the C ABI) with the FP64 oracle.

Histograms and ranges must match bit for bit, mapping tables to 1e-6 and the
output to 1e-5 max-abs (the output lies in [0, 1]).  Small cases span several
kernels and ragged tails in 1-4 dimensions; the workload cases run the full
synthetic volumes in the launch configuration the benchmark times."""
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


def run_case(torch, orc, x, ks, nb, clip, adaptive=False, global_range=None):
    from paper_1906_11355_gb300.api import MCLAHE

    clip = f32(clip)
    op = MCLAHE(x.shape, ks, n_bins=nb, clip_limit=clip, adaptive=adaptive,
                global_range=global_range)
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


@pytest.mark.parametrize("name", WORKLOADS)
def test_workload_full_size(torch_cuda, orc, name):
    from paper_1906_11355_gb300 import synth

    w = synth.WORKLOADS[name]
    x = synth.make_volume(w["gen"], w["shape"], w["seed"])
    run_case(torch_cuda, orc, x, w["kernel"], w["n_bins"], w["clip_limit"], w["adaptive"])
