"""The contrast metrics (mclahe_metrics) and the paper's comparison of D-
dimensional CLAHE on the whole volume against (D-1)-dimensional CLAHE per
frame, against the CPU oracles.

Metrics: mean, STD and MSE within 1e-5 relative of the FP64 oracle (the GPU
sums in compensated fp32 and fp64), entropy within 1e-9 (the bins are the same
integers), PSNR within 1e-4 dB.  The comparison workload is the 4-D
photoemission-like volume stored frame-major (t, kx, ky, E): every frame's
3-D result and the 4-D result must match the MCLAHE oracle, and their metrics
the metrics oracle."""
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


def check_metrics(got, x, ref=None, eps=0.0):
    """got: GPU metrics; x, ref: the oracle's inputs.  eps > 0: the GPU's volume
    differs from x by at most eps per voxel (both normalised to [0, 1] by the
    same min 0 and max 1 of a CLAHE output), which moves the mean and STD by at
    most eps, the MSE by at most 2 eps sqrt(MSE) + eps^2, and the entropy by the
    few voxels that may cross a bin edge."""
    from oracle import metrics as om

    want = om.metrics(x, ref)
    assert got["mean"] == pytest.approx(want["mean"], rel=1e-5, abs=1e-7 + eps)
    assert got["std"] == pytest.approx(want["std"], rel=1e-5, abs=1e-7 + eps)
    assert got["entropy"] == pytest.approx(want["entropy"], rel=1e-9, abs=1e-9 + (1e-3 if eps else 0.0))
    if ref is not None:
        tol = 2 * eps * np.sqrt(want["mse"]) + eps * eps
        assert got["mse"] == pytest.approx(want["mse"], rel=1e-5, abs=1e-9 + tol)
        assert got["psnr"] == pytest.approx(want["psnr"], abs=1e-4 + 10 * np.log10(1 + tol / want["mse"]))


@pytest.mark.parametrize("n", [1, 7, 4096, 1000003])
def test_metrics_match_oracle(torch_cuda, n):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import contrast_metrics

    rng = np.random.default_rng(n)
    x = rng.gamma(2.0, 1.0, size=n).astype(np.float32)
    r = (x + rng.normal(0.0, 0.3, size=n)).astype(np.float32)
    xd, rd = torch.from_numpy(x).cuda(), torch.from_numpy(r).cuda()
    check_metrics(contrast_metrics(xd, rd), x, r)
    check_metrics(contrast_metrics(xd), x)


def test_metrics_constant_and_two_level(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import contrast_metrics

    c = torch.full((64, 64), 2.5, device="cuda")
    m = contrast_metrics(c, c.clone())
    assert m["std"] == 0.0 and m["entropy"] == 0.0 and m["mse"] == 0.0 and m["psnr"] == float("inf")
    t = torch.zeros((32, 32), device="cuda")
    t[:, :16] = 1.0
    m = contrast_metrics(t, 1.0 - t)
    assert m["std"] == pytest.approx(0.5) and m["entropy"] == pytest.approx(1.0) and m["mse"] == 1.0


def test_metrics_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat

    x = torch.zeros(100, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    ws = torch.empty(nat.mclahe_metrics_workspace_bytes(100), dtype=torch.uint8, device="cuda")
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_metrics(x, x, 100, ws, ws.numel(), out)
    assert e.value.status == nat.MCLAHE_ERR_INVALID_ARG
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_metrics(x, None, 100, ws, 8, out)
    assert e.value.status == nat.MCLAHE_ERR_WORKSPACE


@pytest.mark.parametrize("shape,ks,adaptive", [
    ((6, 16, 20, 24), (3, 4, 5, 8), False),
    ((5, 12, 16, 20), (5, 6, 8, 10), True),
])
def test_frames_vs_volume_small(torch_cuda, orc, shape, ks, adaptive):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import compare_frames_vs_volume

    rng = np.random.default_rng(sum(shape))
    x = rng.poisson(rng.uniform(0.2, 20.0, size=shape)).astype(np.float32)
    clip = float(np.float32(0.02))
    out_v, out_f, m = compare_frames_vs_volume(torch.from_numpy(x).cuda(), ks, 64, clip, adaptive)
    want_v = orc.mclahe(x, ks, 64, clip, mode=int(adaptive))
    assert np.abs(out_v.cpu().numpy() - want_v).max() <= 1e-5
    want_f = np.stack([orc.mclahe(x[t], ks[1:], 64, clip, mode=int(adaptive)) for t in range(shape[0])])
    assert np.abs(out_f.cpu().numpy() - want_f).max() <= 1e-5
    check_metrics(m["volume"], want_v.astype(np.float32), x, eps=1e-5)
    check_metrics(m["frames"], want_f.astype(np.float32), x, eps=1e-5)
    check_metrics(m["input"], x)


def test_frames_vs_volume_photoemission_workload(torch_cuda, orc):
    """The comparison of Sec. IV.A on the synthetic photoemission volume stored
    frame-major, 32 x 128 x 128 x 256 (t, kx, ky, E): 4-D CLAHE with kernel
    8 x 32 x 32 x 32 against 3-D CLAHE of each of the 32 frames with kernel
    32 x 32 x 32; 512 bins, clip 0.01, global range."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import compare_frames_vs_volume

    x = np.ascontiguousarray(np.moveaxis(synth.photoemission((128, 128, 256, 32), seed=2), -1, 0))
    ks, nb, clip = (8, 32, 32, 32), 512, float(np.float32(0.01))
    out_v, out_f, m = compare_frames_vs_volume(torch.from_numpy(x).cuda(), ks, nb, clip, False)
    want_v = orc.mclahe(x, ks, nb, clip, mode=0)
    assert np.abs(out_v.cpu().numpy() - want_v).max() <= 1e-5
    got_f = out_f.cpu().numpy()
    want_f = np.empty_like(got_f)
    for t in range(x.shape[0]):
        want_f[t] = orc.mclahe(x[t], ks[1:], nb, clip, mode=0)
    assert np.abs(got_f - want_f).max() <= 1e-5
    check_metrics(m["volume"], want_v.astype(np.float32), x, eps=1e-5)
    check_metrics(m["frames"], want_f, x, eps=1e-5)
