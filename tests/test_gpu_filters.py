"""The pre-filters (mclahe_filter_gaussian, mclahe_filter_median) against the
oracle, and pre-filter + MCLAHE pipelines of the paper's two cases.

The Gaussian is defined as one exact fp32 evaluation (taps in order, every
product and sum rounded to nearest), which the oracle replays: the results must
be equal bit for bit, so the MCLAHE that follows sees the same intensities on
both sides (exact histograms, output within 1e-5).  The median selects input
values: equal bit for bit."""
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


GAUSS_CASES = [
    ((40,), (1.3,)),
    ((3, 50), (1.3, 0.7)),            # an extent shorter than the radius (repeated reflection)
    ((17, 23, 9), (0.7, 0.9, 1.3)),
    ((9, 10, 11, 12), (0.7, 0.7, 0.9, 1.3)),
    ((12, 1, 30), (0.9, 2.0, 0.0)),   # a dimension of one voxel, one left as it is
]


@pytest.mark.parametrize("shape,sigma", GAUSS_CASES, ids=[str(c[0]) for c in GAUSS_CASES])
def test_gaussian_equals_oracle_bit_for_bit(torch_cuda, shape, sigma):
    torch = torch_cuda
    from oracle import filters as of
    from paper_1906_11355_gb300.api import gaussian_filter

    rng = np.random.default_rng(len(shape))
    x = rng.gamma(2.0, size=shape).astype(np.float32)
    got = gaussian_filter(torch.from_numpy(x).cuda(), sigma).cpu().numpy()
    assert np.array_equal(got, of.gaussian_fp32(x, sigma))


@pytest.mark.parametrize("shape,size", [((19, 21, 7, 5), (2, 2, 2, 1)), ((13, 9), (3, 3)),
                                        ((10, 12, 8), (2, 3, 4)), ((5,), (4,))])
def test_median_equals_oracle(torch_cuda, shape, size):
    torch = torch_cuda
    from oracle import filters as of
    from paper_1906_11355_gb300.api import median_filter

    rng = np.random.default_rng(sum(shape))
    x = rng.integers(0, 256, size=shape).astype(np.float32)
    got = median_filter(torch.from_numpy(x).cuda(), size).cpu().numpy()
    assert np.array_equal(got, of.median(x, size).astype(np.float32))


def test_filters_reject_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat

    x = torch.zeros((8, 8), device="cuda")
    y = torch.zeros((8, 8), device="cuda")
    with pytest.raises(nat.MclaheError):
        nat.mclahe_filter_gaussian(x, x, None, (8, 8), (1.0, 0.0))          # in place
    with pytest.raises(nat.MclaheError):
        nat.mclahe_filter_gaussian(x, y, None, (8, 8), (1.0, 1.0))          # two passes, no tmp
    with pytest.raises(nat.MclaheError):
        nat.mclahe_filter_gaussian(x, y, None, (8, 8), (-1.0, 0.0))
    with pytest.raises(nat.MclaheError):
        nat.mclahe_filter_median(x, y, (8, 8), (6, 6))                      # window above 32


def test_photoemission_pipeline_gaussian_then_mclahe(torch_cuda, orc):
    """Sec. IV.A processing: Gaussian denoising (0.7, 0.7, 0.9, 1.3 along kx,
    ky, E, t), then 4-D CLAHE with an adaptive range, on a photoemission-like
    volume 64x64x128x16 (kernel 16x16x32x4, 256 bins, clip 0.02)."""
    torch = torch_cuda
    from oracle import filters as of
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE, gaussian_filter

    x = synth.photoemission((64, 64, 128, 16), seed=12)
    sigma, ks, nb, clip = (0.7, 0.7, 0.9, 1.3), (16, 16, 32, 4), 256, float(np.float32(0.02))
    xf = gaussian_filter(torch.from_numpy(x).cuda(), sigma)
    op = MCLAHE(x.shape, ks, nb, clip, adaptive=True)
    out = op.forward(xf)
    torch.cuda.synchronize()
    ref_in = of.gaussian_fp32(x, sigma)
    assert np.array_equal(xf.cpu().numpy(), ref_in)
    want, aux = orc.mclahe(ref_in, ks, nb, clip, mode=1, full=True)
    np.testing.assert_array_equal(op.histograms().cpu().numpy(), aux["hist"].astype(np.int64))
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-5


def test_fluorescence_pipeline_median_then_mclahe(torch_cuda, orc):
    """Sec. IV.B processing: median denoising with window (2, 2, 2, 1) of 8-bit
    data, then 4-D CLAHE with a global range, on a fluorescence-like 4-D stack
    (x, y, z, t) = 96x96x40x8 of uint8 counts (kernel 24x24x10x4, 256 bins,
    clip 0.25)."""
    torch = torch_cuda
    from oracle import filters as of
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE, median_filter

    frames = [synth.fluorescence_u16((96, 96, 40), seed=20 + t, peak=200.0, offset=5.0) for t in range(8)]
    x = np.stack(frames, axis=-1).clip(0, 255).astype(np.uint8).astype(np.float32)
    ks, nb, clip = (24, 24, 10, 4), 256, float(np.float32(0.25))
    xm = median_filter(torch.from_numpy(x).cuda(), (2, 2, 2, 1))
    op = MCLAHE(x.shape, ks, nb, clip, adaptive=False)
    out = op.forward(xm)
    torch.cuda.synchronize()
    ref_in = of.median(x, (2, 2, 2, 1)).astype(np.float32)
    assert np.array_equal(xm.cpu().numpy(), ref_in)
    want, aux = orc.mclahe(ref_in, ks, nb, clip, mode=0, full=True)
    np.testing.assert_array_equal(op.histograms().cpu().numpy(), aux["hist"].astype(np.int64))
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-5
