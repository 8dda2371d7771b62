"""End-to-end pins of the oracle (Algorithm 1): the hand-worked example, global
histogram equalisation as a special case, constant images, and symmetries."""
import numpy as np
import pytest

from tests.golden_util import read_golden


def test_hand_worked_1d(orc):
    g = read_golden("hand_1d.txt")
    for clip in ("1.0", "0.5"):
        out = orc.mclahe(g["x"], (int(g["kernel"][0]),), int(g["n_bins"][0]), float(clip),
                         range_=tuple(g["range"]))
        np.testing.assert_allclose(out, g["out_clip_" + clip], rtol=0, atol=1e-15)


def test_hand_worked_as_2d(orc):
    g = read_golden("hand_1d.txt")
    x, nb, r = g["x"], int(g["n_bins"][0]), tuple(g["range"])
    for clip in ("1.0", "0.5"):
        want = g["out_clip_" + clip]
        # one row with a unit kernel along dim 0: the mirror row adds nothing
        out = orc.mclahe(x.reshape(1, 4), (1, 2), nb, float(clip), range_=r)
        np.testing.assert_allclose(out[0], want, atol=1e-15)
        # two equal rows with kernel (2, 2): every count and T double
        out = orc.mclahe(np.stack([x, x]), (2, 2), nb, float(clip), range_=r)
        np.testing.assert_allclose(out, np.stack([want, want]), atol=1e-15)


def _palindromic_tiling(rng, shape, ks, nb, levels=None):
    """Volume tiled with period b by a tile that is symmetric in every dim, so
    that mirror padding continues the tiling and all kernels hold the tile."""
    t = rng.integers(0, nb if levels is None else levels, size=ks)
    for d in range(len(ks)):
        t = np.maximum(t, np.flip(t, axis=d))
    vals = ((t + 0.5) / nb).astype(np.float32)
    reps = [s // b for s, b in zip(shape, ks)]
    return np.tile(vals, reps), vals


@pytest.mark.parametrize("shape,ks", [((24,), (6,)), ((12, 16), (4, 4)), ((8, 6, 10), (4, 2, 5)),
                                      ((6, 4, 6, 4), (3, 2, 3, 2))])
def test_no_clip_equals_global_histogram_equalisation(orc, shape, ks):
    rng = np.random.default_rng(len(shape))
    nb = 16
    x, _ = _palindromic_tiling(rng, shape, ks, nb)
    out = orc.mclahe(x, ks, nb, 1.0, range_=(0.0, 1.0))
    h, _ = np.histogram(x.astype(np.float64), bins=nb, range=(0.0, 1.0))
    c = np.cumsum(h).astype(np.float64)
    he = (c - c[0]) / (c[-1] - c[0])
    bins = np.floor(x.astype(np.float64) * nb).astype(int)
    np.testing.assert_allclose(out, he[bins], rtol=0, atol=1e-13)


def test_adaptive_equals_global_when_every_kernel_spans_the_range(orc):
    rng = np.random.default_rng(9)
    nb = 16
    x, tile = _palindromic_tiling(rng, (12, 20), (4, 5), nb)
    assert tile.min() == x.min() and tile.max() == x.max()
    a = orc.mclahe(x, (4, 5), nb, 0.05, mode=orc.ADAPTIVE)
    b = orc.mclahe(x, (4, 5), nb, 0.05, mode=orc.GLOBAL)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode", [0, 1])
def test_constant_image_maps_to_zero(orc, mode):
    x = np.full((9, 7, 5), 0.3, np.float32)
    for clip in (0.0, 0.01, 0.5, 1.0):
        np.testing.assert_array_equal(orc.mclahe(x, (3, 7, 2), 32, clip, mode=mode), 0.0)


@pytest.mark.parametrize("mode", [0, 1])
def test_transpose_equivariance(orc, mode):
    rng = np.random.default_rng(11)
    x = rng.random((9, 13, 6), dtype=np.float32)
    ks = (4, 5, 3)
    out = orc.mclahe(x, ks, 24, 0.03, mode=mode)
    perm = (2, 0, 1)
    outp = orc.mclahe(np.ascontiguousarray(x.transpose(perm)), tuple(ks[i] for i in perm), 24,
                      0.03, mode=mode)
    np.testing.assert_allclose(outp, out.transpose(perm), rtol=0, atol=1e-14)


@pytest.mark.parametrize("mode", [0, 1])
def test_flip_equivariance_when_padding_is_even(orc, mode):
    # b | s with b even gives p0 = p1, so the kernel grid is symmetric under a
    # flip of each axis and MCLAHE commutes with the flip
    rng = np.random.default_rng(12)
    x = rng.random((8, 12), dtype=np.float32)
    ks = (4, 6)
    out = orc.mclahe(x, ks, 16, 0.02, mode=mode)
    for ax in (0, 1):
        outf = orc.mclahe(np.ascontiguousarray(np.flip(x, ax)), ks, 16, 0.02, mode=mode)
        np.testing.assert_allclose(outf, np.flip(out, ax), rtol=0, atol=1e-14)


def test_unit_dimension_reduces_to_lower_dimension(orc):
    rng = np.random.default_rng(13)
    x = rng.random(37, dtype=np.float32)
    a = orc.mclahe(x, (6,), 20, 0.02)
    b = orc.mclahe(x.reshape(1, 37), (1, 6), 20, 0.02)
    c = orc.mclahe(x.reshape(37, 1, 1), (6, 1, 1), 20, 0.02)
    np.testing.assert_allclose(b.ravel(), a, atol=1e-15)
    np.testing.assert_allclose(c.ravel(), a, atol=1e-15)


def test_output_in_unit_interval(orc):
    rng = np.random.default_rng(14)
    x = rng.gamma(2.0, size=(10, 9, 8)).astype(np.float32)
    for mode in (0, 1):
        out = orc.mclahe(x, (3, 4, 4), 64, 0.01, mode=mode)
        assert out.min() >= 0.0 and out.max() <= 1.0
