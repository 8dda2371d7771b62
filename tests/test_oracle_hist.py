"""Pins of the oracle's histograms (Algorithm 1, steps 3-5; Sec. III.D for the
adaptive range): brute-force counts over numpy-padded kernels, np.histogram on
edge-free data, the exact rational bin, and the voxel-count invariant."""
from fractions import Fraction

import numpy as np
import pytest


def _kernels(padded, ks):
    """Split a padded array into its kernels (C order over the kernel grid)."""
    n = [s // b for s, b in zip(padded.shape, ks)]
    blocks = []
    for k in np.ndindex(*n):
        sl = tuple(slice(kj * b, (kj + 1) * b) for kj, b in zip(k, ks))
        blocks.append(padded[sl])
    return blocks


def _np_pad(orc, x, ks):
    g = orc.geometry(x.shape, ks)
    return np.pad(x, list(zip(g["p0"], g["p1"])), mode="symmetric")


def test_quantiser_special_values(orc):
    # exactly representable edges of [0, 1) with 4 bins: 0.25, 0.5, 0.75
    sc = orc.scale(0.0, 1.0, 4)
    assert sc == 4.0
    for x, j in [(0.0, 0), (0.2, 0), (0.25, 1), (0.5, 2), (0.74, 2), (0.75, 3), (1.0, 3),
                 (-3.0, 0), (7.0, 3)]:
        assert orc.bin_index(x, 0.0, sc, 4) == j
    assert orc.scale(2.0, 2.0, 16) == 0.0          # hi == lo: everything in bin 0
    assert orc.bin_index(2.0, 2.0, 0.0, 16) == 0
    assert orc.bin_index(float("nan"), 0.0, 4.0, 4) == 0


def test_quantiser_close_to_exact_rational_bin(orc):
    rng = np.random.default_rng(5)
    lo, hi, nb = np.float32(0.0123), np.float32(0.9871), 256
    sc = orc.scale(float(lo), float(hi), nb)
    xs = rng.uniform(lo, hi, 4000).astype(np.float32)
    width = Fraction(float(hi)) - Fraction(float(lo))
    off = 0
    for x in xs:
        exact = int((Fraction(float(x)) - Fraction(float(lo))) * nb / width)
        exact = min(max(exact, 0), nb - 1)
        got = orc.bin_index(float(x), float(lo), sc, nb)
        assert abs(got - exact) <= 1
        if got != exact:
            off += 1
            edge = float(lo) + (max(got, exact)) * float(width) / nb
            assert abs(float(x) - edge) < 1e-6
    assert off < 10


@pytest.mark.parametrize("ndim,mode", [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (4, 0), (4, 1)])
def test_histograms_brute_force(orc, ndim, mode):
    rng = np.random.default_rng(100 + 10 * ndim + mode)
    shape = tuple(int(v) for v in rng.integers(3, 11 if ndim < 4 else 7, size=ndim))
    ks = tuple(int(rng.integers(1, s + 1)) for s in shape)
    nb = 8
    x = rng.random(shape, dtype=np.float32)
    hist, lo, sc, n = orc.histograms(x, ks, nb, mode=mode)
    blocks = _kernels(_np_pad(orc, x, ks), ks)
    assert len(blocks) == hist.shape[0] == int(np.prod(n))
    V = int(np.prod(ks))
    for k, blk in enumerate(blocks):
        if mode == 1:
            assert lo[k] == blk.min()
            assert sc[k] == orc.scale(float(blk.min()), float(blk.max()), nb)
        else:
            assert lo[k] == x.min()
            assert sc[k] == orc.scale(float(x.min()), float(x.max()), nb)
        want = np.zeros(nb, dtype=np.uint64)
        for v in blk.ravel():
            want[orc.bin_index(float(v), float(lo[k]), float(sc[k]), nb)] += 1
        np.testing.assert_array_equal(hist[k], want)
        assert int(hist[k].sum()) == V


@pytest.mark.parametrize("ndim", [2, 3])
def test_histograms_match_numpy_histogram(orc, ndim):
    # values at bin centres of [0, 1] so that no value sits near an edge
    rng = np.random.default_rng(7 + ndim)
    nb = 16
    shape = (9, 11) if ndim == 2 else (5, 6, 7)
    ks = (4, 3) if ndim == 2 else (2, 3, 4)
    x = ((rng.integers(0, nb, size=shape) + 0.5) / nb).astype(np.float32)
    x.flat[0], x.flat[1] = 0.0, 1.0   # pin the global range to [0, 1]
    hist, _, _, _ = orc.histograms(x, ks, nb, mode=0)
    for k, blk in enumerate(_kernels(_np_pad(orc, x, ks), ks)):
        want, _ = np.histogram(blk.astype(np.float64), bins=nb, range=(0.0, 1.0))
        np.testing.assert_array_equal(hist[k], want.astype(np.uint64))


def test_given_global_range(orc):
    x = np.linspace(0.0, 1.0, 64, dtype=np.float32).reshape(8, 8)
    hist, lo, sc, _ = orc.histograms(x, (4, 4), 4, mode=0, range_=(0.0, 2.0))
    assert lo[0] == 0.0 and sc[0] == 2.0
    # bin width 0.5: only x = 1.0 (the corner voxel, mirrored into 4 padded
    # voxels of the last kernel) reaches bin 2, and bin 3 stays empty
    assert hist[:, 3].sum() == 0
    assert hist[:, 2].sum() == 4 and hist[-1, 2] == 4
