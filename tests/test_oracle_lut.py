"""Pins of the oracle's clip / redistribute / CDF / normalise step (Algorithm 1,
steps 6-8): textbook histogram equalisation with no clipping, closed forms,
mass conservation and the shape of the normalised mapping."""
import numpy as np
import pytest

from tests.golden_util import read_golden


def test_no_clip_is_textbook_equalisation(orc):
    # clip_limit = 1 means T = V: no bin can exceed it, so the mapping is the
    # plain normalised CDF of the kernel (Hall's histogram equalisation).
    rng = np.random.default_rng(1)
    for _ in range(20):
        nb = int(rng.integers(2, 40))
        h = rng.integers(0, 50, size=nb).astype(np.uint64)
        V = int(h.sum())
        if V == 0 or V == h[0]:
            continue
        c = np.cumsum(h.astype(np.float64))
        want = (c - c[0]) / (c[-1] - c[0])
        np.testing.assert_allclose(orc.clip_lut(h, V, 1.0), want, rtol=0, atol=1e-15)


def test_single_bin_mass(orc):
    # all V voxels in bin 0: clipping at T < V leaves E = V - T spread evenly,
    # so the mapping is j / (nb - 1); without clipping the CDF is constant
    # and the mapping is 0 everywhere.
    nb, V = 10, 64
    h = np.zeros(nb, dtype=np.uint64)
    h[0] = V
    np.testing.assert_allclose(orc.clip_lut(h, V, 0.25), np.arange(nb) / (nb - 1), atol=1e-15)
    np.testing.assert_array_equal(orc.clip_lut(h, V, 1.0), np.zeros(nb))


@pytest.mark.parametrize("clip", [0.0, 0.003, 0.01, 0.02, 0.1, 0.5, 0.999])
def test_clip_invariants(orc, clip):
    rng = np.random.default_rng(int(clip * 1e4) + 3)
    nb = 64
    for _ in range(10):
        h = rng.geometric(0.08, size=nb).astype(np.uint64) * rng.integers(0, 2, size=nb).astype(np.uint64)
        h[rng.integers(0, nb)] += 400
        V = int(h.sum())
        lut, hc = orc.clip_lut(h, V, clip, with_clipped=True)
        T = clip * V
        assert abs(hc.sum() - V) < 1e-9 * V               # mass conserved
        share = hc - np.minimum(h.astype(np.float64), T)   # equal share E / nb
        np.testing.assert_allclose(share, share[0], atol=1e-9)
        E = np.maximum(h.astype(np.float64) - T, 0).sum()
        assert abs(share[0] - E / nb) < 1e-9
        assert lut[0] == 0.0 and abs(lut[-1] - 1.0) < 1e-15
        assert np.all(np.diff(lut) >= 0) and lut.min() >= 0 and lut.max() <= 1


def test_hand_example_tables(orc):
    g = read_golden("hand_1d.txt")
    x = g["x"]
    nb = int(g["n_bins"][0])
    V = int(g["kernel"][0])
    # the three kernel histograms of the worked example
    hists = [np.array([2, 0, 0, 0], np.uint64), np.array([0, 1, 1, 0], np.uint64),
             np.array([0, 0, 0, 2], np.uint64)]
    for clip in ("1.0", "0.5"):
        want = g["lut_clip_" + clip].reshape(3, nb)
        for k in range(3):
            np.testing.assert_allclose(orc.clip_lut(hists[k], V, float(clip)), want[k], atol=1e-15)
    hist, _, _, _ = orc.histograms(x, (V,), nb, mode=0, range_=tuple(g["range"]))
    np.testing.assert_array_equal(hist, np.stack(hists))
