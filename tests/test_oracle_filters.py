"""Pins of the pre-filter oracle (oracle/filters.py): scipy.ndimage's Gaussian
and median filters (mode 'reflect', truncate 4), which are the conventions the
oracle takes, plus closed forms and brute-force loops."""
import itertools

import numpy as np
import pytest

from oracle import filters as of


def test_gaussian_matches_scipy():
    from scipy import ndimage

    rng = np.random.default_rng(0)
    for shape, sigma in (((40,), (1.3,)), ((17, 23, 9), (0.7, 0.9, 1.3)), ((6, 7, 8, 9), (0.7, 0.7, 0.9, 1.3)),
                         ((30, 4), (2.5, 0.0))):
        x = rng.gamma(2.0, size=shape)
        want = ndimage.gaussian_filter(x, sigma, mode="reflect", truncate=4.0)
        assert np.abs(of.gaussian(x, sigma) - want).max() <= 1e-12


def test_gaussian_closed_forms():
    w, r = of.gaussian_weights(1.3)
    assert r == 5 and abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w[::-1])
    c = np.full((9, 11), 2.75)
    assert np.abs(of.gaussian(c, (0.9, 1.3)) - 2.75).max() < 1e-14
    # a delta far from the borders returns the weights
    x = np.zeros(41)
    x[20] = 1.0
    assert np.abs(of.gaussian(x, (1.3,))[15:26] - w).max() < 1e-15
    # symmetric normalised weights keep a linear ramp where no tap reaches a border
    ramp = 0.5 + 0.25 * np.arange(40.0)
    assert np.abs(of.gaussian(ramp, (1.3,))[r:-r] - ramp[r:-r]).max() < 1e-12


def test_median_matches_scipy():
    from scipy import ndimage

    rng = np.random.default_rng(1)
    for shape, size in (((19, 21, 7, 5), (2, 2, 2, 1)), ((13, 9), (3, 3)), ((10, 12, 8), (2, 3, 4))):
        x = rng.integers(0, 256, size=shape).astype(np.float64)
        assert np.array_equal(of.median(x, size), ndimage.median_filter(x, size=size, mode="reflect"))


def test_median_brute_force_and_closed_forms():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 50, size=(5, 4, 3)).astype(np.float64)
    size = (2, 3, 2)
    got = of.median(x, size)
    for p in itertools.product(*[range(s) for s in x.shape]):
        vals = []
        for o in itertools.product(*[range(-(k // 2), -(k // 2) + k) for k in size]):
            q = []
            for j, (pj, oj) in enumerate(zip(p, o)):
                i, s = pj + oj, x.shape[j]
                while i < 0 or i >= s:
                    i = -1 - i if i < 0 else 2 * s - 1 - i
                q.append(i)
            vals.append(x[tuple(q)])
        assert got[p] == sorted(vals)[len(vals) // 2]
    assert np.array_equal(of.median(x, (1, 1, 1)), x)
    assert np.array_equal(of.median(np.full((4, 4), 3.0), (2, 2)), np.full((4, 4), 3.0))


def test_fp32_form_is_within_rounding_of_fp64():
    rng = np.random.default_rng(3)
    x = rng.gamma(2.0, size=(9, 10, 11, 12)).astype(np.float32)
    sigma = (0.7, 0.7, 0.9, 1.3)
    a = of.gaussian_fp32(x, sigma).astype(np.float64)
    b = of.gaussian(x, sigma)
    # each pass: at most 2r+1 roundings of terms summing to at most max|x| (weights sum to 1)
    taps = sum(2 * of.gaussian_weights(s)[1] + 2 for s in sigma)
    assert np.abs(a - b).max() <= taps * 2.0 ** -24 * np.abs(x).max() * 1.01


def test_library_gaussian_weights_equal_the_oracle_fp32_weights(nat):
    """mclahe_gaussian_weights is host code (no GPU needed): the same fp32
    weights as the oracle, bit for bit, so the fp32 forms agree exactly."""
    import ctypes

    lib = nat.load()
    for sg in (0.5, 0.7, 0.9, 1.3, 2.0, 3.7):
        w = (ctypes.c_float * 129)()
        r = ctypes.c_int()
        assert lib.mclahe_gaussian_weights(ctypes.c_float(sg), w, 129, ctypes.byref(r)) == 0
        want, rr = of.gaussian_weights_fp32(np.float32(sg))
        assert r.value == rr
        assert np.array_equal(np.frombuffer(w, dtype=np.float32)[:2 * rr + 1], want)
