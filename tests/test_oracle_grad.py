"""Pins of the oracle's gradient (reverse mode of Algorithm 1 with respect to
the mapping tables and clip_limit): a hand-derived closed form of d lut / d T,
central finite differences of the forward away from kinks, and exactness of
the table gradient (the mapping is linear in the tables)."""
import numpy as np
import pytest


def _closed_form_dlut_dT(h, T):
    # lut_j = (C_j - C_0) / (V - C_0), C_j = sum_{i<=j} min(h_i, T) + (j+1) E / nb,
    # E = sum_{h>T} (h - T).  With A_j = #{i <= j : h_i > T} and N_c = A_{nb-1}:
    # dC_j/dT = A_j - (j+1) N_c / nb (derived by hand, independent of the
    # oracle's reverse-mode sweep).
    h = h.astype(np.float64)
    nb = len(h)
    V = h.sum()
    clipped = h > T
    A = np.cumsum(clipped)
    Nc = A[-1]
    E = (h[clipped] - T).sum()
    C = np.cumsum(np.minimum(h, T)) + (np.arange(nb) + 1) * E / nb
    j = np.arange(nb)
    num = (A - A[0] - j * Nc / nb) * (V - C[0]) + (C - C[0]) * (A[0] - Nc / nb)
    return num / (V - C[0]) ** 2


def test_lut_backward_matches_closed_form(orc):
    rng = np.random.default_rng(21)
    for _ in range(30):
        nb = int(rng.integers(4, 50))
        h = rng.integers(0, 60, size=nb).astype(np.uint64)
        V = int(h.sum())
        if V == 0:
            continue
        clip = float(rng.uniform(0.0, 0.6))
        T = clip * V
        if np.any(np.abs(h.astype(np.float64) - T) < 1e-9):
            continue
        want = _closed_form_dlut_dT(h, T)
        for j in range(nb):
            gl = np.zeros(nb)
            gl[j] = 1.0
            assert abs(orc.lut_backward(h, V, clip, gl) - want[j]) < 1e-12


def test_lut_backward_matches_finite_differences(orc):
    rng = np.random.default_rng(22)
    nb, eps = 32, 1e-6
    for _ in range(10):
        h = rng.integers(0, 100, size=nb).astype(np.uint64)
        V = int(h.sum())
        clip = float(rng.uniform(0.01, 0.2))
        if np.any(np.abs(h.astype(np.float64) - clip * V) < 2 * eps * V):
            continue
        gl = rng.normal(size=nb)
        fd = (gl @ orc.clip_lut(h, V, clip + eps) - gl @ orc.clip_lut(h, V, clip - eps)) / (2 * eps)
        assert abs(V * orc.lut_backward(h, V, clip, gl) - fd) < 1e-6 * max(1.0, abs(fd))


def _kink_free_clip(hist, V, lo, hi, h_step, rng):
    counts = np.unique(hist.astype(np.float64))
    for _ in range(1000):
        c = float(rng.uniform(lo, hi))
        if np.min(np.abs(counts - c * V)) > 1.5 * h_step * V:
            return c
    raise AssertionError("no kink-free clip value found")


@pytest.mark.parametrize("mode,shape,ks", [(0, (24, 20), (6, 5)), (1, (10, 12, 9), (4, 4, 3)),
                                           (0, (8, 6, 8, 4), (4, 3, 4, 2))])
def test_clip_gradient_matches_finite_differences(orc, mode, shape, ks):
    rng = np.random.default_rng(23 + mode)
    x = rng.gamma(2.0, size=shape).astype(np.float32)
    nb, h = 16, 1e-5
    hist, _, _, _ = orc.histograms(x, ks, nb, mode=mode)
    V = int(np.prod(ks))
    clip = _kink_free_clip(hist, V, 0.02, 0.3, h, rng)
    g = rng.normal(size=shape)
    _, gc = orc.mclahe_backward(x, ks, nb, clip, g, mode=mode)
    fd = (np.sum(g * orc.mclahe(x, ks, nb, clip + h, mode=mode))
          - np.sum(g * orc.mclahe(x, ks, nb, clip - h, mode=mode))) / (2 * h)
    assert abs(gc - fd) <= 1e-5 * max(1.0, abs(fd))
    assert abs(gc) > 1e-3          # the check is not vacuous


@pytest.mark.parametrize("mode", [0, 1])
def test_table_gradient_is_exact(orc, mode):
    # out = map(lut) is linear in lut, so <grad_lut, d> = sum(g * map(d))
    rng = np.random.default_rng(31 + mode)
    shape, ks, nb = (9, 11, 5), (3, 4, 2), 12
    x = rng.random(shape, dtype=np.float32)
    g = rng.normal(size=shape)
    gl, _ = orc.mclahe_backward(x, ks, nb, 0.05, g, mode=mode)
    _, lo, sc, n = orc.histograms(x, ks, nb, mode=mode)
    for _ in range(5):
        d = rng.normal(size=gl.shape)
        lhs = float(np.sum(gl * d))
        rhs = float(np.sum(g * orc.map_volume(x, ks, d, lo, sc)))
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(rhs))
