"""Pins of the oracle's multilinear mapping (Sec. III.C, Eq. (12)-(13)) against
scipy's RegularGridInterpolator over the grid of kernel centres."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator


def _centres(orc, shape, ks):
    g = orc.geometry(shape, ks)
    grid = [np.arange(n) * b + (b - 1) / 2.0 for n, b in zip(g["n"], ks)]
    return g, grid


def _positions(g, shape):
    idx = np.indices(shape).reshape(len(shape), -1).T.astype(np.float64)
    return idx + np.asarray(g["p0"], dtype=np.float64)


@pytest.mark.parametrize("ndim", [1, 2, 3, 4])
def test_global_range_map_is_multilinear_interpolation(orc, ndim):
    rng = np.random.default_rng(40 + ndim)
    shape = tuple(int(v) for v in rng.integers(4, 12 if ndim < 4 else 7, size=ndim))
    ks = tuple(int(rng.integers(1, s + 1)) for s in shape)
    nb = 6
    g, grid = _centres(orc, shape, ks)
    K = int(np.prod(g["n"]))
    lut = rng.random((K, nb))
    x = rng.random(shape, dtype=np.float32)
    lo = np.zeros(K, np.float32)
    sc = np.full(K, orc.scale(0.0, 1.0, nb), np.float32)
    out = orc.map_volume(x, ks, lut, lo, sc).ravel()
    bins = np.array([orc.bin_index(float(v), 0.0, float(sc[0]), nb) for v in x.ravel()])
    pos = _positions(g, shape)
    want = np.empty_like(out)
    for j in range(nb):
        sel = bins == j
        if sel.any():
            f = RegularGridInterpolator(grid, lut[:, j].reshape(g["n"]), method="linear")
            want[sel] = f(pos[sel])
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
def test_adaptive_range_map_uses_each_neighbours_range(orc, ndim):
    # With mapping[k][j] = j / nb for every kernel, the output at voxel v is
    # the interpolation over the kernel centres of bin_k(v) / nb, where each
    # kernel k quantises v with its own range.
    rng = np.random.default_rng(60 + ndim)
    shape = (7, 9) if ndim == 2 else (5, 6, 7)
    ks = (3, 4) if ndim == 2 else (2, 3, 4)
    nb = 32
    g, grid = _centres(orc, shape, ks)
    K = int(np.prod(g["n"]))
    lo = rng.uniform(0.0, 0.4, K).astype(np.float32)
    hi = rng.uniform(0.6, 1.0, K).astype(np.float32)
    sc = np.array([orc.scale(float(a), float(b), nb) for a, b in zip(lo, hi)], np.float32)
    lut = np.tile(np.arange(nb) / nb, (K, 1))
    x = rng.random(shape, dtype=np.float32)
    out = orc.map_volume(x, ks, lut, lo, sc).ravel()
    pos = _positions(g, shape)
    for q, v in enumerate(x.ravel()):
        vals = np.array([orc.bin_index(float(v), float(lo[k]), float(sc[k]), nb) / nb
                         for k in range(K)]).reshape(g["n"])
        want = RegularGridInterpolator(grid, vals, method="linear")(pos[q:q + 1])[0]
        assert abs(out[q] - want) < 1e-12


def test_constant_tables_give_constant_output(orc):
    # the Lagrange coefficients of Eq. (13) sum to one
    rng = np.random.default_rng(3)
    shape, ks, nb = (6, 5, 7, 4), (2, 5, 3, 3), 5
    g = orc.geometry(shape, ks)
    K = int(np.prod(g["n"]))
    x = rng.random(shape, dtype=np.float32)
    out = orc.map_volume(x, ks, np.full((K, nb), 0.625), np.zeros(K, np.float32),
                         np.full(K, 5.0, np.float32))
    np.testing.assert_allclose(out, 0.625, rtol=0, atol=1e-14)
