"""The mapping kernels' folded bin quantiser gives the same bins as the
unfolded one wherever they use it (host-side check of the arithmetic).

The histogram step of Algorithm 1 bins a voxel as floor((x - lo) * scale),
clamped, with both operations rounded to float32.  The kernels evaluate it
as t = sat(fp32(y * 2^-k)), bin = floor(t * 2^k), y = fp32(fp32(x - lo) *
scale).  With an adaptive range the mapping folds 2^-k into the scale
(t = sat(fp32(fp32(x - lo) * fp32(scale * 2^-k)))) when scale is zero or
non-finite or the exact product scale * 2^-k is a normal number
(|scale| >= 2^-126 * 2^k).  This test emulates both forms in IEEE float32
(numpy rounds to nearest even and keeps subnormals) and checks that they give
the same bin on random and edge inputs whenever that condition holds.
"""
import numpy as np
import pytest

F32_MIN_NORMAL = np.float32(1.17549435e-38)


def sat(t):
    t = np.where(np.isnan(t), np.float32(0), t)
    return np.clip(t, np.float32(0), np.float32(1)).astype(np.float32)


def bins_unfolded(x, lo, sc, qk):
    with np.errstate(all="ignore"):
        y = (x - lo).astype(np.float32) * sc
        t = sat((y * np.float32(1.0 / qk)).astype(np.float32))
    return np.floor(t.astype(np.float64) * qk).astype(np.int64)


def bins_folded(x, lo, sc, qk):
    with np.errstate(all="ignore"):
        scq = np.float32(sc * np.float32(1.0 / qk))
        t = sat(((x - lo).astype(np.float32) * scq).astype(np.float32))
    return np.floor(t.astype(np.float64) * qk).astype(np.int64)


def fold_exact(sc, qk):
    # the exact product sc * 2^-k must be normal: |sc| >= 2^-126 * qk
    return sc == 0 or not (abs(sc) < np.float32(F32_MIN_NORMAL * np.float32(qk)))


def fold_exact_rounded(sc, qk):
    # a check on the rounded product (too weak: it can round up to 2^-126)
    with np.errstate(all="ignore"):
        scq = np.float32(sc * np.float32(1.0 / qk))
    return sc == 0 or not (abs(scq) < F32_MIN_NORMAL)


@pytest.mark.parametrize("qk", [1, 2, 128, 256, 512, 4096])
def test_folded_bins_equal_unfolded(qk):
    rng = np.random.default_rng(1234 + qk)
    n_bins = qk + 1 if qk > 1 else 2
    checked = 0
    for _ in range(400):
        # ranges from tiny to huge, the voxels inside, around and far outside them
        e_lo = rng.uniform(-40, 38)
        lo = np.float32(rng.choice([-1, 1]) * 10.0 ** e_lo)
        width = np.float32(10.0 ** rng.uniform(-44, 38))
        hi = np.float32(lo + width)
        if not np.isfinite(hi) or not hi > lo:
            continue
        with np.errstate(all="ignore"):
            sc = np.float32(np.float32(n_bins) / np.float32(hi - lo))
        if not fold_exact(sc, qk):
            continue
        x = np.concatenate([
            lo + (hi - lo) * rng.random(2000, dtype=np.float32),
            np.array([lo, hi, np.nextafter(lo, np.float32(-np.inf)), np.nextafter(hi, np.float32(np.inf)),
                      np.float32(0), np.float32(-0.0), np.float32(np.inf), np.float32(-np.inf),
                      np.float32(np.nan), np.float32(3.0e38), np.float32(-3.0e38)], dtype=np.float32),
            (lo + (hi - lo) * np.float32(1 + 4 * rng.random(200, dtype=np.float32))).astype(np.float32),
        ]).astype(np.float32)
        a, b = bins_unfolded(x, lo, sc, qk), bins_folded(x, lo, sc, qk)
        np.testing.assert_array_equal(a, b, err_msg=f"lo={lo!r} hi={hi!r} sc={sc!r} qk={qk}")
        checked += 1
    assert checked > 100


def test_fold_condition_edge_scales():
    # zero and non-finite scales fold exactly; a scale whose fold is subnormal does not
    assert fold_exact(np.float32(0), 256)
    assert fold_exact(np.float32(np.inf), 256)
    assert fold_exact(np.float32(np.nan), 256)
    assert fold_exact(np.float32(2.0 ** -100), 256)
    assert not fold_exact(np.float32(2.0 ** -120), 256)
    # at the boundary: scale * 2^-8 is the smallest normal number
    assert fold_exact(np.float32(2.0 ** -118), 256)
    below = np.float32(np.nextafter(np.float32(2.0 ** -118), np.float32(0)))
    assert not fold_exact(below, 256)
    # the product of the float just below rounds (ties to even) up to 2^-126,
    # so a check on the rounded product would wrongly accept it
    with np.errstate(all="ignore"):
        assert np.float32(below * np.float32(1.0 / 256)) == F32_MIN_NORMAL
    assert fold_exact_rounded(below, 256)
    # and folding it would change a bin: (x - lo) = 3.32307e35 is bin 0 with
    # the two roundings of the histogram step but bin 1 after the fold
    d = np.array([np.float32(3.32307e35)], dtype=np.float32)
    zero = np.float32(0)
    assert bins_unfolded(d, zero, below, 256)[0] == 0
    assert bins_folded(d, zero, below, 256)[0] == 1


def test_unfolded_matches_the_rational_bin_on_exact_inputs():
    # on voxels where every float32 step is exact the quantiser is the plain
    # floor((x - lo) * scale) of the histogram step, clamped to [0, qk]
    qk, lo, sc = 256, np.float32(-3.0), np.float32(4.0)
    x = (lo + np.arange(0, 80, dtype=np.float32) / np.float32(4)).astype(np.float32)
    expect = np.clip(np.floor((x.astype(np.float64) - float(lo)) * float(sc)), 0, qk).astype(np.int64)
    np.testing.assert_array_equal(bins_unfolded(x, lo, sc, qk), expect)
    np.testing.assert_array_equal(bins_folded(x, lo, sc, qk), expect)
