"""Pins of the contrast-metric oracle (oracle/metrics.py) against the paper and
closed forms.

PSNR: every (MSE, PSNR) pair of Tables I and II (tests/golden/psnr_tables.txt)
must satisfy PSNR = 10 log10((2^23)^2 / MSE) within the printed rounding of
both numbers -- the peak the tables imply.  STD, ENT and MSE: constant,
two-level and ramp volumes with known values, and brute-force loops."""
import math
import os

import numpy as np
import pytest

from oracle import metrics as om

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "psnr_tables.txt")


def table_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, name, m, md, p, pd = line.split()
        rows.append((t, name, float(m), int(md), float(p), int(pd)))
    return rows


@pytest.mark.parametrize("row", table_rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_psnr_reproduces_the_tables_from_their_mse(row):
    _, _, m, md, p, pd = row
    h = 0.5 * 10.0 ** -md          # half a unit of the printed MSE
    lo_p, hi_p = om.psnr(m + h), om.psnr(m - h)
    assert lo_p - 0.5 * 10.0 ** -pd <= p <= hi_p + 0.5 * 10.0 ** -pd, (m, p, lo_p, hi_p)


def test_psnr_rejects_other_peaks():
    # a peak of 1 (the usual normalised-image convention) misses every table value
    for _, _, m, _, p, _ in table_rows():
        assert abs(10.0 * math.log10(1.0 / m) - p) > 100.0


def test_constant_volume():
    x = np.full((5, 7), 3.25, np.float32)
    assert om.std(x) == 0.0 and om.entropy(x) == 0.0 and om.mse(x, x) == 0.0
    assert om.psnr(0.0) == float("inf")


def test_two_level_volume():
    x = np.zeros((8, 8), np.float32)
    x[:, :4] = 5.0
    assert om.std(x) == pytest.approx(0.5, abs=1e-15)
    assert om.entropy(x) == pytest.approx(1.0, abs=1e-15)
    assert om.mse(x, 5.0 - x) == pytest.approx(1.0, abs=1e-15)   # the inverse image


def test_ramp_of_256_levels():
    x = np.arange(256, dtype=np.float32).reshape(16, 16)
    assert np.array_equal(np.sort(om.bins_fp32(x).ravel()), np.arange(256))
    assert om.entropy(x) == pytest.approx(8.0, abs=1e-12)
    want = math.sqrt((256 ** 2 - 1) / 12.0) / 255.0
    assert om.std(x) == pytest.approx(want, rel=1e-12)


def test_brute_force_small():
    rng = np.random.default_rng(1)
    a = rng.gamma(2.0, size=(3, 4, 5)).astype(np.float32)
    b = rng.gamma(2.0, size=(3, 4, 5)).astype(np.float32)
    fa, fb = [float(v) for v in a.ravel()], [float(v) for v in b.ravel()]
    na = [(v - min(fa)) / (max(fa) - min(fa)) for v in fa]
    nb_ = [(v - min(fb)) / (max(fb) - min(fb)) for v in fb]
    n = len(na)
    mean = sum(na) / n
    assert om.std(a) == pytest.approx(math.sqrt(sum((v - mean) ** 2 for v in na) / n), rel=1e-12)
    assert om.mse(a, b) == pytest.approx(sum((u - v) ** 2 for u, v in zip(na, nb_)) / n, rel=1e-12)
    # bins: fp32 quantiser written out per voxel
    lo, hi = np.float32(min(fa)), np.float32(max(fa))
    sc = np.float32(np.float32(256) / np.float32(hi - lo))
    counts = [0] * 256
    for v in a.ravel():
        k = int(np.floor(np.float32(np.float32(v - lo) * sc)))
        counts[min(max(k, 0), 255)] += 1
    ent = -sum(c / n * math.log2(c / n) for c in counts if c)
    assert om.entropy(a) == pytest.approx(ent, rel=1e-12)
