"""Contrast metrics of the paper's comparisons, plain numpy in FP64 (the CPU
oracle of mclahe_metrics; test infrastructure only: nothing on the product
path imports it).

The paper compares its results with four classic metrics (Sec. II; Tables I
and II, Sec. IV): the mean squared error to the original data (MSE), the peak
signal-to-noise ratio derived from it (PSNR), the standard deviation
(root-mean-square contrast, STD) and the Shannon (grey-level) entropy (ENT).
It does not print their formulas.  Readings taken here:
  - every volume is first normalised to [0, 1] by its own minimum and maximum
    (a constant volume becomes all zeros), since MCLAHE's output lies in
    [0, 1] and the tables compare it with the raw data;
  - MSE = mean((a - b)^2) of the normalised volumes;
  - PSNR = 10 log10(peak^2 / MSE) with peak = 2^23: every PSNR in Tables I
    and II follows from its row's MSE with that peak (tests/golden/psnr_tables.txt);
  - STD = the population standard deviation (1/N) of the normalised volume;
  - ENT = -sum_i p_i log2 p_i over a 256-bin histogram of the volume over its
    own [min, max], binned with the quantiser MCLAHE itself uses (fp32:
    floor((x - lo) * (256 / (hi - lo))), clamped to [0, 255]).
Parity pinned by: the PSNR/MSE relation of the tables, closed forms on small
arrays (constant, two-level and uniform-ramp volumes), and brute-force loops.
"""
from __future__ import annotations

import numpy as np

PSNR_PEAK = 2.0 ** 23


def normalise(x):
    """x scaled to [0, 1] by its own min and max (FP64; all zeros if constant)."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = x.min(), x.max()
    if hi > lo:
        return (x - lo) / (hi - lo)
    return np.zeros_like(x)


def mse(a, b):
    """Mean squared error of the normalised volumes."""
    return float(np.mean((normalise(a) - normalise(b)) ** 2))


def psnr(mse_value):
    """Peak signal-to-noise ratio (dB) of an MSE, peak 2^23 (inf for MSE 0)."""
    if mse_value <= 0.0:
        return float("inf")
    return float(10.0 * np.log10(PSNR_PEAK * PSNR_PEAK / mse_value))


def std(a):
    """Population standard deviation of the normalised volume."""
    return float(np.std(normalise(a)))


def bins_fp32(a, n_bins=256):
    """Bin of every voxel over the volume's own [min, max] with the fp32
    quantiser of Algorithm 1's histograms: scale = fp32(n_bins / (hi - lo))
    (0 if hi == lo), bin = clamp(floor(fp32(fp32(x - lo) * scale)), 0, n_bins - 1)."""
    x = np.asarray(a, dtype=np.float32)
    lo, hi = np.float32(x.min()), np.float32(x.max())
    if hi > lo:
        scale = np.float32(np.float32(n_bins) / np.float32(hi - lo))
    else:
        scale = np.float32(0.0)
    y = (x - lo).astype(np.float32) * scale
    return np.clip(np.floor(y.astype(np.float32)), 0, n_bins - 1).astype(np.int64)


def entropy(a, n_bins=256):
    """Shannon entropy (bits) of the volume's n_bins-bin grey-level histogram."""
    counts = np.bincount(bins_fp32(a, n_bins).ravel(), minlength=n_bins).astype(np.float64)
    p = counts[counts > 0] / counts.sum()
    return float(-(p * np.log2(p)).sum())


def metrics(x, ref=None, n_bins=256):
    """All four for x (MSE and PSNR against ref when given), as a dict."""
    out = {"std": std(x), "entropy": entropy(x, n_bins), "mean": float(np.mean(normalise(x)))}
    if ref is not None:
        m = mse(x, ref)
        out["mse"] = m
        out["psnr"] = psnr(m)
    return out
