"""Pre-filters the paper applies before MCLAHE, plain numpy in FP64 (the CPU
oracle of mclahe_filter_gaussian and mclahe_filter_median; test infrastructure
only: nothing on the product path imports it).

Sec. IV.A denoises the photoemission data with a Gaussian filter (standard
deviations per dimension) and Sec. IV.B the fluorescence data with a median
filter of window (2, 2, 2, 1).  The paper does not define the boundary, the
truncation or the median of an even window; readings taken here:
  - boundary: the edge-inclusive mirror (index j < 0 -> -1 - j, j >= s ->
    2 s - 1 - j, reflected as often as needed), the same mirror as MCLAHE's
    padding (Sec. III.B);
  - Gaussian: separable, dimension 0 first; along a dimension with sigma > 0
    the weights w_k = exp(-k^2 / (2 sigma^2)), |k| <= r, r = floor(4 sigma +
    0.5), divided by their sum; sigma = 0 leaves that dimension as it is;
  - median: window [x - floor(k/2), x - floor(k/2) + k - 1] along each
    dimension; the element of rank floor(n / 2) (0-based) of the n window
    values in ascending order (the upper median when n is even).
These are the conventions of scipy.ndimage (mode 'reflect'), which pins them
(tests/test_oracle_filters.py), as do closed forms.
"""
from __future__ import annotations

import itertools

import numpy as np


def mirror_index(j, s):
    """Edge-inclusive mirror of index j into [0, s)."""
    period = 2 * s
    j = j % period
    return np.where(j < s, j, period - 1 - j)


def gaussian_weights(sigma):
    """Normalised 1-D weights of radius floor(4 sigma + 0.5) (FP64)."""
    r = int(4.0 * float(sigma) + 0.5)
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * float(sigma) * float(sigma)))
    return w / w.sum(), r


def gaussian(x, sigma):
    """Separable Gaussian of x (FP64 result), one sigma per dimension."""
    y = np.asarray(x, dtype=np.float64)
    for d, sg in enumerate(sigma):
        if sg <= 0:
            continue
        w, r = gaussian_weights(sg)
        s = y.shape[d]
        acc = np.zeros_like(y)
        for i, k in enumerate(range(-r, r + 1)):
            idx = mirror_index(np.arange(s) + k, s)
            acc += w[i] * np.take(y, idx, axis=d)
        y = acc
    return y


def gaussian_weights_fp32(sigma):
    """The fp32 weights the exact form uses: sigma taken as an fp32 value (the
    interface passes it as float), the FP64 weights of it rounded to fp32."""
    w, r = gaussian_weights(float(np.float32(sigma)))
    return w.astype(np.float32), r


def gaussian_fp32(x, sigma):
    """The Gaussian evaluated exactly as the fp32 form defines it: dimension by
    dimension, each output the fp32 sum over the taps k = -r..r, in that order,
    of fp32(w_k * x), every product and sum rounded to nearest (numpy float32
    arithmetic).  Within fp32 rounding of gaussian() (tests pin the bound)."""
    y = np.asarray(x, dtype=np.float32)
    for d, sg in enumerate(sigma):
        if sg <= 0:
            continue
        w, r = gaussian_weights_fp32(sg)
        s = y.shape[d]
        acc = np.zeros(y.shape, dtype=np.float32)
        for i, k in enumerate(range(-r, r + 1)):
            idx = mirror_index(np.arange(s) + k, s)
            acc = (acc + (w[i] * np.take(y, idx, axis=d)).astype(np.float32)).astype(np.float32)
        y = acc
    return y


def median(x, size):
    """Median filter of x with window `size` (FP64 result; values of x exactly)."""
    y = np.asarray(x, dtype=np.float64)
    shape = y.shape
    offs = [range(-(k // 2), -(k // 2) + k) for k in size]
    stack = []
    for o in itertools.product(*offs):
        idx = [mirror_index(np.arange(s) + oj, s) for s, oj in zip(shape, o)]
        stack.append(y[np.ix_(*idx)])
    v = np.sort(np.stack(stack), axis=0)
    return v[len(stack) // 2]
