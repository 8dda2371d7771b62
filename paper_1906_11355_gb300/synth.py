"""Seeded synthetic volumes shaped like the paper's workloads.

The paper's datasets (4D photoemission spectroscopy of WSe2, Sec. IV.A, and 4D
fluorescence microscopy of an ascidian embryo, Sec. IV.B) are not available,
so these generators stand in for them.  This module only draws inputs; it
holds none of MCLAHE's arithmetic and is shared by the tests, the benchmark
and any user who wants reproducible inputs.

Every generator takes a seed and uses ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np


def smooth_field(shape=(512, 512), seed=0, n_gauss=20, sigma=(20.0, 80.0), scale=0.6,
                 noise_sd=0.02):
    """Sum of isotropic Gaussians (sigma uniform in ``sigma`` pixels, amplitude
    U[0,1], centres uniform over the volume), normalised to [0,1], times
    ``scale``, plus Gaussian noise, clipped to [0,1].  float32."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    field = np.zeros(shape, dtype=np.float64)
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    for _ in range(n_gauss):
        amp = rng.uniform(0.0, 1.0)
        sig = rng.uniform(*sigma)
        centre = [rng.uniform(0, s) for s in shape]
        g = None
        for d, ax in enumerate(axes):
            e = np.exp(-((ax - centre[d]) ** 2) / (2.0 * sig * sig))
            e = e.reshape([-1 if i == d else 1 for i in range(len(shape))])
            g = e if g is None else g * e
        field += amp * g
    lo, hi = field.min(), field.max()
    field = (field - lo) / (hi - lo) if hi > lo else np.zeros_like(field)
    field = field * scale + rng.normal(0.0, noise_sd, size=shape)
    return np.clip(field, 0.0, 1.0).astype(np.float32)


def fluorescence_u16(shape=(64, 512, 512), seed=1, n_emitters=None, psf_sigma=(3.0, 1.5, 1.5),
                     atten=40.0, peak=4000.0, offset=100.0):
    """Fluorescence-like stack (z, y, x), uint16 counts.

    Point emitters at uniform voxel positions with brightness U[0.5,1]
    (2000 per 64x512x512, scaled by volume otherwise), blurred by an
    anisotropic Gaussian PSF (sigma in z, y, x voxels), attenuated with depth
    as exp(-z/atten), scaled to ``peak`` counts, plus ``offset``, then Poisson
    shot noise, clipped to the uint16 range."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    if n_emitters is None:
        n_emitters = max(1, int(round(2000 * np.prod(shape) / (64 * 512 * 512))))
    vol = np.zeros(shape, dtype=np.float32)
    pos = tuple(rng.integers(0, s, size=n_emitters) for s in shape)
    np.add.at(vol, pos, rng.uniform(0.5, 1.0, size=n_emitters).astype(np.float32))
    sig = tuple(psf_sigma[-len(shape):]) if len(psf_sigma) >= len(shape) else psf_sigma
    vol = gaussian_filter(vol, sigma=sig, mode="constant")
    m = float(vol.max())
    if m > 0:
        vol *= np.float32(1.0 / m)
    z = np.arange(shape[0], dtype=np.float32)
    vol *= np.exp(-z / np.float32(atten)).reshape([-1] + [1] * (len(shape) - 1))
    lam = vol * np.float32(peak) + np.float32(offset)
    counts = rng.poisson(lam)
    return np.clip(counts, 0, 65535).astype(np.uint16)


def fluorescence(shape=(64, 512, 512), seed=1, **kw):
    """``fluorescence_u16`` normalised to float32 by 1/65535."""
    return (fluorescence_u16(shape, seed, **kw).astype(np.float32) / np.float32(65535.0))


def photoemission(shape=(128, 128, 256, 32), seed=2, n_bands=3, gamma=0.05, tau=10.0,
                  e_fermi=0.6, kt=0.01, peak=50.0):
    """Photoemission-like (kx, ky, E, t) volume of Poisson counts, float32.

    Axes: kx, ky in [-1, 1], E in [0, 1], t = 0, 1, ...  Three parabolic bands
    E = a (kx^2 + ky^2) + c (a, c seeded) broadened by a Lorentzian of
    half-width ``gamma`` in E, cut by a Fermi edge 1 / (1 + exp((E - E_F)/kT)),
    decaying along t as exp(-t/tau), scaled to ``peak`` counts, Poisson."""
    rng = np.random.default_rng(seed)
    nkx, nky, ne, nt = (int(s) for s in shape)
    kx = np.linspace(-1.0, 1.0, nkx).reshape(-1, 1, 1)
    ky = np.linspace(-1.0, 1.0, nky).reshape(1, -1, 1)
    e = np.linspace(0.0, 1.0, ne).reshape(1, 1, -1)
    a = rng.uniform(-0.35, 0.35, size=n_bands)
    c = rng.uniform(0.15, 0.75, size=n_bands)
    spec = np.zeros((nkx, nky, ne), dtype=np.float64)
    for i in range(n_bands):
        eb = a[i] * (kx * kx + ky * ky) + c[i]
        spec += gamma * gamma / ((e - eb) ** 2 + gamma * gamma)
    spec *= 1.0 / (1.0 + np.exp((e - e_fermi) / kt))
    spec *= peak / spec.max()
    decay = np.exp(-np.arange(nt, dtype=np.float64) / tau)
    out = np.empty((nkx, nky, ne, nt), dtype=np.float32)
    for i in range(nkx):  # slab by slab to bound host memory
        lam = spec[i][:, :, None] * decay[None, None, :]
        out[i] = rng.poisson(lam).astype(np.float32)
    return out


def _mult8(rng, lo, hi):
    return int(rng.integers(lo // 8, hi // 8 + 1)) * 8


def batch_shapes(seed=3):
    """Shape list of the batched workload: 16 2D in [256..2048]x[256..1536],
    24 3D in [32..96]x[256..512]^2, 8 4D in [64..128]^2x[128..256]x[16..24];
    every extent a multiple of 8 drawn uniformly (seeded)."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(16):
        shapes.append((_mult8(rng, 256, 2048), _mult8(rng, 256, 1536)))
    for _ in range(24):
        shapes.append((_mult8(rng, 32, 96), _mult8(rng, 256, 512), _mult8(rng, 256, 512)))
    for _ in range(8):
        n = _mult8(rng, 64, 128)
        shapes.append((n, _mult8(rng, 64, 128), _mult8(rng, 128, 256), _mult8(rng, 16, 24)))
    return shapes


def batch_specs(seed=3, shapes=None):
    """Per-volume parameters of the batched workload: kernel size 1/8 of each
    extent, 256 bins for even and 512 for odd volume index, 2D and 4D with a
    global and 3D with an adaptive histogram range."""
    shapes = batch_shapes(seed) if shapes is None else shapes
    specs = []
    for v, shp in enumerate(shapes):
        nd = len(shp)
        specs.append(dict(
            shape=tuple(shp),
            kernel=tuple(max(1, s // 8) for s in shp),
            n_bins=256 if v % 2 == 0 else 512,
            clip_limit=0.02 if nd == 3 else 0.01,
            adaptive=(nd == 3),
            seed=1000 + v,
        ))
    return specs


def batch_volume(spec):
    """Volume for one entry of ``batch_specs`` (generator by dimensionality)."""
    nd = len(spec["shape"])
    if nd == 2:
        return smooth_field(spec["shape"], seed=spec["seed"])
    if nd == 3:
        return fluorescence(spec["shape"], seed=spec["seed"])
    return photoemission(spec["shape"], seed=spec["seed"])


# Named workloads (shape, kernel size, bins, clip limit, adaptive range).
WORKLOADS = {
    "2d-smooth-512x512": dict(shape=(512, 512), kernel=(64, 64), n_bins=256, clip_limit=0.01,
                              adaptive=False, gen="smooth", seed=0),
    "3d-fluorescence-64x512x512": dict(shape=(64, 512, 512), kernel=(16, 64, 64), n_bins=256,
                                       clip_limit=0.02, adaptive=True, gen="fluorescence",
                                       seed=1),
    "4d-photoemission-128x128x256x32": dict(shape=(128, 128, 256, 32), kernel=(32, 32, 32, 8),
                                            n_bins=512, clip_limit=0.01, adaptive=False,
                                            gen="photoemission", seed=2),
}


def make_volume(gen, shape, seed):
    if gen == "smooth":
        return smooth_field(shape, seed=seed)
    if gen == "fluorescence":
        return fluorescence(shape, seed=seed)
    if gen == "photoemission":
        return photoemission(shape, seed=seed)
    raise ValueError(gen)


# ---------------------------------------------------------------------------
# The same recipes drawn with torch on a device (for large benchmark inputs).
# They follow the numpy generators above step by step but use torch's random
# streams (torch.Generator seeded with the same seed), so they give volumes of
# the same distribution, not the same samples.
# ---------------------------------------------------------------------------
def _tgen(seed, device):
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def smooth_field_t(shape, seed=0, device="cuda", n_gauss=20, sigma=(20.0, 80.0), scale=0.6,
                   noise_sd=0.02):
    """smooth_field drawn on a device (float32 tensor)."""
    import torch

    g = _tgen(seed, device)
    shape = tuple(int(s) for s in shape)
    u = lambda lo, hi: float(torch.rand((), generator=g, device=device)) * (hi - lo) + lo
    field = torch.zeros(shape, dtype=torch.float32, device=device)
    for _ in range(n_gauss):
        amp = u(0.0, 1.0)
        sig = u(*sigma)
        prod = None
        for d, s in enumerate(shape):
            c = u(0.0, s)
            ax = torch.arange(s, dtype=torch.float32, device=device)
            e = torch.exp(-((ax - c) ** 2) / (2.0 * sig * sig))
            e = e.reshape([-1 if i == d else 1 for i in range(len(shape))])
            prod = e if prod is None else prod * e
        field += amp * prod
    lo, hi = field.min(), field.max()
    field = (field - lo) / (hi - lo).clamp_min(1e-30)
    field = field * scale + noise_sd * torch.randn(shape, generator=g, device=device)
    return field.clamp_(0.0, 1.0).contiguous()


def _gauss_blur_t(vol, sigmas):
    """Separable Gaussian blur (zero boundary), kernel radius 4 sigma."""
    import torch
    import torch.nn.functional as F

    nd = vol.dim()
    for d, sig in enumerate(sigmas):
        if sig <= 0:
            continue
        r = max(1, int(4.0 * sig + 0.5))
        x = torch.arange(-r, r + 1, dtype=torch.float32, device=vol.device)
        k = torch.exp(-x * x / (2.0 * sig * sig))
        k = (k / k.sum()).view(1, 1, -1)
        v = vol.movedim(d, -1)
        sh = v.shape
        v = F.conv1d(v.reshape(-1, 1, sh[-1]), k, padding=r).reshape(sh)
        vol = v.movedim(-1, d)
    return vol.contiguous()


def fluorescence_t(shape=(64, 512, 512), seed=1, device="cuda", n_emitters=None,
                   psf_sigma=(3.0, 1.5, 1.5), atten=40.0, peak=4000.0, offset=100.0):
    """fluorescence (normalised uint16 counts, float32) drawn on a device."""
    import torch

    g = _tgen(seed, device)
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    if n_emitters is None:
        n_emitters = max(1, int(round(2000 * n / (64 * 512 * 512))))
    vol = torch.zeros(n, dtype=torch.float32, device=device)
    idx = torch.randint(0, n, (n_emitters,), generator=g, device=device)
    br = 0.5 + 0.5 * torch.rand(n_emitters, generator=g, device=device)
    vol.index_add_(0, idx, br)
    vol = _gauss_blur_t(vol.view(shape), psf_sigma[-len(shape):])
    vol = vol / vol.max().clamp_min(1e-30)
    z = torch.arange(shape[0], dtype=torch.float32, device=device)
    vol = vol * torch.exp(-z / atten).view([-1] + [1] * (len(shape) - 1))
    lam = vol * peak + offset
    counts = torch.poisson(lam, generator=g).clamp_(0, 65535)
    return (counts / 65535.0).contiguous()


def photoemission_t(shape=(128, 128, 256, 32), seed=2, device="cuda", n_bands=3, gamma=0.05,
                    tau=10.0, e_fermi=0.6, kt=0.01, peak=50.0):
    """photoemission drawn on a device (float32 Poisson counts)."""
    import torch

    g = _tgen(seed, device)
    nkx, nky, ne, nt = (int(s) for s in shape)
    kx = torch.linspace(-1.0, 1.0, nkx, device=device).view(-1, 1, 1)
    ky = torch.linspace(-1.0, 1.0, nky, device=device).view(1, -1, 1)
    e = torch.linspace(0.0, 1.0, ne, device=device).view(1, 1, -1)
    a = (torch.rand(n_bands, generator=g, device=device) * 0.7 - 0.35).tolist()
    c = (torch.rand(n_bands, generator=g, device=device) * 0.6 + 0.15).tolist()
    spec = torch.zeros((nkx, nky, ne), dtype=torch.float32, device=device)
    for i in range(n_bands):
        eb = a[i] * (kx * kx + ky * ky) + c[i]
        spec += gamma * gamma / ((e - eb) ** 2 + gamma * gamma)
    spec *= 1.0 / (1.0 + torch.exp((e - e_fermi) / kt))
    spec *= peak / spec.max()
    decay = torch.exp(-torch.arange(nt, dtype=torch.float32, device=device) / tau)
    lam = spec.unsqueeze(-1) * decay
    return torch.poisson(lam, generator=g).contiguous()


def batch_volume_t(spec, device="cuda"):
    """batch_volume drawn on a device."""
    nd = len(spec["shape"])
    if nd == 2:
        return smooth_field_t(spec["shape"], seed=spec["seed"], device=device)
    if nd == 3:
        return fluorescence_t(spec["shape"], seed=spec["seed"], device=device)
    return photoemission_t(spec["shape"], seed=spec["seed"], device=device)
