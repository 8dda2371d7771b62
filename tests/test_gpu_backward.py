"""Parity of the CUDA backward pass (mclahe_backward through the C ABI) with
the FP64 oracle's reverse mode and with central finite differences.

Table gradients (dL/dlut, linear in the upstream gradient) and the clip-limit
gradient (through clip, redistribution, cumulative sum and normalisation) must
agree with the oracle within 1e-4 relative; the clip gradient is also checked
against central differences of the oracle's forward at kink-free clip values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_11355_gb300 import build

    build.build()
    return torch


def f32(c):
    return float(np.float32(c))


def gpu_backward(torch, x, ks, nb, clip, g, adaptive):
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE(x.shape, ks, n_bins=nb, clip_limit=clip, adaptive=adaptive)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    gd = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    out = op.forward(xd)
    glut = torch.empty(op.n_kernels * nb, dtype=torch.float32, device="cuda")
    gclip = torch.empty(1, dtype=torch.float32, device="cuda")
    nat.mclahe_backward(op.plan, xd, gd, op.ws, op.ws_bytes, None, glut, gclip)
    torch.cuda.synchronize()
    return out, glut.view(op.n_kernels, nb).cpu().numpy().astype(np.float64), float(gclip.item())


def close(got, want, rel=REL):
    scale = max(np.abs(want).max(), 1e-12)
    return np.abs(got - want).max() <= rel * scale


CASES = [
    # (shape, kernel, n_bins, clip, adaptive)
    ((37,), (6,), 16, 0.05, False),
    ((53, 47), (8, 7), 64, 0.01, False),
    ((53, 47), (8, 7), 64, 0.01, True),
    ((64, 64), (16, 16), 256, 0.0, False),
    ((30, 41), (30, 41), 32, 0.1, True),         # b = s
    ((19, 23, 29), (5, 4, 7), 100, 0.02, False),
    ((19, 23, 29), (5, 4, 7), 100, 0.02, True),
    ((16, 64, 64), (4, 16, 16), 256, 0.02, True),
    ((11, 9, 13, 10), (3, 4, 5, 2), 50, 0.03, False),
    ((8, 8, 16, 12), (4, 4, 8, 3), 512, 0.01, True),
]


@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) + ("A" if c[4] else "G") for c in CASES])
def test_backward_matches_oracle(torch_cuda, orc, case):
    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, 7)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    g = rng.normal(size=shape).astype(np.float32)
    clip = f32(clip)
    _, glut, gclip = gpu_backward(torch_cuda, x, ks, nb, clip, g, adaptive)
    want_lut, want_clip = orc.mclahe_backward(x, ks, nb, clip, g.astype(np.float64), mode=int(adaptive))
    assert close(glut, want_lut), np.abs(glut - want_lut).max()
    assert abs(gclip - want_clip) <= REL * max(abs(want_clip), 1e-3 * np.abs(want_lut).max()), \
        (gclip, want_clip)


def _kink_free_clip(hist, V, lo, hi, h_step, rng):
    counts = np.unique(hist.astype(np.float64))
    for _ in range(2000):
        c = f32(rng.uniform(lo, hi))
        if np.min(np.abs(counts - c * V)) > 1.5 * h_step * V:
            return c
    raise AssertionError("no kink-free clip value found")


@pytest.mark.parametrize("mode,shape,ks,nb,crange", [
    (0, (24, 20), (6, 5), 16, (0.02, 0.3)),
    (1, (10, 12, 9), (4, 4, 3), 16, (0.02, 0.3)),
    (1, (16, 32, 32), (8, 16, 16), 64, (0.004, 0.02)),   # T below the tallest bins
])
def test_clip_gradient_matches_finite_differences(torch_cuda, orc, mode, shape, ks, nb, crange):
    rng = np.random.default_rng(40 + mode + len(shape))
    x = rng.gamma(2.0, size=shape).astype(np.float32)
    h = 1e-5
    hist, _, _, _ = orc.histograms(x, ks, nb, mode=mode)
    V = int(np.prod(ks))
    clip = _kink_free_clip(hist, V, crange[0], crange[1], h, rng)
    g = rng.normal(size=shape).astype(np.float32)
    _, _, gclip = gpu_backward(torch_cuda, x, ks, nb, clip, g, bool(mode))
    gg = g.astype(np.float64)
    fd = (np.sum(gg * orc.mclahe(x, ks, nb, clip + h, mode=mode))
          - np.sum(gg * orc.mclahe(x, ks, nb, clip - h, mode=mode))) / (2 * h)
    assert abs(gclip - fd) <= REL * max(1.0, abs(fd)), (gclip, fd)
    assert abs(fd) > 1e-3


def test_autograd_function_and_learnable_clip(torch_cuda, orc):
    torch = torch_cuda
    from paper_1906_11355_gb300.autograd import mclahe_autograd

    rng = np.random.default_rng(51)
    shape, ks, nb = (3, 16, 24, 20), (4, 8, 5), 64   # a batch of three 3-D volumes
    x = rng.gamma(2.0, size=shape).astype(np.float32)
    target = rng.random(shape, dtype=np.float32)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    clip0 = np.array([0.01, 0.02, 0.04], np.float32)
    clip = torch.tensor(clip0, device="cuda", requires_grad=True)
    out = mclahe_autograd(xd, clip, ks, nb, adaptive=True)
    loss = ((out - torch.from_numpy(target).cuda()) ** 2).mean()
    loss.backward()
    assert torch.count_nonzero(xd.grad).item() == 0
    got = clip.grad.cpu().numpy()
    for b in range(3):
        want_out = orc.mclahe(x[b], ks, nb, float(clip0[b]), mode=1)
        assert np.abs(out[b].detach().cpu().numpy() - want_out).max() <= 1e-5
        g = 2.0 * (want_out - target[b]) / x.size
        _, want = orc.mclahe_backward(x[b], ks, nb, float(clip0[b]), g, mode=1)
        assert abs(got[b] - want) <= REL * max(abs(want), 1e-6), (b, got[b], want)


def test_backward_is_deterministic_and_clamped_clip_has_zero_gradient(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    rng = np.random.default_rng(61)
    x = torch.from_numpy(rng.random((40, 48), dtype=np.float32)).cuda()
    g = torch.from_numpy(rng.normal(size=(40, 48)).astype(np.float32)).cuda()
    op = MCLAHE((40, 48), (10, 12), 32, 0.05)
    res = []
    for c in (0.05, 0.05, 1.5):
        clip = torch.tensor([c], device="cuda")
        op.forward(x, clip=clip)
        gc = torch.empty(1, device="cuda")
        gl = torch.empty(op.n_kernels * 32, device="cuda")
        nat.mclahe_backward(op.plan, x, g, op.ws, op.ws_bytes, clip, gl, gc)
        res.append((gc.clone(), gl.clone()))
    torch.cuda.synchronize()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    assert res[2][0].item() == 0.0


def test_backward_integer_sums_are_deterministic_and_scale_free(torch_cuda):
    """The adjoint sums fixed-point integers at a scale set by max |g|: repeated
    calls agree bit for bit, and scaling g by powers of two (far below and far
    above 1) scales the gradients by exactly the same power of two."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    rng = np.random.default_rng(77)
    shape, ks, nb = (16, 64, 64), (4, 16, 16), 256
    x = torch.from_numpy(rng.gamma(2.0, 1.0, size=shape).astype(np.float32)).cuda()
    g = torch.from_numpy(rng.normal(size=shape).astype(np.float32)).cuda()
    op = MCLAHE(shape, ks, nb, f32(0.02), adaptive=True)
    op.forward(x)

    def run(gg):
        gl = torch.empty(op.n_kernels * nb, device="cuda")
        gc = torch.empty(1, device="cuda")
        nat.mclahe_backward(op.plan, x, gg, op.ws, op.ws_bytes, None, gl, gc)
        return gl, gc

    a = run(g)
    b = run(g)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    for p in (-60, 60):
        s = run(g * 2.0 ** p)
        torch.cuda.synchronize()
        assert torch.equal(s[0], a[0] * 2.0 ** p), p
        assert torch.equal(s[1], a[1] * 2.0 ** p), p


@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) + ("A" if c[4] else "G") for c in CASES])
def test_clip_gradient_alone_gather_matches_oracle_and_scatter(torch_cuda, orc, case):
    """Without table gradients mclahe_backward takes the gather form (d lut/dT
    tables interpolated like the mapping pass, dotted with g): the same clip
    gradient as the oracle's reverse mode and as the scatter form, repeatable
    bit for bit, and 0 for a clip limit outside [0, 1]."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb, clip, adaptive = case
    rng = np.random.default_rng(hash((shape, ks, nb, 9)) % 2**32)
    x = rng.gamma(2.0, 1.0, size=shape).astype(np.float32)
    g = rng.normal(size=shape).astype(np.float32)
    clip = f32(clip)
    op = MCLAHE(x.shape, ks, n_bins=nb, clip_limit=clip, adaptive=adaptive)
    xd = torch.from_numpy(x).cuda()
    gd = torch.from_numpy(g).cuda()
    op.forward(xd)
    got = []
    for _ in range(2):
        gc = torch.empty(1, dtype=torch.float32, device="cuda")
        nat.mclahe_backward(op.plan, xd, gd, op.ws, op.ws_bytes, None, None, gc)
        got.append(gc.clone())
    glut = torch.empty(op.n_kernels * nb, dtype=torch.float32, device="cuda")
    gsc = torch.empty(1, dtype=torch.float32, device="cuda")
    nat.mclahe_backward(op.plan, xd, gd, op.ws, op.ws_bytes, None, glut, gsc)
    torch.cuda.synchronize()
    assert torch.equal(got[0], got[1])
    _, want = orc.mclahe_backward(x, ks, nb, clip, g.astype(np.float64), mode=int(adaptive))
    want_lut, _ = orc.mclahe_backward(x, ks, nb, clip, g.astype(np.float64), mode=int(adaptive))
    tol = REL * max(abs(want), 1e-3 * np.abs(want_lut).max())
    assert abs(got[0].item() - want) <= tol, (got[0].item(), want)
    assert abs(got[0].item() - gsc.item()) <= tol, (got[0].item(), gsc.item())
    # a clip limit outside [0, 1] is clamped by the forward pass: zero gradient
    out_clip = torch.tensor([1.5], device="cuda")
    op.forward(xd, clip=out_clip)
    gc = torch.empty(1, dtype=torch.float32, device="cuda")
    nat.mclahe_backward(op.plan, xd, gd, op.ws, op.ws_bytes, out_clip, None, gc)
    torch.cuda.synchronize()
    assert gc.item() == 0.0


@pytest.mark.parametrize("n_vol,adaptive", [(35, True), (5, False)])
def test_backward_batch_equals_per_volume_backward(torch_cuda, orc, n_vol, adaptive):
    """mclahe_backward_batch (three launches per 32 volumes, here two groups
    with 35 volumes) gives every volume the clip gradient mclahe_backward gives
    it, bit for bit, with per-volume clip limits on the device (one outside
    [0, 1]: zero gradient); a few checked against the oracle."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb = (12, 20, 28), (4, 8, 7), 64
    rng = np.random.default_rng(71 + n_vol)
    xs = [rng.gamma(2.0, size=shape).astype(np.float32) for _ in range(n_vol)]
    gs = [rng.normal(size=shape).astype(np.float32) for _ in range(n_vol)]
    clips = (0.005 + 0.05 * rng.random(n_vol)).astype(np.float32)
    clips[3] = 1.25
    op = MCLAHE(shape, ks, n_bins=nb, clip_limit=0.02, adaptive=adaptive)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    gd = [torch.from_numpy(g).cuda() for g in gs]
    cd = torch.from_numpy(clips).cuda()
    ws = [torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda") for _ in range(n_vol)]
    out = torch.empty(shape, device="cuda")
    for v in range(n_vol):
        nat.mclahe_forward(op.plan, xd[v], out, ws[v], op.ws_bytes, cd[v:v + 1])
    got = torch.full((n_vol,), float("nan"), device="cuda")
    nat.mclahe_backward_batch(op.plan, xd, gd, ws, op.ws_bytes, cd, got)
    one = torch.empty(n_vol, device="cuda")
    for v in range(n_vol):
        nat.mclahe_backward(op.plan, xd[v], gd[v], ws[v], op.ws_bytes, cd[v:v + 1], None, one[v:v + 1])
    torch.cuda.synchronize()
    assert torch.equal(got, one)
    assert got[3].item() == 0.0
    for v in (0, n_vol - 1):
        _, want = orc.mclahe_backward(xs[v], ks, nb, float(clips[v]), gs[v].astype(np.float64),
                                      mode=int(adaptive))
        want_lut, _ = orc.mclahe_backward(xs[v], ks, nb, float(clips[v]), gs[v].astype(np.float64),
                                          mode=int(adaptive))
        tol = REL * max(abs(want), 1e-3 * np.abs(want_lut).max())
        assert abs(got[v].item() - want) <= tol, (v, got[v].item(), want)


def test_backward_batch_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE((16, 16), (4, 4), n_bins=32, clip_limit=0.02)
    x = [torch.zeros((16, 16), device="cuda") for _ in range(2)]
    ws = torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda")
    gc = torch.zeros(2, device="cuda")
    with pytest.raises(nat.MclaheError):   # one workspace for two volumes
        nat.mclahe_backward_batch(op.plan, x, x[::-1], [ws, ws], op.ws_bytes, None, gc)
    with pytest.raises(nat.MclaheError):   # no output
        nat.mclahe_backward_batch(op.plan, x, x[::-1], [ws, ws], op.ws_bytes, None, None)
    nat.mclahe_backward_batch(op.plan, [], [], [], op.ws_bytes, None, gc)   # nothing to do
