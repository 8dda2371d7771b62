"""The batched and differentiation workloads at their full sizes against the
FP64 oracle.

batch-48-uneven-2d3d4d: 16 2-D, 24 3-D and 8 4-D volumes of uneven shape
(kernel 1/8 of every extent, 256 or 512 bins) through one mclahe_batch call,
captured into a CUDA graph and replayed, exactly as the benchmark times it.
Every volume must match the oracle (output within 1e-5) and the per-volume
forward pass bit for bit.

fwd+bwd-8x64x256x256: eight fluorescence-like volumes with one learnable clip
limit each (U[0.005, 0.05]) and loss = mean squared error to a seeded target.
The table and clip-limit gradients must agree with the oracle's reverse mode
within 1e-4 relative, and the clip-limit gradient with central finite
differences of the oracle's forward pass at a clip limit whose difference
window holds no histogram count (so the loss is smooth across it).

Inputs are drawn on the device with the seeded torch generators the benchmark
uses and copied to the host for the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OUT_TOL = 1e-5
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


def test_batch_48_uneven_volumes_match_oracle_and_plain_forward(torch_cuda, orc):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import synth
    from paper_1906_11355_gb300.api import MCLAHE, MCLAHEBatch

    specs = synth.batch_specs()
    for s in specs:
        s["clip_limit"] = f32(s["clip_limit"])
    assert len(specs) == 48
    xs = [synth.batch_volume_t(s, device="cuda") for s in specs]
    outs = [torch.full_like(x, -1.0) for x in xs]
    batch = MCLAHEBatch(specs)
    batch.forward(xs, outs=outs, use_graph=True)      # capture and first replay
    for o in outs:
        o.fill_(-1.0)
    batch.forward(xs, outs=outs, use_graph=True)      # replay of the cached graph
    torch.cuda.synchronize()
    assert nat.mclahe_sync_status(batch.ws) == nat.MCLAHE_OK
    worst = 0.0
    for v, (s, x, out) in enumerate(zip(specs, xs, outs)):
        op = MCLAHE(s["shape"], s["kernel"], s["n_bins"], s["clip_limit"], s["adaptive"])
        op.set_shapes(**{**op.shapes(), "map_tma": 0})   # the batch's lane assignment
        ref = op.forward(x)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (v, s["shape"])
        xh = x.cpu().numpy()
        want = orc.mclahe(xh, s["kernel"], s["n_bins"], s["clip_limit"], mode=int(s["adaptive"]))
        err = float(np.abs(out.cpu().numpy().astype(np.float64) - want).max())
        worst = max(worst, err)
        assert err <= OUT_TOL, (v, s["shape"], err)
        del op, ref
    assert worst <= OUT_TOL


B, SHAPE, KS, NB = 8, (64, 256, 256), (16, 64, 64), 256


@pytest.fixture(scope="module")
def fb_case(torch_cuda):
    """The differentiation workload: inputs, targets and clip limits as the benchmark draws them."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import synth

    xs = [synth.fluorescence_t(SHAPE, seed=2000 + v, device="cuda") for v in range(B)]
    tgt = [synth.fluorescence_t(SHAPE, seed=3000 + v, device="cuda") for v in range(B)]
    tgt = [t / t.max() for t in tgt]
    g = torch.Generator(device="cpu")
    g.manual_seed(4)
    clips = (0.005 + 0.045 * torch.rand(B, generator=g)).to(torch.float32)
    return xs, tgt, clips


def test_fwd_bwd_table_and_clip_gradients_match_oracle(torch_cuda, orc, fb_case):
    """mclahe_backward through the C ABI on every volume of the workload, with the
    same upstream gradient on both sides (the MSE gradient of the oracle's output)."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    xs, tgt, clips = fb_case
    n = float(B * int(np.prod(SHAPE)))
    op = MCLAHE(SHAPE, KS, NB, 0.02, adaptive=True)
    K = op.n_kernels
    for v in range(B):
        c = float(clips[v])
        xh = xs[v].cpu().numpy()
        th = tgt[v].cpu().numpy().astype(np.float64)
        want_out = orc.mclahe(xh, KS, NB, c, mode=1)
        g = 2.0 * (want_out - th) / n
        want_lut, want_clip = orc.mclahe_backward(xh, KS, NB, c, g, mode=1)
        ws = torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda")
        out = torch.empty_like(xs[v])
        dclip = clips[v:v + 1].cuda()
        nat.mclahe_forward(op.plan, xs[v], out, ws, op.ws_bytes, dclip)
        gd = torch.from_numpy(g.astype(np.float32)).cuda()
        glut = torch.empty(K * NB, dtype=torch.float32, device="cuda")
        gclip = torch.empty(1, dtype=torch.float32, device="cuda")
        nat.mclahe_backward(op.plan, xs[v], gd, ws, op.ws_bytes, dclip, glut, gclip)
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - want_out).max() <= OUT_TOL, v
        gl = glut.view(K, NB).cpu().numpy().astype(np.float64)
        assert np.abs(gl - want_lut).max() <= REL * np.abs(want_lut).max(), v
        assert abs(float(gclip.item()) - want_clip) <= REL * abs(want_clip), (v, gclip.item(), want_clip)


def test_fwd_bwd_autograd_loss_gradients_match_oracle(torch_cuda, orc, fb_case):
    """The whole form as a user writes it: the autograd function over all eight
    volumes, loss = MSE, loss.backward(); clip gradients against the oracle."""
    torch = torch_cuda
    from paper_1906_11355_gb300.autograd import mclahe_autograd

    xs, tgt, clips = fb_case
    x = torch.stack(xs)
    t = torch.stack(tgt)
    clip = clips.cuda().requires_grad_(True)
    out = mclahe_autograd(x, clip, KS, NB, adaptive=True)
    loss = ((out - t) ** 2).mean()
    loss.backward()
    got = clip.grad.cpu().numpy()
    n = float(x.numel())
    for v in range(B):
        c = float(clips[v])
        xh = xs[v].cpu().numpy()
        want_out = orc.mclahe(xh, KS, NB, c, mode=1)
        assert np.abs(out[v].detach().cpu().numpy() - want_out).max() <= OUT_TOL, v
        g = 2.0 * (want_out - tgt[v].cpu().numpy().astype(np.float64)) / n
        _, want = orc.mclahe_backward(xh, KS, NB, c, g, mode=1)
        assert abs(got[v] - want) <= REL * abs(want), (v, got[v], want)


def _kink_free(hist, V, c0, h):
    """A clip limit near c0 whose window [T - hV, T + hV] (T = c V) holds no
    histogram count, found by walking outwards in steps of 1/V."""
    counts = np.unique(hist.astype(np.float64))
    for i in range(4000):
        for sgn in (1, -1):
            c = f32(c0 + sgn * i / V)
            T = c * V
            j = np.searchsorted(counts, T - 1.5 * h * V)
            if j >= len(counts) or counts[j] > T + 1.5 * h * V:
                return c
    return None


def test_fwd_bwd_clip_gradient_matches_finite_differences(torch_cuda, orc, fb_case):
    """dL/dclip of two volumes against central differences of the FP64 oracle's
    loss, at h = 1e-4 where a kink-free window exists, else the largest smaller
    step that has one (the loss is only piecewise smooth in the clip limit)."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    xs, tgt, clips = fb_case
    n = float(B * int(np.prod(SHAPE)))
    V = int(np.prod(KS))
    op = MCLAHE(SHAPE, KS, NB, 0.02, adaptive=True)
    for v in (0, 1):
        xh = xs[v].cpu().numpy()
        th = tgt[v].cpu().numpy().astype(np.float64)
        hist, _, _, _ = orc.histograms(xh, KS, NB, mode=1)
        c = None
        for h in (1e-4, 3e-5, 1e-5, 3e-6):
            c = _kink_free(hist, V, float(clips[v]), h)
            if c is not None:
                break
        assert c is not None, "no kink-free clip limit found"

        def loss(cc):
            return float(np.sum((orc.mclahe(xh, KS, NB, cc, mode=1) - th) ** 2) / n)

        fd = (loss(c + h) - loss(c - h)) / (2 * h)
        want_out = orc.mclahe(xh, KS, NB, c, mode=1)
        g = 2.0 * (want_out - th) / n
        ws = torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda")
        out = torch.empty_like(xs[v])
        dclip = torch.tensor([c], dtype=torch.float32, device="cuda")
        nat.mclahe_forward(op.plan, xs[v], out, ws, op.ws_bytes, dclip)
        gclip = torch.empty(1, dtype=torch.float32, device="cuda")
        nat.mclahe_backward(op.plan, xs[v], torch.from_numpy(g.astype(np.float32)).cuda(), ws,
                            op.ws_bytes, dclip, None, gclip)
        torch.cuda.synchronize()
        assert abs(fd) > 0.0
        assert abs(float(gclip.item()) - fd) <= REL * abs(fd), (v, c, h, gclip.item(), fd)
