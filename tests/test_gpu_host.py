"""Volumes in host memory (mclahe_forward_host): each copied in, mapped and
copied out through two device slots, the copies overlapping the kernels.  The
outputs must equal mclahe_forward's (and mclahe_forward_typed's for integer
inputs) bit for bit, with page-locked and pageable buffers, per-volume clip
limits and a repeated output buffer."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_11355_gb300 import build

    build.build()
    return torch


@pytest.mark.parametrize("n,pinned", [(1, True), (5, True), (4, False)])
def test_host_volumes_equal_device_forward(torch_cuda, orc, n, pinned):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb = (20, 36, 44), (5, 9, 11), 128
    rng = np.random.default_rng(300 + n)
    xs = [torch.from_numpy(rng.gamma(2.0, size=shape).astype(np.float32)) for _ in range(n)]
    if pinned:
        xs = [x.pin_memory() for x in xs]
    op = MCLAHE(shape, ks, n_bins=nb, clip_limit=0.02, adaptive=True)
    outs = op.forward_host(xs)
    torch.cuda.synchronize()
    for v in range(n):
        want = op.forward(xs[v].cuda()).cpu()
        assert torch.equal(outs[v], want), v
    ref = orc.mclahe(xs[0].numpy(), ks, nb, float(np.float32(0.02)), mode=1)
    assert np.abs(outs[0].numpy() - ref).max() <= 1e-5


def test_host_integer_volumes_clip_limits_and_one_output_buffer(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb, n = (16, 24, 32), (4, 6, 8), 256, 6
    rng = np.random.default_rng(41)
    xs = [torch.from_numpy(rng.integers(0, 256, size=shape).astype(np.uint8)).pin_memory() for _ in range(n)]
    clips = torch.from_numpy((0.005 + 0.05 * rng.random(n)).astype(np.float32)).cuda()
    op = MCLAHE(shape, ks, n_bins=nb, clip_limit=0.02, adaptive=False)
    outs = op.forward_host(xs, clip=clips)
    torch.cuda.synchronize()
    for v in range(n):
        want = op.forward(xs[v].cuda(), clip=clips[v:v + 1]).cpu()
        assert torch.equal(outs[v], want), v
    # every volume into one output buffer: the last volume's result remains
    one = torch.empty(shape, dtype=torch.float32).pin_memory()
    op.forward_host(xs, [one] * n, clip=clips)
    torch.cuda.synchronize()
    assert torch.equal(one, outs[-1])


def test_host_forward_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE((16, 16), (4, 4), n_bins=32, clip_limit=0.02)
    h = [torch.zeros((16, 16)).pin_memory() for _ in range(2)]
    d_in = [torch.zeros((16, 16), device="cuda") for _ in range(2)]
    d_out = [torch.zeros((16, 16), device="cuda") for _ in range(2)]
    ws = [torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    with pytest.raises(nat.MclaheError):   # one workspace for both slots
        nat.mclahe_forward_host(op.plan, nat.MCLAHE_F32, h, h, d_in, d_out, [ws[0], ws[0]], op.ws_bytes)
    with pytest.raises(nat.MclaheError):   # a slot's output is the other slot's input
        nat.mclahe_forward_host(op.plan, nat.MCLAHE_F32, h, h, d_in, [d_out[0], d_in[0]], ws, op.ws_bytes)
    with pytest.raises(nat.MclaheError):   # unknown element type
        nat.mclahe_forward_host(op.plan, 7, h, h, d_in, d_out, ws, op.ws_bytes)
    with pytest.raises(ValueError):
        op.forward_host([torch.zeros((8, 8))])
    nat.mclahe_forward_host(op.plan, nat.MCLAHE_F32, [], [], d_in, d_out, ws, op.ws_bytes)   # nothing to do
