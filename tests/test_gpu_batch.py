"""The batched form (mclahe_batch: persistent launches over a work list of
kernel and cell tiles of many volumes, with per-volume ready counters) against
the per-volume forward pass and the FP64 oracle.

The batch runs the same per-kernel and per-cell code as mclahe_forward with
per-thread loads, so its histograms, tables and outputs must equal those
per-volume results bit for bit, whatever the tile order.  (The corner sums of a
voxel run in a lane-rotated order, so a walk that gives voxels to other lanes,
such as the TMA tiles, may differ in the last bits.)  The oracle check keeps
the usual 1e-5 bound."""
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


def _specs():
    f = lambda c: float(np.float32(c))
    return [
        dict(shape=(96, 80), kernel=(12, 10), n_bins=256, clip_limit=f(0.01), adaptive=False),
        dict(shape=(64, 48), kernel=(8, 6), n_bins=512, clip_limit=f(0.02), adaptive=False),
        dict(shape=(40, 56), kernel=(5, 7), n_bins=64, clip_limit=f(0.03), adaptive=False,
             global_range=(0.0, 4.0)),
        dict(shape=(16, 40, 32), kernel=(2, 5, 4), n_bins=256, clip_limit=f(0.02), adaptive=True),
        dict(shape=(24, 32, 40), kernel=(3, 4, 5), n_bins=512, clip_limit=f(0.02), adaptive=True),
        dict(shape=(16, 16, 24, 8), kernel=(2, 2, 3, 1), n_bins=256, clip_limit=f(0.01), adaptive=False),
        dict(shape=(8, 16, 16, 16), kernel=(1, 2, 2, 2), n_bins=512, clip_limit=f(0.01), adaptive=False),
        dict(shape=(37,), kernel=(6,), n_bins=16, clip_limit=f(0.05), adaptive=True),
    ]


def _inputs(specs, seed):
    rng = np.random.default_rng(seed)
    return [rng.gamma(2.0, 1.0, size=s["shape"]).astype(np.float32) for s in specs]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_per_volume_forward_and_oracle(torch_cuda, orc, use_graph):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE, MCLAHEBatch

    specs = _specs()
    xs_h = _inputs(specs, 3)
    xs = [torch.from_numpy(x).cuda() for x in xs_h]
    batch = MCLAHEBatch(specs)
    outs = batch.forward(xs, use_graph=use_graph)
    for rep in range(2):   # a second call (graph replay) gives the same result
        outs2 = batch.forward(xs, outs=[torch.empty_like(x) for x in xs], use_graph=use_graph)
        torch.cuda.synchronize()
        for a, b in zip(outs, outs2):
            assert torch.equal(a, b)
    from paper_1906_11355_gb300 import _native as nat

    assert nat.mclahe_sync_status(batch.ws) == nat.MCLAHE_OK
    for x, xh, s, out in zip(xs, xs_h, specs, outs):
        op = MCLAHE(s["shape"], s["kernel"], s["n_bins"], s["clip_limit"], s["adaptive"],
                    s.get("global_range"))
        op.set_shapes(**{**op.shapes(), "map_tma": 0})   # the batch's lane assignment
        ref = op.forward(x)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), s
        want = orc.mclahe(xh, s["kernel"], s["n_bins"], s["clip_limit"], mode=int(s["adaptive"]),
                          range_=s.get("global_range"))
        assert np.abs(out.cpu().numpy().astype(np.float64) - want).max() <= 1e-5, s


def test_batch_per_volume_clip_and_new_data(torch_cuda, orc):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHEBatch

    specs = _specs()[3:6]
    batch = MCLAHEBatch(specs)
    clips = np.array([0.005, 0.04, 0.2], np.float32)
    clip = torch.from_numpy(clips).cuda()
    xs = [torch.empty(s["shape"], device="cuda") for s in specs]
    outs = [torch.empty_like(x) for x in xs]
    for seed in (11, 12):   # same tensors (graph replay), new contents
        xs_h = _inputs(specs, seed)
        for x, xh in zip(xs, xs_h):
            x.copy_(torch.from_numpy(xh))
        batch.forward(xs, outs=outs, clip=clip)
        torch.cuda.synchronize()
        for xh, s, c, out in zip(xs_h, specs, clips, outs):
            want = orc.mclahe(xh, s["kernel"], s["n_bins"], float(c), mode=int(s["adaptive"]))
            assert np.abs(out.cpu().numpy().astype(np.float64) - want).max() <= 1e-5


def test_batch_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHEBatch

    specs = _specs()[:2]
    batch = MCLAHEBatch(specs)
    xs = [torch.zeros(s["shape"], device="cuda") for s in specs]
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_batch(batch.plans, xs, xs, batch.ws, batch.ws_bytes)   # in == out
    assert e.value.status == nat.MCLAHE_ERR_INVALID_ARG
    with pytest.raises(nat.MclaheError) as e:
        nat.mclahe_batch(batch.plans, xs, [torch.empty_like(x) for x in xs], batch.ws, 256)
    assert e.value.status == nat.MCLAHE_ERR_WORKSPACE


def test_autotune_keeps_results_exact(torch_cuda, orc):
    torch = torch_cuda
    from paper_1906_11355_gb300.api import MCLAHE

    rng = np.random.default_rng(17)
    x = rng.gamma(2.0, size=(32, 64, 64)).astype(np.float32)
    op = MCLAHE(x.shape, (8, 16, 16), 256, float(np.float32(0.02)), adaptive=True)
    xd = torch.from_numpy(x).cuda()
    op.autotune(xd)
    out = op.forward(xd)
    torch.cuda.synchronize()
    want, aux = orc.mclahe(x, (8, 16, 16), 256, float(np.float32(0.02)), mode=1, full=True)
    np.testing.assert_array_equal(op.histograms().cpu().numpy(), aux["hist"].astype(np.int64))
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-5


def test_batch_wait_that_gives_up_reports_timeout_and_the_launch_ends(torch_cuda, orc):
    """Failure detection of the persistent launches: every wait target is raised
    out of reach (mclahe_batch_set_wait's test switch), so the first wait on a
    ready counter polls a short while, gives up and records MCLAHE_ERR_TIMEOUT;
    the later waits then return at once and the launch ends.  Nothing faults or
    hangs: the status is read back on the host, and the next normal call on the
    same workspace is correct."""
    import time

    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHEBatch

    specs = _specs()[:7]   # 2-D global (range tiles), 3-D adaptive and 4-D volumes
    xs_h = _inputs(specs, 21)
    xs = [torch.from_numpy(x).cuda() for x in xs_h]
    batch = MCLAHEBatch(specs)
    outs = [torch.empty_like(x) for x in xs]
    torch.cuda.synchronize()
    nat.mclahe_batch_set_wait(2000, unreachable=True)
    try:
        t0 = time.time()
        batch.forward(xs, outs=outs, use_graph=False)
        status = nat.mclahe_sync_status(batch.ws)
        elapsed = time.time() - t0
    finally:
        nat.mclahe_batch_set_wait(0, unreachable=False)
    assert status == nat.MCLAHE_ERR_TIMEOUT
    assert elapsed < 30.0
    assert nat.mclahe_sync_status(batch.ws) == nat.MCLAHE_OK   # reading it cleared it
    for use_graph in (False, True):
        batch.forward(xs, outs=outs, use_graph=use_graph)
        torch.cuda.synchronize()
        assert nat.mclahe_sync_status(batch.ws) == nat.MCLAHE_OK
        for xh, s, out in zip(xs_h, specs, outs):
            want = orc.mclahe(xh, s["kernel"], s["n_bins"], s["clip_limit"], mode=int(s["adaptive"]),
                              range_=s.get("global_range"))
            assert np.abs(out.cpu().numpy().astype(np.float64) - want).max() <= 1e-5, s


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("branches", [1, 3, 16])
def test_concurrent_batch_equals_per_volume_forward(torch_cuda, orc, use_graph, branches):
    """mclahe_batch_concurrent runs each volume's own forward pass on parallel
    branches: every output equals mclahe_forward's with the same plan bit for bit
    (the plans' own shapes and walks), call after call."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE, MCLAHEBatch

    specs = _specs()
    xs_h = _inputs(specs, 31)
    xs = [torch.from_numpy(x).cuda() for x in xs_h]
    batch = MCLAHEBatch(specs)
    for rep in range(2):
        outs = batch.forward(xs, outs=[torch.full_like(x, -1.0) for x in xs], use_graph=use_graph,
                             concurrent=branches)
        torch.cuda.synchronize()
        for v, (x, xh, s, out) in enumerate(zip(xs, xs_h, specs, outs)):
            op = MCLAHE(s["shape"], s["kernel"], s["n_bins"], s["clip_limit"], s["adaptive"],
                        s.get("global_range"))
            op.set_shapes(**batch_shapes(nat, batch.plans[v]))
            assert torch.equal(out, op.forward(x)), (rep, s)
            if rep == 0:
                want = orc.mclahe(xh, s["kernel"], s["n_bins"], s["clip_limit"], mode=int(s["adaptive"]),
                                  range_=s.get("global_range"))
                assert np.abs(out.cpu().numpy().astype(np.float64) - want).max() <= 1e-5, s


def batch_shapes(nat, plan):
    i = nat.mclahe_plan_query(plan)
    return {k: int(i[k]) for k in ("hist_group", "hist_cluster", "hist_copies", "hist_shares", "hist_walk",
                                   "hist_threads", "map_chunks", "map_tma", "map_flat")}


@pytest.mark.parametrize("branches", [1, 4, 16])
def test_forward_batch_of_one_plan_equals_forward(torch_cuda, orc, branches):
    """mclahe_forward_batch: volumes of one plan, each with its own workspace,
    on parallel branches: outputs, histograms and tables equal mclahe_forward's
    bit for bit (per-volume clip limits on the device), and the workspaces
    serve the batched backward."""
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    shape, ks, nb, n = (24, 40, 36), (6, 8, 9), 128, 11
    rng = np.random.default_rng(90 + branches)
    xs = torch.from_numpy(rng.gamma(2.0, size=(n,) + shape).astype(np.float32)).cuda()
    clips = torch.from_numpy((0.01 + 0.04 * rng.random(n)).astype(np.float32)).cuda()
    op = MCLAHE(shape, ks, n_bins=nb, clip_limit=0.02, adaptive=True)
    ws = [torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda") for _ in range(n)]
    out = torch.full_like(xs, -1.0)
    nat.mclahe_forward_batch(op.plan, list(xs), list(out), ws, op.ws_bytes, clips, None, branches)
    one_ws = torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda")
    one = torch.empty(shape, device="cuda")
    info = nat.mclahe_plan_query(op.plan)
    for v in range(n):
        nat.mclahe_forward(op.plan, xs[v], one, one_ws, op.ws_bytes, clips[v:v + 1])
        torch.cuda.synchronize()
        assert torch.equal(out[v], one), v
        a, b = info["ws_hist"], info["ws_scratch"]   # histograms, ranges and tables
        assert torch.equal(ws[v][a:b], one_ws[a:b]), v
    want = orc.mclahe(xs[n - 1].cpu().numpy(), ks, nb, float(clips[n - 1].item()), mode=1)
    assert np.abs(out[n - 1].cpu().numpy() - want).max() <= 1e-5
    g = torch.from_numpy(rng.normal(size=(n,) + shape).astype(np.float32)).cuda()
    gc = torch.empty(n, device="cuda")
    nat.mclahe_backward_batch(op.plan, list(xs), list(g), ws, op.ws_bytes, clips, gc)
    gc1 = torch.empty(1, device="cuda")
    nat.mclahe_backward(op.plan, xs[3], g[3], ws[3], op.ws_bytes, clips[3:4], None, gc1)
    torch.cuda.synchronize()
    assert gc[3].item() == gc1.item()


def test_forward_batch_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300.api import MCLAHE

    op = MCLAHE((16, 16), (4, 4), n_bins=32, clip_limit=0.02)
    x = torch.zeros((2, 16, 16), device="cuda")
    o = torch.zeros((2, 16, 16), device="cuda")
    ws = [torch.zeros(op.ws_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    with pytest.raises(nat.MclaheError):   # one workspace for two volumes
        nat.mclahe_forward_batch(op.plan, list(x), list(o), [ws[0], ws[0]], op.ws_bytes)
    with pytest.raises(nat.MclaheError):   # one output for two volumes
        nat.mclahe_forward_batch(op.plan, list(x), [o[0], o[0]], ws, op.ws_bytes)
    with pytest.raises(nat.MclaheError):   # an output that is another volume's input
        nat.mclahe_forward_batch(op.plan, list(x), [o[0], x[0]], ws, op.ws_bytes)
    with pytest.raises(nat.MclaheError):
        nat.mclahe_forward_batch(op.plan, list(x), list(o), ws, op.ws_bytes, branches=0)
    nat.mclahe_forward_batch(op.plan, [], [], [], op.ws_bytes)   # nothing to do
