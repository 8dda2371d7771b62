"""mclahe_forward_noalloc, the forward entry point that allocates nothing.

Callers that cannot allocate device memory (for example a plugin interface that
receives only the input and output buffers) cannot pass the workspace
mclahe_forward needs; this entry point uses the library's built-in scratch
array instead.  Its output must match mclahe_forward's on the same input,
call after call, although every call reuses the same array.

The file name makes pytest collect it last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the output tolerance of the forward parity tests


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import build

    build.build()
    return torch, nat, nat.load()


def _regular_forward(torch, nat, lib, plan, x):
    ws_bytes = nat.mclahe_workspace_bytes(plan)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(x)
    st = lib.mclahe_forward(plan.handle, x.data_ptr(), out.data_ptr(), ws.data_ptr(), ws_bytes,
                            None, torch.cuda.current_stream().cuda_stream)
    assert st == nat.MCLAHE_OK
    return out


CASES = [
    ((24, 96, 80), (8, 16, 20), 256, 0.02, 1),
    ((16, 12, 40, 8), (4, 4, 8, 2), 512, 0.01, 0),
]


@pytest.mark.parametrize("shape,ks,nb,clip,mode", CASES)
def test_noalloc_matches_forward_on_two_calls_in_a_row(env, shape, ks, nb, clip, mode):
    torch, nat, lib = env
    plan = nat.mclahe_plan(shape, ks, nb, float(np.float32(clip)), mode)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(77)
    for call in range(2):   # a second call on new data must not see the first call's state
        x = torch.from_numpy(rng.gamma(2.0 + call, 1.0, size=shape).astype(np.float32)).cuda()
        want = _regular_forward(torch, nat, lib, plan, x)
        got = torch.full_like(x, -1.0)
        st = lib.mclahe_forward_noalloc(plan.handle, x.data_ptr(), got.data_ptr(), None, stream)
        assert st == nat.MCLAHE_OK, nat.status_string(st)
        torch.cuda.synchronize()
        err = (got - want).abs().max().item()
        assert err <= TOL, f"call {call}: max abs difference {err}"
    # no device code recorded an error in the built-in array's status word, and
    # reading it cleared it
    assert nat.mclahe_noalloc_sync_status() == nat.MCLAHE_OK
    assert nat.mclahe_noalloc_sync_status() == nat.MCLAHE_OK


def test_noalloc_rejects_plans_beyond_its_scratch(env):
    torch, nat, lib = env
    # 9^4 kernels x 512 bins of histograms alone exceed the 8 MiB scratch array
    plan = nat.mclahe_plan((64, 64, 64, 64), (8, 8, 8, 8), 512, 0.01, 0)
    assert nat.mclahe_plan_query(plan)["ws_scratch"] > nat.MCLAHE_NOALLOC_SCRATCH_BYTES
    x = torch.zeros(16, device="cuda")
    y = torch.zeros(16, device="cuda")
    st = lib.mclahe_forward_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), None,
                                    torch.cuda.current_stream().cuda_stream)
    assert st == nat.MCLAHE_ERR_UNSUPPORTED
