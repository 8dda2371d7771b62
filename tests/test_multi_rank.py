"""Host logic of multi-GPU runs, exercised with gloo ranks on the CPU (world
size 2): every rank gets its own seed, a batch is split across ranks with no
volume lost or duplicated, and the step time reduces to the maximum over
ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1906_11355_gb300 import dist as md

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [5, 9, 1, 7, 7, 3, 12, 2]
        mine = md.shard(sizes, rank, world)
        t = md.max_over_ranks(10.0 + 5.0 * rank)
        q.put((rank, md.rank_seed(1, rank), mine, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, t0), (r1, s1, m1, t1) = res
    assert s0 != s1
    assert sorted(m0 + m1) == list(range(8)) and not set(m0) & set(m1)
    sizes = [5, 9, 1, 7, 7, 3, 12, 2]
    assert abs(sum(sizes[i] for i in m0) - sum(sizes[i] for i in m1)) <= max(sizes)
    assert t0 == t1 == 15.0


def test_single_process_defaults():
    from paper_1906_11355_gb300 import dist as md

    assert md.max_over_ranks(3.5) == 3.5
    assert md.shard([4, 2, 9], 0, 1) == [0, 1, 2]
    assert md.whole_job_rate(1e9, 4, 1000.0) == pytest.approx(4e9)


def _slab_worker(rank, world, port, q):
    """One volume split across gloo ranks: each rank holds the oracle's tables
    of its own kernel rows only (standing in for its histogram pass), exchanges
    the one-row halo with its neighbours, and must then hold every table its
    cell rows interpolate; the range keys combine to the global ones."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1906_11355_gb300 import _native as nat
    from paper_1906_11355_gb300 import dist as md

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shape, ks, nb = (40, 12, 16), (8, 4, 8), 32
        x = np.random.default_rng(0).gamma(2.0, size=shape).astype(np.float32)
        _, aux = oracle.mclahe(x, ks, nb, 0.02, mode=1, full=True)
        plan = nat.mclahe_plan(shape, ks, nb, 0.02, nat.MCLAHE_RANGE_ADAPTIVE)
        part = md.SlabRank(plan, rank, world, device="cpu")
        K1, LS = part.K1, part.LS
        lut = np.zeros((aux["lut"].shape[0], LS), np.float32)
        lut[:, :nb] = aux["lut"]
        for k in range(part.ka, part.kb):   # this rank's own rows only
            rows = slice(k * K1, (k + 1) * K1)
            part.put_row_tables(k, torch.from_numpy(np.concatenate(
                [lut[rows].ravel(), aux["lo"][rows], aux["scale"][rows]])))
        got = md.exchange_halo(part.first_row_tables(), rank, world, K1 * (LS + 2))
        k = part.needs_row()
        if k is not None:
            part.put_row_tables(k, got)
        ok = True
        for k in range(part.ca, part.cb + 1 if part.cb < part.n0 else part.cb):   # rows the cells interpolate
            t, lo, sc = part._rows(k)
            rows = slice(k * K1, (k + 1) * K1)
            ok &= np.array_equal(t.numpy().reshape(K1, LS)[:, :nb], lut[rows, :nb])
            ok &= np.array_equal(lo.numpy(), aux["lo"][rows]) and np.array_equal(sc.numpy(), aux["scale"][rows])
        # keys: a maximum of each 32-bit word, including words with the top bit set
        mine = torch.tensor([0x7000_0000 + rank, -(rank + 1)], dtype=torch.int32)
        comb = md.combine_keys(mine)
        q.put((rank, (part.ka, part.kb, part.ca, part.cb), bool(ok), comb.tolist()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_one_volume_split_across_gloo_ranks(world):
    import torch.multiprocessing as mp

    import oracle
    from paper_1906_11355_gb300 import build

    build.build()   # the workers load the library and the oracle as built here
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = []
    for _ in range(world):
        res.append(q.get(timeout=120))
    res.sort()
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = [r[1] for r in res]
    # the kernel rows cover [0, n0) once; the cell rows cover [0, n0 - 1) once
    n0 = parts[-1][1]
    assert [a for a, _, _, _ in parts] == sorted(a for a, _, _, _ in parts) and parts[0][0] == 0
    assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
    assert sum(cb - ca for _, _, ca, cb in parts) == n0 - 1
    assert all(r[2] for r in res), "a rank lacks a table its cells interpolate"
    want_hi = 0x7000_0000 + world - 1
    for r in res:
        assert r[3][0] == want_hi and r[3][1] == -1   # unsigned max of 0xffffffff - rank


def _failing_worker(rank, world, port, q):
    """Rank 1 fails on the host before the split-volume range exchange (an
    exception between steps, none of its work in flight); rank 0 must get an
    error from its next collective instead of waiting for ever."""
    import datetime

    import torch
    import torch.distributed as dist

    from paper_1906_11355_gb300 import dist as md

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    dist.barrier()
    if rank == 1:
        q.put((rank, "failed"))
        q.close()
        q.join_thread()
        os._exit(3)   # the rank dies on the host
    try:
        md.combine_keys(torch.tensor([1, 2], dtype=torch.int32))
        q.put((rank, "no error"))
    except Exception as e:   # the peer's loss surfaces as an error of the collective
        q.put((rank, "error: " + type(e).__name__))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_failed_rank_surfaces_as_an_error_on_the_others():
    import time

    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "failed" and procs[1].exitcode == 3
    assert res[0].startswith("error"), res[0]
    assert procs[0].exitcode == 0
    assert time.time() - t0 < 100
