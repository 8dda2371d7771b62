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
