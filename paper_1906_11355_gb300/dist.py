"""Host-side logic of multi-GPU runs (one process per GPU).

The units of the MCLAHE hot path -- whole volumes -- are independent, so they
are sharded across ranks with no exchange on the data path (weak scaling).
The only collectives there are a barrier around the timed region and the
max-over-ranks reduction of the step time.  One volume can also be split
across ranks along dimension 0 (forward_distributed below), with a range
all-reduce and a one-row table halo between neighbours.  Collectives use
whatever process group is initialised (NCCL on GPUs, gloo on CPUs in tests).
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed, rank):
    """Seed of a rank's own volume: every rank draws a different volume of
    the same recipe."""
    return int(seed) + 7919 * int(rank)


def shard(sizes, rank, world):
    """Indices of the volumes (given by their sizes) that `rank` processes:
    longest-processing-time-first assignment, so every rank gets about the
    same number of voxels.  Deterministic; every index goes to one rank."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(sizes[i])
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(value, device="cpu"):
    """The maximum of a float over all ranks (the value itself without an
    initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput in units per second from the slowest rank's time."""
    return float(units_per_rank) * int(world) / (float(ms_max) * 1e-3)


# ---------------------------------------------------------------------------
# One volume split across ranks along dimension 0 (slabs on kernel rows).
# Rank r owns the kernel rows [ka, kb) of a balanced contiguous partition and
# the cell rows [ka, min(kb, n0 - 1)); the cells of its last row also need the
# tables of kernel row kb, which rank r + 1 computes: one table row (and its
# ranges) is exchanged per neighbour pair.  With a global range found from the
# data, the ranks' range keys are combined by a maximum of each word first
# (the minimum is stored complemented).  Every step of MCLAHE runs in the
# library's kernels (mclahe_forward_slab); this module only moves the keys and
# the halo rows between ranks.
# ---------------------------------------------------------------------------
def kernel_row_partition(n_rows, world):
    """Balanced contiguous kernel rows [ka, kb) along dimension 0 per rank."""
    return [(n_rows * r // world, n_rows * (r + 1) // world) for r in range(world)]


def range_row_partition(s0, world):
    """Original rows per rank for the global range pass (any cover works)."""
    return [(s0 * r // world, s0 * (r + 1) // world) for r in range(world)]


class SlabRank:
    """The part of one volume a rank processes (device tensors in the rank's
    own workspace).  Phases, in order: range() [global range from the data],
    set_keys(keys) with the keys combined over ranks, hist(), halo rows out
    (first_row_tables) and in (put_row_tables) between neighbours, map()."""

    def __init__(self, plan, rank, world, device="cuda"):
        import torch

        from . import _native as nat

        self.nat = nat
        self.plan = plan
        self.info = nat.mclahe_plan_query(plan)
        self.rank, self.world = rank, world
        self.n0 = int(self.info["n_kernels_dim"][0])
        if not 1 <= world <= self.n0 or int(self.info["ndim"]) < 2:
            raise ValueError("one volume splits over at most n[0] ranks (kernel rows along dimension 0), 2-D and up")
        self.ka, self.kb = kernel_row_partition(self.n0, world)[rank]
        self.ca, self.cb = self.ka, min(self.kb, self.n0 - 1)
        self.ra, self.rb = range_row_partition(int(self.info["shape"][0]), world)[rank]
        self.row = int(self.info["n_voxels"]) // int(self.info["shape"][0])
        # rows of the input slab: the range rows, the footprints of the kernel
        # rows, the cell rows
        spans = [(self.ra, self.rb)] if self.rb > self.ra else []
        if self.kb > self.ka:
            spans.append(nat.mclahe_slab_rows(plan, nat.MCLAHE_PASS_HIST, self.ka, self.kb))
        if self.cb > self.ca:
            spans.append(nat.mclahe_slab_rows(plan, nat.MCLAHE_PASS_MAP, self.ca, self.cb))
        self.lo = min(a for a, _ in spans)
        self.hi = max(b for _, b in spans)
        self.first = (self.lo * self.row) & ~3   # element the slab starts at
        self.ws_bytes = nat.mclahe_workspace_bytes(plan)
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=device)
        self.K1 = int(self.info["n_kernels"]) // self.n0
        self.LS = int(self.info["table_stride"])
        self.device = device

    def slab_bounds(self):
        """Elements [first, end) of the volume this rank's input slab holds."""
        return self.first, self.hi * self.row

    def keys(self):
        off = int(self.info["ws_range_keys"])
        return self.ws[off:off + 8].view(torch_int32())

    def range(self, slab):
        """Min/max of the rank's range rows into its keys (global range from the data)."""
        self.keys().zero_()
        if self.rb > self.ra:
            self.nat.mclahe_forward_slab(self.plan, self.nat.MCLAHE_PASS_RANGE, slab, self.first, None, self.ws,
                                         self.ws_bytes, self.ra, self.rb)

    def set_keys(self, keys):
        self.keys().copy_(keys)

    def hist(self, slab, d_clip=None):
        if self.kb > self.ka:
            self.nat.mclahe_forward_slab(self.plan, self.nat.MCLAHE_PASS_HIST, slab, self.first, None, self.ws,
                                         self.ws_bytes, self.ka, self.kb, d_clip)

    def _rows(self, k):
        """Views of kernel row k's tables, lo and scale in the workspace."""
        i = self.info
        lut = self.ws[int(i["ws_lut"]):].view(torch_float32())[: int(i["n_kernels"]) * self.LS]
        lo = self.ws[int(i["ws_lo"]):].view(torch_float32())[: int(i["n_kernels"])]
        sc = self.ws[int(i["ws_scale"]):].view(torch_float32())[: int(i["n_kernels"])]
        a, b = k * self.K1, (k + 1) * self.K1
        return lut[a * self.LS:b * self.LS], lo[a:b], sc[a:b]

    def first_row_tables(self):
        """One flat float32 tensor: the tables, lo and scale of kernel row ka."""
        import torch

        return torch.cat(self._rows(self.ka)).clone()

    def needs_row(self):
        """The kernel row whose tables this rank receives (None if none)."""
        return self.kb if (self.cb > self.ca and self.kb < self.n0 and self.cb == self.kb) else None

    def put_row_tables(self, k, flat):
        lut, lo, sc = self._rows(k)
        n1, n2 = lut.numel(), lo.numel()
        lut.copy_(flat[:n1])
        lo.copy_(flat[n1:n1 + n2])
        sc.copy_(flat[n1 + n2:])

    def map(self, slab, out_slab):
        if self.cb > self.ca:
            self.nat.mclahe_forward_slab(self.plan, self.nat.MCLAHE_PASS_MAP, slab, self.first, out_slab,
                                         self.ws, self.ws_bytes, self.ca, self.cb)

    def out_rows(self):
        """Original rows [a, b) of the output this rank computes (its cell rows)."""
        if self.cb <= self.ca:
            return 0, 0
        return self.nat.mclahe_slab_rows(self.plan, self.nat.MCLAHE_PASS_MAP, self.ca, self.cb)


def torch_int32():
    import torch

    return torch.int32


def torch_float32():
    import torch

    return torch.float32


def combine_keys(keys, group=None):
    """The global range keys over all ranks: a maximum of each word (the minimum
    is stored complemented); int64 for the collective."""
    import torch
    import torch.distributed as dist

    k = keys.to(torch.int64) & 0xFFFFFFFF
    dist.all_reduce(k, op=dist.ReduceOp.MAX, group=group)
    return k.to(torch.int64).where(k < 2 ** 31, k - 2 ** 32).to(torch.int32)


def exchange_halo(first_row, rank, world, recv_numel, group=None):
    """Send this rank's first kernel row's tables to rank - 1 and receive rank +
    1's (None when there is no next rank).  Point-to-point, both directions posted
    before waiting."""
    import torch
    import torch.distributed as dist

    reqs, got = [], None
    if rank > 0:
        reqs.append(dist.isend(first_row.contiguous(), rank - 1, group=group))
    if rank + 1 < world:
        got = torch.empty(recv_numel, dtype=first_row.dtype, device=first_row.device)
        reqs.append(dist.irecv(got, rank + 1, group=group))
    for r in reqs:
        r.wait()
    return got


def forward_distributed(plan, slab, out_slab, rank, world, d_clip=None, group=None):
    """One volume across ranks (one GPU each): slab holds SlabRank.slab_bounds()
    of the volume; out_slab receives the output rows SlabRank.out_rows() at the
    same element offsets.  Returns the SlabRank."""
    import torch

    part = SlabRank(plan, rank, world, device=slab.device)
    info = part.info
    if info["mode"] == part.nat.MCLAHE_RANGE_GLOBAL:   # (a given range makes it a no-op)
        part.range(slab)
        part.set_keys(combine_keys(part.keys(), group))
    part.hist(slab, d_clip)
    n = part.K1 * (part.LS + 2)
    got = exchange_halo(part.first_row_tables(), rank, world, n, group)
    k = part.needs_row()
    if k is not None:
        part.put_row_tables(k, got)
    part.map(slab, out_slab)
    if slab.is_cuda:
        torch.cuda.synchronize(slab.device)
    return part
