"""Multi-GPU launch logic of the coupled step (host side; one process per GPU).

A single lattice has no exchange step that one box would shard: under torchrun
every rank runs an independent replica of the workload with its own seed
(replicas only).  An ensemble shards by realization: rank k runs the
contiguous block [lo_k, hi_k) of the whole ensemble with real_base = lo_k, so
its realizations draw the noise streams of the unsplit run and evolve exactly
as they would there.  No collective touches the data path; the only
collectives are the timing barrier and the reductions of the job's totals.
"""
from __future__ import annotations

import os

import numpy as np


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of n items for this rank; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_workload(w: dict, rank: int, world: int) -> dict:
    """The part of workload w that this rank runs."""
    if world == 1:
        return dict(w)
    if int(w.get("n_real", 1)) > 1:
        lo, hi = shard(int(w["n_real"]), rank, world)
        if hi <= lo:
            raise ValueError("more ranks than realizations")
        return dict(w, n_real=hi - lo, real_base=int(w.get("real_base", 0)) + lo, shard=(lo, hi),
                    full_n_real=int(w["n_real"]))
    return dict(w, seed=int(w["seed"]) + 1000 * rank)


def rank_inputs(w_rank: dict, build_inputs) -> dict:
    """Inputs of this rank's part: the whole ensemble's seeded inputs sliced to
    its realizations (so they are those of the unsplit run), or the inputs of
    its replica."""
    if "shard" not in w_rank:
        return build_inputs(w_rank)
    lo, hi = w_rank["shard"]
    full = build_inputs(dict(w_rank, n_real=w_rank["full_n_real"], real_base=0))
    off = np.asarray(full["offsets"])
    b0, b1 = int(off[lo]), int(off[hi])
    out = dict(full)
    out["offsets"] = (off[lo:hi + 1] - b0).astype(np.int32)
    out["r0"] = np.asarray(full["r0"])[b0:b1]
    return out


def max_over_ranks(x: float, world: int) -> float:
    """Largest x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    """Sum of x over all ranks (units processed by the whole job)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _device():
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


# ---------------------------------------------------------------------------
# One lattice over several handles: x-slabs (the paper's domain
# decomposition, Sec. III, along x).  The library does the slab's work; these
# functions only move the exchanged buffers between handles, in one process
# (several slabs on one device, for tests) or over torch.distributed ranks.
# ---------------------------------------------------------------------------
def slab_partition(nx: int, world: int) -> list[tuple[int, int]]:
    """(first plane, planes) of each of `world` slabs covering [0, nx), as
    equal as possible; every slab holds at least 2 planes."""
    if world < 1 or 2 * world > nx:
        raise ValueError(f"cannot split {nx} planes into {world} slabs of at least 2")
    base, extra = divmod(nx, world)
    out, x0 = [], 0
    for r in range(world):
        w = base + (1 if r < extra else 0)
        out.append((x0, w))
        x0 += w
    return out


def slab_workload(w: dict, rank: int, world: int) -> dict:
    """The workload dict of slab `rank` of `world` (the whole lattice's
    parameters, plus the slab)."""
    out = dict(w)
    out["slab"] = slab_partition(w["nx"], world)[rank]
    return out


def _join(streams, into):
    """Make stream `into` wait for the work queued so far on `streams`."""
    import torch
    for st in streams:
        if st != into:
            ev = torch.cuda.Event()
            ev.record(st)
            into.wait_event(ev)


def slab_step_local(sims: list) -> None:
    """One coupled step of slabs held in this process (in order of x):
    gather, sum u_p, advance, pass the planes on, import.  The copies run on
    the first slab's stream, ordered by events against every slab's own
    stream."""
    import torch
    views = [s.slab_views() for s in sims]
    streams = [s.stream for s in sims]
    tr = streams[0]
    for s in sims:
        s.slab_gather()
    _join(streams, tr)
    with torch.cuda.stream(tr):
        up = views[0]["up"].clone()
        for v in views[1:]:
            up += v["up"]
        for v in views:
            v["up"].copy_(up)
    for st in streams:
        _join([tr], st)
    for s in sims:
        s.slab_advance()
    _join(streams, tr)
    n = len(sims)
    with torch.cuda.stream(tr):
        for r, v in enumerate(views):
            views[(r - 1) % n]["recv_hi"].copy_(v["send_lo"])
            views[(r + 1) % n]["recv_lo"].copy_(v["send_hi"])
    for st in streams:
        _join([tr], st)
    for s in sims:
        s.slab_import()


def exchange_slab_buffers(views: dict, rank: int, world: int, group=None) -> None:
    """The collective part of a slab step over torch.distributed ranks (one
    slab per rank, rank order = x order, periodic): the sum of u_p, then
    send_lo to the left neighbour's recv_hi and send_hi to the right
    neighbour's recv_lo.  With one rank the slab is its own neighbour."""
    import torch.distributed as dist
    if world == 1:
        views["recv_hi"].copy_(views["send_lo"])
        views["recv_lo"].copy_(views["send_hi"])
        return
    left, right = (rank - 1) % world, (rank + 1) % world
    ops = [dist.P2POp(dist.isend, views["send_lo"], left, group, tag=0),
           dist.P2POp(dist.irecv, views["recv_hi"], right, group, tag=0),
           dist.P2POp(dist.isend, views["send_hi"], right, group, tag=1),
           dist.P2POp(dist.irecv, views["recv_lo"], left, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def allreduce_up(views: dict, world: int, group=None) -> None:
    """Sum the u_p partials of all slabs in place (exact: one non-zero term
    per bead)."""
    import torch.distributed as dist
    if world > 1:
        dist.all_reduce(views["up"], group=group)


def slab_step_dist(sim, views: dict, rank: int, world: int, group=None) -> None:
    """One coupled step of this rank's slab; the collectives run on the
    slab's own stream, in order with its kernels."""
    import torch
    with torch.cuda.stream(sim.stream):
        sim.slab_gather()
        allreduce_up(views, world, group)
        sim.slab_advance()
        exchange_slab_buffers(views, rank, world, group)
        sim.slab_import()
