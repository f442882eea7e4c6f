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
