"""The multi-GPU host logic on two CPU ranks (gloo): an ensemble splits into
disjoint contiguous blocks of realizations that cover it, with real_base set
so that the noise streams are those of the unsplit run and inputs that are
slices of the unsplit inputs; a single lattice runs as replicas with distinct
seeds; the job's time is the slowest rank's and its units the sum over ranks."""
import os
import socket

import numpy as np
import pytest

from paper_0711_2665_gb300 import dist as pdist
from paper_0711_2665_gb300 import workloads


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ens = pdist.rank_workload(workloads.get("ensemble_fp32"), rank, world)
        plain = pdist.rank_workload(workloads.get("plain_fp32"), rank, world)
        tmax = pdist.max_over_ranks(10.0 + 3.0 * rank, world)
        units = pdist.sum_over_ranks(ens["n_real"] * 1000.0, world)
        inp = pdist.rank_inputs(ens, workloads.build_inputs)
        q.put((rank, ens["shard"], ens["real_base"], ens["n_real"], ens["seed"], plain["seed"], tmax, units,
               inp["offsets"].tolist(), np.asarray(inp["r0"]).tolist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    import multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    full_w = workloads.get("ensemble_fp32")
    full = workloads.build_inputs(full_w)
    (r0_, sh0, base0, n0, es0, ps0, t0, u0, off0, x0), (r1_, sh1, base1, n1, es1, ps1, t1, u1, off1, x1) = res
    assert sh0 == (0, 32) and sh1 == (32, 64) and base0 == 0 and base1 == 32 and n0 == n1 == 32
    assert es0 == es1 == full_w["seed"]                 # one ensemble, one seed
    assert ps0 != ps1                                    # replicas differ
    assert t0 == t1 == 13.0 and u0 == u1 == 64 * 1000.0  # slowest rank, whole job
    off = np.asarray(full["offsets"])
    assert np.array_equal(np.asarray(off0), off[:33])
    assert np.array_equal(np.asarray(off1), off[32:] - off[32])
    assert np.array_equal(np.concatenate([np.asarray(x0), np.asarray(x1)]), np.asarray(full["r0"]))


def test_shard_blocks():
    for n in (1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            blocks = [pdist.shard(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pdist.shard(4, 4, 4)
    w = workloads.get("plain_fp32")
    assert pdist.rank_workload(w, 0, 1) == w
