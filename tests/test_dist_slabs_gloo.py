"""Host logic of the x-slab split of one lattice (the paper's domain
decomposition, Sec. III, along x) on CPU ranks (gloo): the partition covers
the lattice with slabs of at least two planes; the exchange hands every
rank's send_lo to its left neighbour's recv_hi and its send_hi to its right
neighbour's recv_lo (periodic in x), and the u_p partials are summed.  The
buffers here are CPU tensors of the slab buffers' shapes, filled with values
that name their rank, plane and population."""
import os
import socket

import pytest
import torch

from paper_0711_2665_gb300 import dist as pdist


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _views(rank, ny=5, nz=3, beads=7):
    def tag(planes, which):
        t = torch.arange(19 * planes * nz * ny, dtype=torch.float32).reshape(19, planes, nz, ny)
        return t + 1e5 * (rank + 1) + 1e4 * which
    up = torch.zeros(beads, 4)
    up[rank::3, :3] = float(rank + 1)  # each bead non-zero on one rank (3 ranks at most)
    return {"up": up, "send_lo": tag(2, 1), "send_hi": tag(1, 2),
            "recv_lo": torch.full((19, 1, nz, ny), -1.0), "recv_hi": torch.full((19, 2, nz, ny), -1.0)}


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = _views(rank)
        pdist.allreduce_up(v, world)
        pdist.exchange_slab_buffers(v, rank, world)
        q.put((rank, v["up"].tolist(), v["recv_lo"].tolist(), v["recv_hi"].tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_exchange_over_gloo_ranks(world):
    import multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {r: (up, lo, hi) for r, up, lo, hi in (q.get(timeout=300) for _ in range(world))}
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want_up = sum(_views(r)["up"] for r in range(world))
    for r in range(world):
        up, lo, hi = (torch.tensor(x) for x in res[r])
        assert torch.equal(up, want_up)
        assert torch.equal(hi, _views((r + 1) % world)["send_lo"])   # right neighbour's first planes
        assert torch.equal(lo, _views((r - 1) % world)["send_hi"])   # left neighbour's last plane


def test_single_rank_is_its_own_neighbour():
    v = _views(0)
    pdist.exchange_slab_buffers(v, 0, 1)
    assert torch.equal(v["recv_hi"], v["send_lo"]) and torch.equal(v["recv_lo"], v["send_hi"])


def test_slab_partition():
    for nx in (4, 5, 40, 256):
        for world in (1, 2, 3, 8):
            if 2 * world > nx:
                with pytest.raises(ValueError):
                    pdist.slab_partition(nx, world)
                continue
            parts = pdist.slab_partition(nx, world)
            assert parts[0][0] == 0 and sum(w for _, w in parts) == nx
            assert all(a[0] + a[1] == b[0] for a, b in zip(parts, parts[1:]))
            assert min(w for _, w in parts) >= 2 and max(w for _, w in parts) - min(w for _, w in parts) <= 1
    w = pdist.slab_workload({"nx": 40, "ny": 8}, 1, 3)
    assert w["slab"] == (14, 13) and w["nx"] == 40
