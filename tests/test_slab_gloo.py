"""The halo exchange of the slab decomposition across ranks (gloo, CPU, no
GPU): a periodic field cut into slabs along its slowest axis, one slab per
rank; each rank packs its boundary planes as tfs_get_halo lays them out
([2 levels][nc][2 planes][plane]), exchanges them with slab.exchange, and must
receive exactly the neighbours' planes of the whole field (periodic ring),
for two and three ranks and uneven slabs."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _field(dim, n, nc, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(2, nc) + tuple(reversed(n)))   # [level][c][slow]...[x]


def _pack(part, planes):
    """[level][c][slow][...] -> [level][c][R][plane] of the given slow-axis planes."""
    sel = part[:, :, planes]
    return np.ascontiguousarray(sel.reshape(sel.shape[0], sel.shape[1], len(planes), -1))


def _rank_main(rank, world, port, dim, n, slabs, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2411_17294_gb300 import slab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nc = 3 if dim == 2 else 6
    F = _field(dim, n, nc, 77)
    starts = np.cumsum((0,) + tuple(slabs))
    k0, k1 = starts[rank], starts[rank + 1]
    mine = F[:, :, k0:k1]
    send_lo = torch.from_numpy(_pack(mine, list(range(R)))).reshape(-1)
    send_hi = torch.from_numpy(_pack(mine, list(range(k1 - k0 - R, k1 - k0)))).reshape(-1)
    recv_lo, recv_hi = torch.empty_like(send_lo), torch.empty_like(send_hi)
    slab.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world)
    ns = n[-1]
    want_lo = _pack(F, [(k0 - R + i) % ns for i in range(R)]).reshape(-1)
    want_hi = _pack(F, [(k1 + i) % ns for i in range(R)]).reshape(-1)
    ok = np.array_equal(recv_lo.numpy(), want_lo) and np.array_equal(recv_hi.numpy(), want_hi)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dim,n,slabs", [(3, (4, 3, 8), (4, 4)), (2, (5, 9), (3, 4, 2)), (3, (2, 2, 7), (2, 3, 2))])
def test_ring_exchange_delivers_neighbour_planes(tmp_path, dim, n, slabs):
    mp = pytest.importorskip("torch.multiprocessing")
    world = len(slabs)
    mp.start_processes(_rank_main, args=(world, _free_port(), dim, n, slabs, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for rank in range(world):
        assert open(tmp_path / f"rank{rank}.txt").read() == "ok", rank


def test_single_rank_wraps_onto_itself():
    import torch
    sys.path.insert(0, ROOT)
    from paper_2411_17294_gb300 import slab
    lo, hi = torch.arange(6.0), torch.arange(6.0) + 10
    rlo, rhi = torch.empty(6), torch.empty(6)
    slab.exchange(lo, hi, rlo, rhi, 0, 1)
    assert torch.equal(rlo, hi) and torch.equal(rhi, lo)
    assert slab.neighbours(0, 3) == (2, 1) and slab.neighbours(2, 3) == (1, 0)
