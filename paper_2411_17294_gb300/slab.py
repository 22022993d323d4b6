"""Halo exchange of a slab decomposition (one periodic domain cut along its
slowest axis, one slab per rank).

The paper runs its solver on MPI ranks over partitioned meshes (Section 5,
experimental setup); here every rank owns a slab handle (tfs.Solver on the
slab's grid) and, before each step, sends its first two planes to the lower
neighbour and its last two to the upper one (tfs_get_halo), receiving the
neighbours' planes as its own halo_lo / halo_hi for tfs_step_slab.  The
domain is periodic, so the ranks form a ring.  This module is the exchange
only: argument marshalling for torch.distributed point-to-point messages (NCCL
on GPU tensors, gloo on host tensors), no arithmetic.
"""
from __future__ import annotations

TAG_DOWN, TAG_UP = 7101, 7102     # planes travelling to the lower / upper neighbour


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """(lower, upper) neighbour ranks on the periodic ring."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """Ring exchange of boundary planes: send_lo (this slab's first planes) goes
    to the lower neighbour, which receives it as its recv_hi; send_hi goes to
    the upper neighbour, which receives it as its recv_lo.  Blocks until the
    four messages are done.  One rank: the domain wraps onto itself."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist
    lower, upper = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, send_lo, lower, group, TAG_DOWN),
           dist.P2POp(dist.irecv, recv_hi, upper, group, TAG_DOWN),
           dist.P2POp(dist.isend, send_hi, upper, group, TAG_UP),
           dist.P2POp(dist.irecv, recv_lo, lower, group, TAG_UP)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def exchange_local(sends):
    """The same exchange among slabs held by one process: sends[k] = (lo, hi)
    of slab k in ring order; returns [(recv_lo, recv_hi)] with recv_lo[k] =
    hi of slab k-1 and recv_hi[k] = lo of slab k+1 (device-to-device copies)."""
    n = len(sends)
    return [(sends[(k - 1) % n][1].clone(), sends[(k + 1) % n][0].clone()) for k in range(n)]
