"""Multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1), no GPU.

Under torchrun every rank times its own problem (weak scaling, no data-path
collective); the whole-job number uses the slowest rank's time, and only rank
0 prints.  The reference arm (the oracle on the host cores) runs on rank 0
alone; the other ranks return without work.
"""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    t_max = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(2.0e9, world, t_max)
    # the reference arm: rank != 0 returns at once and prints nothing
    buf = io.StringIO()
    if rank != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "gpus": world})(), rank)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{t_max} {rate} {len(buf.getvalue())}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        t_max, rate, printed = open(tmp_path / f"rank{rank}.txt").read().split()
        assert float(t_max) == 15.0
        # 2 ranks x 2e9 units in 15 ms
        assert abs(float(rate) - 2 * 2.0e9 / 15e-3 / 1e9) < 1e-9
        assert int(printed) == 0


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert abs(bench.whole_job_rate(16777216 * 32 * 20, 1, 173.0) - 62.06) < 0.01
