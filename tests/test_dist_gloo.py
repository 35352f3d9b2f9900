"""Multi-rank benchmark logic on CPU with the gloo backend (world size 2):
the whole-job rate takes the slowest rank's time, every rank simulates its own
independent envs, and the reference arm prints from rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.dist_max(0.25 * (rank + 1), device="cpu")
    dist.barrier()
    rate = bench.whole_job_rate(1 << 20, world, 100, t)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    out[rank] = (t, rate, seeds)
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_independent_seeds():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, rate, seeds = res[rank]
        assert t == pytest.approx(0.5)
        assert rate == pytest.approx((1 << 20) * 2 * 100 / 0.5)
        assert len(set(seeds)) == world


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    assert buf.getvalue() == ""
