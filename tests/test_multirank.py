"""The multi-GPU path of bench.py (replicas, one process per GPU) on CPU: two gloo ranks.

Solves are independent, so ranks exchange only the timing and the count of converged solves:
each rank draws its own seeded batch, the job's time is the slowest rank's (max) and its work is
the sum over ranks.  The reference arm runs on rank 0 alone.
"""

import argparse
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    probs, cfg = bench.make_workload("batch", rank, argparse.Namespace(instances=3))
    slowest = bench.reduce_over_ranks(10.0 * (rank + 1), "max", "cpu")
    total = bench.reduce_over_ranks(rank + 1, "sum", "cpu")
    q.put((rank, [float(p.phi.sum()) for p in probs], cfg["instances"], slowest, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_draw_their_own_batches_and_reduce_time_and_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, sums0, n0, mx0, tot0), (r1, sums1, n1, mx1, tot1) = got
    assert (r0, r1) == (0, 1) and n0 == n1 == 3
    assert sums0 != sums1                      # each rank's own seeded batch
    assert mx0 == mx1 == 20.0                  # the slowest rank's time, on every rank
    assert tot0 == tot1 == 3.0                 # every rank's work



def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main() == 0
    assert buf.getvalue() == ""
