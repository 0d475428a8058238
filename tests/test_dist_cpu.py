"""The benchmark's multi-process plumbing on CPU (gloo, world size 2).

bench.py runs one replica per GPU under torchrun: a barrier brackets the timed
region, the slowest rank's time is taken (max over ranks) and the whole-job
value counts every rank's units.  These are checked here with two CPU ranks
on the gloo backend (no GPU); the reference arm's rule that only rank 0 runs
is checked too.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, w)   # rank 1 is the slow one
    out.put((rank, ms, bench.job_value(1000, ms, w)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_max_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, val in res:
        assert ms == 15.0                              # every rank sees the slowest time
        assert val == pytest.approx(2 * 1000 / 15e-3)  # both ranks' units over that time


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup(1) == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(10, 2.0, 1) == pytest.approx(5000.0)
