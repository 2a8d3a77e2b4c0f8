"""The multi-process plumbing of bench.py (one process per GPU, launched by
torchrun) exercised on CPU: two gloo ranks join the group, meet at the
barrier, take the job time as the maximum and the work as the sum over
ranks, seed different queries, and only rank 0 runs the reference arm.  The
localization path has no collective (queries are independent), so nothing
else crosses ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    r, w, local = bench.dist_setup(world, backend="gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    out[rank] = (bench.max_over_ranks(10.0 + rank, w), bench.sum_over_ranks(100.0 * (rank + 1), w),
                 bench.rank_seed(100, r))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 11.0           # the job's time: the slowest rank
    assert out[0][1] == out[1][1] == 300.0          # the job's work: every rank's
    assert out[0][2] != out[1][2]                   # different queries per rank


def _reference_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse
    import contextlib
    import io

    import bench

    called = []
    bench.oracle_queries = lambda *a, **k: called.append(1) or (1.0, 10)
    bench.make_queries = lambda n, seed: [None] * n
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(argparse.Namespace(gpus=world, steps=2, warmup=3, queries=16))
    out[rank] = (rc, buf.getvalue(), len(called))


def test_reference_arm_runs_on_rank_0_only():
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.spawn(_reference_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    rc0, text0, calls0 = out[0]
    rc1, text1, calls1 = out[1]
    assert rc0 == 0 and rc1 == 0
    assert '"impl": "reference"' in text0 and calls0 > 0
    assert text1 == "" and calls1 == 0
