"""Multi-GPU bench path on CPU: replicas only (every rank solves its own copy of
the workload, no data-path collective), so N ranks report N x the units over the
slowest rank's time.  Two gloo ranks exercise the max-over-ranks reduction and
the reference arm's rank-0-only output."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank              # rank 1 is the slowest
        ms = bench.max_over_ranks(ms_local, world, "cpu")
        value = bench.replica_throughput(5, ms, world)
        w, r, loc = bench.dist_setup(None)
        # the reference arm prints on rank 0 only; other ranks leave without work
        buf = io.StringIO()
        if r != 0:
            with redirect_stdout(buf):
                bench.reference_arm(None, w, r)
        q.put((rank, ms, value, (w, r, loc), buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, 29517
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, env, out in res:
        assert ms == 150.0                           # max over ranks on every rank
        assert value == pytest.approx(2 * 5 / 0.150)
        assert env == (2, rank, rank)
        if rank != 0:
            assert out == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(123.0, 1) == 123.0
    assert bench.replica_throughput(5, 1000.0, 1) == pytest.approx(5.0)
