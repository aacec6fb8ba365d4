"""The bench's multi-rank path on CPU: world size 2 over gloo (replicas, no data-path collective).

Every rank solves its own replica; the job's time is the slowest rank's (an all-reduce MAX of
one scalar), the job's value counts every rank's solves, and only rank 0 prints. Ranks are
spawned processes (start method spawn) rendezvousing on 127.0.0.1.
"""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        # per-rank times differ: the job's time is the largest
        t = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"), w)
        value = bench.job_value(w, 3, t)
        # the reference arm runs on rank 0 only; other ranks leave without work or output
        class A:
            omega, ref_iterations, warmup, steps, gpus = 1e-4, 25, 0, 1, w
        ref_rc = bench.run_reference(A) if r != 0 else None
        out.put((r, w, local, t, value, ref_rc))
    finally:
        dist.destroy_process_group()


def test_replica_timing_and_value_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, t, value, _ in res:
        assert t == 15.0                       # the slowest rank's time on both ranks
        assert value == pytest.approx(2 * 3 / 15.0)
    assert res[1][5] == 0                      # rank 1: reference arm returns at once


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.5, torch.device("cpu"), 1) == 7.5
    assert bench.job_value(1, 5, 2.0) == 2.5
