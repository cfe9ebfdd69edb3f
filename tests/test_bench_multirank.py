"""The benchmark's multi-rank bookkeeping on two CPU ranks (gloo over
127.0.0.1): the barrier, the max over ranks of the timed region, the
whole-job value (units of all ranks / the slowest rank's time), and the
reference arm running on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), GNB_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_init()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    # rank r's timed region: 100 ms + 25 ms per rank; the slowest decides
    tmax = bench.reduce_max(100.0 + 25.0 * r, w)
    value = bench.whole_job_value(1 << 20, 10, w, tmax)
    out.put((r, tmax, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0), (r1, t1, v1) = res
    assert t0 == t1 == 125.0  # both ranks see the slower rank's time
    expect = (1 << 20) * 10 * 2 / 0.125  # particle-steps of both replicas per second
    assert abs(v0 - expect) < 1e-6 * expect and v0 == v1


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, config = 1, 0, "tiny"

    # ranks other than 0 return without work and print nothing
    assert bench.run_reference(A(), 2, 1, 0) is None
