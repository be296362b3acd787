"""The multi-GPU path of bench.py is replicas only: every rank solves its own
problems and the job reports its slowest rank's time.  The aggregation over
ranks runs here on CPU with two gloo ranks (no GPU, no NCCL)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        # rank-dependent timings: ms, e2e seconds, serial e2e seconds
        mine = [10.0 + 5.0 * rank, 2.0 - rank, 3.0 + rank]
        got = bench.slowest_rank(mine, torch.device("cpu"), w)
        q.put((r, w, got, bench.whole_job_rate(w, 1000, 7, got[0] * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, got, rate in out:
        assert w == world
        # element-wise maximum over the ranks, the same on every rank
        assert got == [15.0, 2.0, 4.0]
        # whole job: both replicas' points over the slowest time
        assert rate == pytest.approx(world * 1000 * 7 / 15e-3)
    assert sorted(r for r, *_ in out) == [0, 1]


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.slowest_rank([1.5, 2.5], torch.device("cpu"), 1) == [1.5, 2.5]
    assert bench.whole_job_rate(1, 100, 4, 2.0) == 200.0
