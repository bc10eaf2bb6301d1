"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
steps its own replica (no data-path collective), the timing takes the slowest
rank, and the whole-job value counts every rank's updates.  The GPU work of a
rank cannot run here; the rank bookkeeping around it does."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [12.5, 20.0][rank]  # per-rank timed totals (ms)
    slowest = bench.reduce_max_ms(mine, world, dist, torch.device("cpu"))
    q.put((rank, bench.dist_env(), slowest, bench.replica_value(36864, 10, world, slowest)))
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_the_whole_job():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        rank, env, slowest, value = q.get(timeout=120)
        got[rank] = (env, slowest, value)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        env, slowest, value = got[rank]
        assert env == (rank, 2, rank)
        assert slowest == 20.0
        assert value == pytest.approx(2 * 36864 * 10 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_ms(7.0, 1) == 7.0
    assert bench.replica_value(1000, 5, 1, 10.0) == pytest.approx(5e5)
