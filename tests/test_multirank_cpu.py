"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
steps its own replica (no data-path collective), the timing takes the slowest
rank, and the whole-job value counts every rank's updates.  The GPU work of a
rank cannot run here; the rank bookkeeping around it does."""
import os
import socket
import sys

import numpy as np
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


def _oracle_worker(rank, world, port, q):
    """Each rank steps its own problem (a lattice with a rank-dependent jitter
    seed) through the oracle, times it, and the ranks gather their results
    and times over gloo, as bench.py's replicas do over NCCL."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import time
    import torch.distributed as dist
    import bench
    import oracle as O
    from paper_1709_04488_gb300 import ics
    O.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, p = ics.lattice(8, seed=10 + rank)
    P = O.Params(**p)
    s = O.State(**a)
    t0 = time.perf_counter()
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    for _ in range(3):
        assert O.step(P, s, O.cfl_dt(P, s)) == O.OK
    ms = 1e3 * (time.perf_counter() - t0)
    slowest = bench.reduce_max_ms(ms, world, dist, torch.device("cpu"))
    mine = {"rank": rank, "ms": ms, "x": s.x.copy(), "vx": s.vx.copy(), "rho": s.rho.copy()}
    allr = [None] * world
    dist.all_gather_object(allr, mine)
    if rank == 0:
        q.put((allr, slowest, bench.replica_value(s.n, 4, world, slowest)))
    dist.destroy_process_group()


def test_two_ranks_step_their_own_problems_through_the_oracle(oracle_mod):
    """Gathered per-rank results equal the same problems stepped in one
    process (bit for bit: the oracle's sums do not depend on the process),
    the timing is the slowest rank's, and the whole-job value counts both
    ranks' particle updates (one evaluation and three steps each)."""
    O = oracle_mod
    from paper_1709_04488_gb300 import ics
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allr, slowest, value = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r["rank"] for r in allr] == [0, 1]
    assert slowest == max(r["ms"] for r in allr)
    assert value == pytest.approx(2 * 512 * 4 / (slowest * 1e-3))
    for r in allr:
        a, p = ics.lattice(8, seed=10 + r["rank"])
        P = O.Params(**p)
        s = O.State(**a)
        assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
        for _ in range(3):
            assert O.step(P, s, O.cfl_dt(P, s)) == O.OK
        assert np.array_equal(r["x"], s.x) and np.array_equal(r["vx"], s.vx)
        assert np.array_equal(r["rho"], s.rho)
    # the two ranks stepped different problems
    assert not np.array_equal(allr[0]["x"], allr[1]["x"])


def test_route_covers_and_balances_requests():
    """Multi-GPU serving: every request goes to exactly one GPU, the same
    stream routes the same way every time, saturated queues are balanced
    within one request's work, and with arrivals spread out a request goes
    to an idle GPU."""
    from paper_1709_04488_gb300 import serve
    reqs = serve.make_requests(40, seed=3, n_min=1e3, n_max=2e4, nsteps=10)
    work = np.array([len(r["arrays"]["x"]) * r["nsteps"] for r in reqs], dtype=float)
    for nr in (1, 2, 3, 4):
        rt = serve.route(reqs, np.zeros(len(reqs)), nr)
        assert rt.min() >= 0 and rt.max() < nr
        assert np.array_equal(rt, serve.route(reqs, np.zeros(len(reqs)), nr))
        load = np.array([work[rt == r].sum() for r in range(nr)])
        assert load.max() - load.min() <= work.max()
    # arrivals far apart (each request done before the next arrives): all on GPU 0
    rt = serve.route(reqs, np.arange(len(reqs)) * 10.0, 3)
    assert np.all(rt == 0)
    with pytest.raises(ValueError):
        serve.route(reqs, np.zeros(len(reqs)), 0)


def _route_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_1709_04488_gb300 import serve
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reqs = serve.make_requests(30, seed=4, n_min=1e3, n_max=2e4, nsteps=10)
    arr = serve.poisson_arrivals(30, 50.0, seed=6)
    rt = serve.route(reqs, arr, world, rate=2e6)
    mine = [i for i in range(len(reqs)) if rt[i] == rank]
    allr = [None] * world
    dist.all_gather_object(allr, (rank, rt.tolist(), mine))
    if rank == 0:
        q.put(allr)
    dist.destroy_process_group()


def test_two_ranks_route_the_same_stream_the_same_way():
    """Each rank routes the shared request stream by itself: the two
    assignments agree, and the ranks' shares partition the requests."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_route_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allr = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert allr[0][1] == allr[1][1]
    shares = [set(a[2]) for a in allr]
    assert shares[0].isdisjoint(shares[1]) and shares[0] | shares[1] == set(range(30))
    assert len(shares[0]) > 0 and len(shares[1]) > 0


def _serving_worker(rank, world, port, q):
    """bench.py's serving leg on two gloo ranks, with the GPU server replaced
    by a stand-in that finishes each request at its arrival plus its work at
    a fixed rate (the routing and the gathering of the ranks' records run as
    they do on GPUs)."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    from paper_1709_04488_gb300 import serve

    def fake_run_stream(reqs, arrivals, pool_bytes, **kw):
        t, recs = 0.0, []
        for r, a in sorted(zip(reqs, arrivals), key=lambda x: x[1]):
            t = max(t, a) + len(r["arrays"]["x"]) * r["nsteps"] / 1e8
            recs.append({"status": 0, "latency": t - a})
        return recs, t

    serve.run_stream = fake_run_stream
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = bench.serving(12, [0.5], 0, rank, world, dist)
    q.put((rank, out))
    dist.destroy_process_group()


def test_serving_leg_routes_and_gathers_across_ranks():
    """Every rank serves its routed share; the whole job's saturated
    throughput is all the work over the slowest rank's makespan, and the
    latency percentiles cover every request of the stream."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out = got[0]
    assert out == got[1]  # the gathered records are the same on every rank
    assert out["requests"] == 12 and out["gpus"] == 2
    assert out["saturated_updates_per_s"] == pytest.approx(out["particle_steps"] / out["saturated_makespan_s"])
    # two GPUs at 1e8 each: the routed saturated stream takes about half the work time of one
    assert out["saturated_makespan_s"] < 0.75 * out["particle_steps"] / 1e8
    assert len(out["loads"]) == 1 and out["loads"][0]["p99_s"] >= out["loads"][0]["p50_s"] > 0
