"""Serving: continuous batching of independent runs through sph_server_*.

Each served result must equal the same request run alone through a context
(sph_setup, sph_density_h, sph_forces, then its steps): the batched step
gives bit-identical per-problem results, so the comparison is exact.  Also
checks admission by memory budget, overlap of requests that arrive while
others run, and the too-big rejection."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _alone(S, req):
    prob = S.Problem(req["arrays"], S.make_params(S.PREC_MIXED, **req["params"]))
    prob.density_h()
    prob.forces()
    for _ in range(req["nsteps"]):
        prob.step(-1.0)
    out = prob.numpy("x", "vx", "u", "h", "rho")
    prob.close()
    return out


def test_served_results_equal_alone(S):
    from paper_1709_04488_gb300 import serve
    reqs = serve.make_requests(8, seed=11, n_min=1e3, n_max=2e4, nsteps=4)
    arrivals = np.array([0.0, 0.0, 0.0, 1e-4, 2e-4, 3e-4, 4e-4, 5e-4])
    srv = serve.Server(2 << 30, max_slots=16)
    tickets = [srv.submit(r["arrays"], r["params"], r["nsteps"], t) for r, t in zip(reqs, arrivals)]
    srv.run(virtual_clock=True)
    overlapped = 0
    recs = []
    for r, tk in zip(reqs, tickets):
        o = srv.poll(tk, len(r["arrays"]["x"]), want_state=True)
        assert o is not None and o["status"] == S.OK and o["steps_done"] == r["nsteps"]
        recs.append(o)
    for k, o in enumerate(recs):
        ref = _alone(S, reqs[k])
        for f in ("x", "vx", "u", "h", "rho"):
            assert np.array_equal(o[f], ref[f]), (k, f)
    # requests that arrived later were admitted while earlier ones were resident
    for k in range(3, 8):
        if any(recs[j]["admitted"] <= recs[k]["admitted"] < recs[j]["completed"] for j in range(3)):
            overlapped += 1
    assert overlapped >= 1
    srv.close()


def test_admission_by_memory_budget(S):
    """A pool that holds two requests at a time (footprint: particle arrays,
    own workspace and the batch-workspace share): the others wait in the
    queue, are admitted as memory frees up, and all finish correctly."""
    from paper_1709_04488_gb300 import ics, serve
    reqs = []
    for k in range(5):
        a, p = ics.lattice(16, seed=50 + k)
        reqs.append({"arrays": a, "params": p, "nsteps": 2})
    n = 4096
    ws = S.sph_workspace_bytes(n, S.make_params(S.PREC_MIXED))
    foot = 18 * 8 * n + 18 * 256 + 2 * ws + 1024
    srv = serve.Server(int(2.5 * foot), max_slots=16)
    tickets = [srv.submit(r["arrays"], r["params"], r["nsteps"], 0.0) for r in reqs]
    srv.run(virtual_clock=True)
    recs = [srv.poll(t, n) for t in tickets]
    assert all(o is not None and o["status"] == S.OK for o in recs)
    admitted = sorted(o["admitted"] for o in recs)
    assert admitted[1] == admitted[0] == 0.0  # two fit at once
    assert admitted[2] > 0.0                  # the third waited for a retirement
    srv.close()


def test_too_big_and_busy(S):
    from paper_1709_04488_gb300 import serve
    reqs = serve.make_requests(2, seed=13, n_min=3e4, n_max=3e4, nsteps=1)
    srv = serve.Server(1 << 20, max_slots=4, max_queue=1)
    with pytest.raises(S.SPHError) as e:
        srv.submit(reqs[0]["arrays"], reqs[0]["params"], 1, 0.0)
    assert e.value.code == S.ETOOBIG
    srv.close()


def test_one_failing_request_fails_alone(S):
    """A request that cannot converge (four isolated particles) is served
    beside three healthy ones: it comes back with an error status, and the
    healthy ones finish with SPH_OK and the same bits as each run alone (each
    request takes its own problem's status, not the batch's)."""
    from paper_1709_04488_gb300 import serve
    reqs = serve.make_requests(3, seed=17, n_min=1e3, n_max=8e3, nsteps=3)
    rng = np.random.default_rng(0)
    bad = {k: rng.uniform(0, 1, 4) for k in ("x", "y", "z")}
    bad.update(vx=np.zeros(4), vy=np.zeros(4), vz=np.zeros(4), u=np.ones(4), m=np.ones(4), h=np.full(4, 0.1))
    srv = serve.Server(1 << 30, max_slots=8)
    tickets = [srv.submit(r["arrays"], r["params"], r["nsteps"], 0.0) for r in reqs[:2]]
    tb = srv.submit(bad, {"periodic": False, "box_lo": (0.0, 0.0, 0.0), "box_len": (0.0, 0.0, 0.0),
                          "eos": "adiabatic", "gamma": 5.0 / 3.0}, 3, 0.0)
    tickets.append(srv.submit(reqs[2]["arrays"], reqs[2]["params"], reqs[2]["nsteps"], 0.0))
    srv.run(virtual_clock=True)
    ob = srv.poll(tb, 4)
    assert ob is not None and ob["status"] != S.OK
    for r, tk in zip(reqs, tickets):
        o = srv.poll(tk, len(r["arrays"]["x"]), want_state=True)
        assert o is not None and o["status"] == S.OK and o["steps_done"] == r["nsteps"]
        ref = _alone(S, r)
        for f in ("x", "vx", "u", "h", "rho"):
            assert np.array_equal(o[f], ref[f]), f
    srv.close()


def test_zero_step_request_is_rejected(S):
    from paper_1709_04488_gb300 import serve
    reqs = serve.make_requests(1, seed=19, n_min=1e3, n_max=1e3, nsteps=1)
    srv = serve.Server(1 << 28, max_slots=4)
    with pytest.raises(S.SPHError) as e:
        srv.submit(reqs[0]["arrays"], reqs[0]["params"], 0, 0.0)
    assert e.value.code == S.EINVAL
    srv.close()
