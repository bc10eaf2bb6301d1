"""The resident batch (sph_batch_*): many independent problems of uneven sizes
stepped by one captured graph per batch, each result equal to the problem
stepped alone; per-problem statuses; a context stepped alone after batched
steps (with tree reuse) still matches the oracle."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

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


def _moving_lattice(n_side, seed, vel=0.3):
    a, p = ics.lattice(n_side, seed=seed)
    rng = np.random.default_rng(seed + 100)
    for c in ("vx", "vy", "vz"):
        a[c] = rng.normal(0.0, vel, len(a["x"]))
    a["u"] = a["u"] * (1.0 + 0.2 * rng.uniform(-1, 1, len(a["x"])))
    return a, p


def _cases():
    return [_moving_lattice(10, seed=7), ics.sod(left=(32, 16, 16), right=(16, 8, 8), width=0.25),
            _moving_lattice(14, seed=8), ics.sedov(12, seed=9), ics.cloud(5000, seed=10)]


def _prob(S, a, p, stream, **kw):
    prob = S.Problem(a, S.make_params(S.PREC_MIXED, **p, flags=S.FLAG_ASYNC, **kw), stream=stream)
    prob.density_h()
    prob.forces()
    prob.sync()
    return prob


def test_resident_batch_graph_equals_alone(S):
    """Five problems (lattices, a Sod tube, a Sedov blast, an isolated cloud)
    in one resident batch: the first step runs eagerly and is captured, the
    next ones replay the graph; after 4 steps every state equals the same
    problem stepped alone, bit for bit."""
    import torch
    st = torch.cuda.Stream()
    cases = _cases()
    alone = []
    for a, p in cases:
        prob = _prob(S, a, p, st)
        for _ in range(4):
            prob.step(-1.0)
        alone.append(prob.numpy())
        prob.close()
    probs = [_prob(S, a, p, st) for a, p in cases]
    batch = S.Batch(probs, flags=S.FLAG_TIMING)
    batch.run(1)
    batch.run(3)
    assert batch.sync() == [S.OK] * len(probs)
    assert batch.kernel_count() > 5
    assert batch.stage_times()[S.STAGES.index("forces")] > 0
    for pr, ref in zip(probs, alone):
        g = pr.numpy()
        for f in ("x", "vx", "u", "h", "rho", "ax", "du", "vsig"):
            assert np.array_equal(g[f], ref[f]), f
    batch.close()


def test_resident_batch_reports_each_problems_status(S):
    """A problem that cannot converge (four isolated particles: no h gives
    Eq. HRHO's neighbour mass) fails on its own: its status is an error
    (SPH_ENOCONV, or SPH_ENONFINITE once its state has blown up), the others
    report SPH_OK and equal their states stepped alone."""
    import torch
    st = torch.cuda.Stream()
    rng = np.random.default_rng(0)
    bad = {k: rng.uniform(0, 1, 4) for k in ("x", "y", "z")}
    bad.update(vx=np.zeros(4), vy=np.zeros(4), vz=np.zeros(4), u=np.ones(4), m=np.ones(4), h=np.full(4, 0.1))
    good = [_moving_lattice(10, seed=11), ics.sedov(12, seed=12)]
    alone = []
    for a, p in good:
        prob = _prob(S, a, p, st)
        for _ in range(2):
            prob.step(-1.0)
        alone.append(prob.numpy())
        prob.close()
    pb = S.Problem(bad, S.make_params(S.PREC_MIXED, periodic=False, flags=S.FLAG_ASYNC), stream=st)
    pb.density_h()
    pb.forces()
    pb.sync(allow=(S.ENOCONV,))
    probs = [_prob(S, *good[0], st), pb, _prob(S, *good[1], st)]
    batch = S.Batch(probs)
    batch.run(2)
    st = batch.sync()
    assert st[0] == S.OK and st[2] == S.OK and st[1] in (S.ENOCONV, S.ENONFINITE), st
    for pr, ref in zip((probs[0], probs[2]), alone):
        g = pr.numpy()
        for f in ("x", "vx", "u", "rho", "ax"):
            assert np.array_equal(g[f], ref[f]), f
    batch.close()


def test_alone_step_with_tree_reuse_after_batched_steps(S, oracle_mod):
    """After batched steps (which sort every problem in the batch's layout),
    a context stepped alone with tree reuse rebuilds its leaves first and
    matches the oracle stepped with the same time-steps."""
    import torch
    O = oracle_mod
    st = torch.cuda.Stream()
    a, p = _moving_lattice(12, seed=13)
    P = O.Params(**p)
    ref = O.State(**a)
    assert O.density(P, ref) == O.OK and O.forces(P, ref) == O.OK
    prob = _prob(S, a, p, st, tree_rebuild_every=3)
    other = _prob(S, *_moving_lattice(9, seed=14), st)
    wb = S.sph_batch_workspace_bytes([prob.ctx, other.ctx])
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    dts = []
    for _ in range(2):
        dts.append(prob.diagnostics().dt_next)
        S.check(S.sph_batch_step([prob.ctx, other.ctx], 1, ws.data_ptr(), wb), "sph_batch_step")
    for _ in range(3):
        dt = prob.diagnostics().dt_next
        dts.append(dt)
        prob.step(dt)
    for dt in dts:
        assert O.step(P, ref, dt) == O.OK
    g = prob.numpy()
    assert np.max(np.abs(g["rho"] / ref.rho - 1.0)) < 1e-5
    ra = np.stack([ref.ax, ref.ay, ref.az], 1)
    ga = np.stack([g["ax"], g["ay"], g["az"]], 1)
    assert np.max(np.linalg.norm(ga - ra, axis=1)) < 1e-4 * np.sqrt(np.mean(np.sum(ra ** 2, 1)))


def test_block_step_with_tree_reuse_after_batched_steps(S, oracle_mod):
    """A block step with tree reuse starts from the context's leaves; after a
    batched step (which sorts the problems in the batch's layout) it builds
    them first, and matches the oracle's block step from the same state."""
    import torch
    O = oracle_mod
    st = torch.cuda.Stream()
    a, p = ics.sedov(12, seed=15)
    prob = S.Problem(a, S.make_params(S.PREC_FP64, **p, block_levels=4, tree_rebuild_every=4, flags=S.FLAG_ASYNC),
                     stream=st)
    prob.density_h()
    prob.forces()
    prob.sync()
    b_, q_ = _moving_lattice(9, seed=16)
    other = S.Problem(b_, S.make_params(S.PREC_FP64, **q_, flags=S.FLAG_ASYNC), stream=st)
    other.density_h()
    other.forces()
    other.sync()
    dt = prob.diagnostics().dt_next
    wb = S.sph_batch_workspace_bytes([prob.ctx, other.ctx])
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    S.check(S.sph_batch_step([prob.ctx, other.ctx], 1, ws.data_ptr(), wb), "sph_batch_step")
    # the oracle takes the same KDK step (its forces, like the GPU's, from the predicted v)
    P = O.Params(**p, use_grid=True)
    ref = O.State(**a)
    assert O.density(P, ref) == O.OK and O.forces(P, ref) == O.OK
    assert O.step(P, ref, dt) == O.OK
    lv = np.zeros(ref.n, np.int32)
    nm = np.zeros(ref.n, np.int32)
    rc, dtmax, passes, evals = O.block_step(P, ref, lv, nm, 4, 2)
    assert rc == O.OK
    # the GPU context from the same state: its forces were evaluated by the batched step
    dt_g, ev_g = prob.block_step()
    assert ev_g == evals and np.array_equal(prob.levels(), lv)
    assert dt_g == pytest.approx(dtmax, rel=1e-12)
    g = prob.numpy()
    for f in ("vx", "vy", "vz", "u"):
        r = getattr(ref, f)
        assert np.max(np.abs(g[f] - r)) < 1e-11 * np.max(np.abs(r)), f
    prob.close()
    other.close()
