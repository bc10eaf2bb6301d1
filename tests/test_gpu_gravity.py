"""GPU parity with self-gravity (Sec. 2.1.2, Eq. SPHSELFGRAV): the zeta term
over the neighbours and the direct-sum softened attraction, against the FP64
oracle with the same summation (isolated problems, M4 kernel).

Tolerances as for the hydro accelerations: mixed a within 1e-4 rms|a|, FP64
1e-12; momentum drift < 1e-10."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

pytestmark = pytest.mark.gpu

GR = dict(gravity=1, G=1.0)


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _oracle(O, a, p, **kw):
    P = O.Params(**p, use_grid=True, **kw)
    s = O.State(**a)
    assert O.density(P, s) == O.OK
    assert O.forces(P, s) == O.OK
    return P, s


def _gpu(S, a, p, prec, **kw):
    prob = S.Problem(a, S.make_params(prec, **p, **kw))
    prob.density_h()
    prob.forces()
    return prob


def _acc(d):
    return np.stack([d["ax"], d["ay"], d["az"]], 1)


def _cloud(n=3000, seed=71, vel=0.3):
    a, p = ics.cloud(n, seed=seed)
    rng = np.random.default_rng(seed)
    for c in ("vx", "vy", "vz"):
        a[c] = a[c] * vel
    a["m"] = a["m"] * rng.uniform(0.7, 1.3, n)
    return a, p


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_gravity_matches_oracle(S, oracle_mod, prec):
    O = oracle_mod
    a, p = _cloud()
    gr = dict(GR, G=10.0)  # gravity comparable with the pressure forces
    _, ref = _oracle(O, a, p, **gr)
    fp64 = prec == "fp64"
    g = _gpu(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, **gr).numpy()
    ra = _acc({"ax": ref.ax, "ay": ref.ay, "az": ref.az})
    arms = np.sqrt(np.mean(np.sum(ra ** 2, 1)))
    tol = 1e-12 if fp64 else 1e-4
    assert np.max(np.linalg.norm(_acc(g) - ra, axis=1)) < tol * arms
    ma = g["m"][:, None] * _acc(g)
    drift = np.abs(ma.sum(0)) / np.abs(ma).sum(0)
    assert np.all(drift < 1e-10), drift
    # gravity matters here: without it the accelerations differ grossly
    _, hyd = _oracle(O, a, p)
    ha = _acc({"ax": hyd.ax, "ay": hyd.ay, "az": hyd.az})
    assert np.sqrt(np.mean(np.sum((ra - ha) ** 2, 1))) > 0.1 * arms


def test_cold_clump_gravity_only(S, oracle_mod):
    """u = 0, v = 0: no pressure, no viscosity; the accelerations are the
    zeta term plus the direct sum alone."""
    O = oracle_mod
    a, p = ics.cloud(2000, seed=72)
    a["u"][:] = 0.0
    for c in ("vx", "vy", "vz"):
        a[c][:] = 0.0
    p = dict(p, eos="adiabatic", gamma=5.0 / 3.0)
    _, ref = _oracle(O, a, p, **GR)
    g = _gpu(S, a, p, S.PREC_MIXED, **GR).numpy()
    ra = _acc({"ax": ref.ax, "ay": ref.ay, "az": ref.az})
    assert np.max(np.linalg.norm(_acc(g) - ra, axis=1)) < 1e-4 * np.sqrt(np.mean(np.sum(ra ** 2, 1)))


def test_gravity_steps_match_oracle(S, oracle_mod):
    O = oracle_mod
    a, p = _cloud(2500, seed=73)
    P, ref = _oracle(O, a, p, **GR)
    prob = _gpu(S, a, p, S.PREC_MIXED, **GR)
    T = 0.0
    for _ in range(5):
        dt = O.cfl_dt(P, ref)
        assert O.step(P, ref, dt) == O.OK
        prob.step(dt)
        T += dt
    g = prob.numpy()
    rv = np.stack([ref.vx, ref.vy, ref.vz], 1)
    gv = np.stack([g["vx"], g["vy"], g["vz"]], 1)
    vtol = 1e-4 * np.sqrt(np.mean(np.sum(rv ** 2, 1)))
    assert np.max(np.linalg.norm(gv - rv, axis=1)) < vtol
    assert np.max(np.abs(g["x"] - ref.x)) < vtol * T
    assert np.max(np.abs(g["rho"] / ref.rho - 1.0)) < 1e-5


def test_batch_with_gravity_equals_alone(S):
    import torch
    cases = [(_cloud(1500, seed=74), GR), (_cloud(1200, seed=75), {}), (_cloud(900, seed=76), dict(GR, G=0.5))]
    alone = []
    for (a, p), kw in cases:
        prob = _gpu(S, a, p, S.PREC_MIXED, **kw)
        for _ in range(2):
            prob.step(-1.0)
        alone.append(prob.numpy())
    probs = [_gpu(S, a, p, S.PREC_MIXED, **kw) for (a, p), kw in cases]
    ctxs = [pr.ctx for pr in probs]
    wb = S.sph_batch_workspace_bytes(ctxs)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    S.check(S.sph_batch_step(ctxs, 2, ws.data_ptr(), wb), "sph_batch_step")
    for pr, ref in zip(probs, alone):
        g = pr.numpy()
        for f in ("x", "vx", "u", "h", "rho", "ax", "du", "vsig"):
            assert np.array_equal(g[f], ref[f]), f


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_split_partner_ranges_match_oracle(S, oracle_mod, prec):
    """N = 20000: too few particle blocks to fill the GPU, so the direct sum
    splits the partners into ranges whose FP64 partials a second kernel
    adds; same tolerances as the unsplit sum."""
    O = oracle_mod
    a, p = _cloud(20000, seed=77)
    _, ref = _oracle(O, a, p, **GR)
    fp64 = prec == "fp64"
    g = _gpu(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, **GR).numpy()
    ra = _acc({"ax": ref.ax, "ay": ref.ay, "az": ref.az})
    arms = np.sqrt(np.mean(np.sum(ra ** 2, 1)))
    assert np.max(np.linalg.norm(_acc(g) - ra, axis=1)) < (1e-12 if fp64 else 1e-4) * arms
    ma = g["m"][:, None] * _acc(g)
    assert np.all(np.abs(ma.sum(0)) / np.abs(ma).sum(0) < 1e-10)


def test_batch_with_split_gravity_equals_alone(S):
    """A split problem (N = 9000), an unsplit one and one without gravity in
    one batch: bit-identical to each stepped alone."""
    import torch
    cases = [(_cloud(9000, seed=78), GR), (_cloud(1500, seed=79), GR), (_cloud(2000, seed=80), {})]
    alone = []
    for (a, p), kw in cases:
        prob = _gpu(S, a, p, S.PREC_MIXED, **kw)
        prob.step(-1.0)
        alone.append(prob.numpy())
    probs = [_gpu(S, a, p, S.PREC_MIXED, **kw) for (a, p), kw in cases]
    ctxs = [pr.ctx for pr in probs]
    wb = S.sph_batch_workspace_bytes(ctxs)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    S.check(S.sph_batch_step(ctxs, 1, ws.data_ptr(), wb), "sph_batch_step")
    for pr, ref in zip(probs, alone):
        g = pr.numpy()
        for f in ("x", "vx", "u", "h", "rho", "ax", "du", "vsig"):
            assert np.array_equal(g[f], ref[f]), f


def test_gravity_rejected_for_periodic_or_m6(S):
    for kw in (dict(periodic=True), dict(periodic=False, kernel=1)):
        p = S.make_params(S.PREC_MIXED, gravity=1, G=1.0, **kw)
        assert S.sph_workspace_bytes(100, p) == 0
