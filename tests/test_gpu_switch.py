"""GPU parity with the Morris & Monaghan (1997) viscosity switch (Sec. 2.1.1):
alpha per particle, its rate d alpha/dt from the force pass, and its
kick-drift-kick integration, against the FP64 oracle run with the switch.

Tolerances (as for the other outputs): mixed precision a within 1e-4
rms|a|, du and d alpha/dt within 1e-4 of their rms; FP64 path 1e-12;
momentum drift < 1e-10."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

pytestmark = pytest.mark.gpu

SW = dict(av_switch=1, alpha_min=0.1, av_decay=0.1)


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _oracle(O, a, p, grid=True, **kw):
    P = O.Params(**p, use_grid=grid, **kw)
    s = O.State(**a)
    assert O.density(P, s) == O.OK
    assert O.forces(P, s) == O.OK
    return P, s


def _gpu(S, a, p, prec, **kw):
    prob = S.Problem(a, S.make_params(prec, **p, **kw))
    prob.density_h()
    prob.forces()
    return prob


def _rms_err(x, y):
    s = np.sqrt(np.mean(y ** 2))
    return np.max(np.abs(x - y)) / (s if s > 0 else 1.0)


def _acc(d):
    return np.stack([d["ax"], d["ay"], d["az"]], 1)


def _moving_lattice(n_side=14, seed=51):
    a, p = ics.lattice(n_side, seed=seed)
    rng = np.random.default_rng(seed)
    for c in ("vx", "vy", "vz"):
        a[c] = rng.normal(0.0, 0.4, len(a["x"]))
    a["alpha"] = rng.uniform(0.1, 1.0, len(a["x"]))
    return a, p


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_switch_rates_match_oracle(S, oracle_mod, prec):
    O = oracle_mod
    a, p = _moving_lattice()
    P, ref = _oracle(O, a, p, **SW)
    fp64 = prec == "fp64"
    g = _gpu(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, **SW).numpy()
    tol = 1e-12 if fp64 else 1e-4
    ra = np.stack([ref.ax, ref.ay, ref.az], 1)
    arms = np.sqrt(np.mean(np.sum(ra ** 2, 1)))
    assert np.max(np.linalg.norm(_acc(g) - ra, axis=1)) < tol * arms
    assert _rms_err(g["du"], ref.du) < tol
    assert _rms_err(g["dalpha"], ref.dalpha) < tol
    assert np.max(np.abs(g["vsig"] / ref.vsig - 1.0)) < (1e-12 if fp64 else 1e-5)
    ma = g["m"][:, None] * _acc(g)
    drift = np.abs(ma.sum(0)) / np.abs(ma).sum(0)
    assert np.all(drift < 1e-10), drift


def test_switch_homologous_compression(S, oracle_mod):
    """v = -k r on an isolated cloud: div v = -3k exactly, so the GPU's rate
    is the decay plus 3k (alpha_max - alpha) at every particle."""
    a, p = ics.cloud(6000, seed=7)
    k = 0.7
    for c, x in (("vx", "x"), ("vy", "y"), ("vz", "z")):
        a[c] = -k * a[x]
    a["alpha"] = np.random.default_rng(7).uniform(0.1, 1.0, 6000)
    g = _gpu(S, a, p, S.PREC_FP64, **SW).numpy()
    want = -(a["alpha"] - 0.1) * 0.1 * g["c"] / g["h"] + 3 * k * (1.0 - a["alpha"])
    assert np.max(np.abs(g["dalpha"] - want)) < 1e-10 * np.max(np.abs(want))


def test_switch_sod_steps_match_oracle(S, oracle_mod):
    """Shock tube with the switch: alpha grows at the shock and decays
    elsewhere; 6 KDK steps against the oracle's."""
    O = oracle_mod
    a, p = ics.sod(left=(32, 16, 16), right=(16, 8, 8), width=0.25)
    a["alpha"] = np.full(len(a["x"]), 0.1)
    P, ref = _oracle(O, a, p, **SW)
    prob = _gpu(S, a, p, S.PREC_MIXED, **SW)
    for _ in range(6):
        dt = O.cfl_dt(P, ref)
        assert O.step(P, ref, dt) == O.OK
        prob.step(dt)
    g = prob.numpy()
    assert np.max(ref.alpha) > 0.12  # compression at the shock raised it above alpha_min
    assert np.max(np.abs(g["alpha"] - ref.alpha)) < 1e-5 * np.max(ref.alpha)
    assert np.max(np.abs(g["rho"] / ref.rho - 1.0)) < 1e-5
    rv = np.stack([ref.vx, ref.vy, ref.vz], 1)
    gv = np.stack([g["vx"], g["vy"], g["vz"]], 1)
    assert np.max(np.linalg.norm(gv - rv, axis=1)) < 1e-4 * np.sqrt(np.mean(np.sum(rv ** 2, 1)))


def test_batch_with_and_without_switch_equals_alone(S):
    """Problems with the switch, with Price conductivity and with neither,
    stepped in one batch, give bit-identical states to each alone."""
    import torch
    la, lp = _moving_lattice(12, seed=52)
    cases = [((la, lp), SW), ((dict(la, alpha=None), lp), {}),
             (ics.sod(left=(32, 16, 16), right=(16, 8, 8), width=0.25), dict(ac_signal=1)),
             (_moving_lattice(10, seed=53), dict(SW, ac_signal=1))]
    alone = []
    for (a, p), kw in cases:
        a = {k: v for k, v in a.items() if v is not None}
        prob = _gpu(S, a, p, S.PREC_MIXED, **kw)
        for _ in range(2):
            prob.step(-1.0)
        alone.append(prob.numpy())
    probs = [_gpu(S, {k: v for k, v in a.items() if v is not None}, p, S.PREC_MIXED, **kw) for (a, p), kw in cases]
    ctxs = [pr.ctx for pr in probs]
    wb = S.sph_batch_workspace_bytes(ctxs)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    S.check(S.sph_batch_step(ctxs, 2, ws.data_ptr(), wb), "sph_batch_step")
    for pr, ref in zip(probs, alone):
        g = pr.numpy()
        for f in ("x", "vx", "u", "h", "rho", "ax", "du", "vsig", "alpha", "dalpha"):
            assert np.array_equal(g[f], ref[f]), f


def test_switch_rejected_without_alpha_arrays_and_by_the_server(S):
    """The switch needs state.alpha and state.dalpha (SPH_EINVAL before any
    workspace check); the server, which keeps no per-particle alpha, refuses
    such requests."""
    import torch
    from paper_1709_04488_gb300 import serve
    a, p = _moving_lattice(6, seed=54)
    n = len(a["x"])
    prm = S.make_params(S.PREC_MIXED, **p, **SW)
    t = {f: torch.zeros(n, dtype=torch.float64, device="cuda") for f in S.STATE_FIELDS if f not in ("alpha", "dalpha")}
    st = S.State(**{f: v.data_ptr() for f, v in t.items()})
    rc, _ = S.sph_setup(prm, n, st, 0, 0, 0)
    assert rc == S.EINVAL
    srv = serve.Server(64 << 20, max_slots=4)
    with pytest.raises(S.SPHError) as e:
        srv.submit(a, dict(p, **SW), nsteps=1, arrival=0.0)
    assert e.value.code == S.EINVAL


# ---- the Cullen & Dehnen (2010) switch (av_switch = 2) ----------------------
CD = dict(av_switch=2, av_decay=0.1)


def _cd_inputs(seed=61, n_side=14):
    """A cold jittered lattice with a compressive, sheared velocity field
    plus noise (the compression steepens as the particles coast, so
    d(div v)/dt < 0), alpha per particle, and the previous evaluation's div v
    with both signs (it sets the signs in R)."""
    a, p = ics.lattice(n_side, seed=seed)
    p = dict(p, periodic=False)
    rng = np.random.default_rng(seed)
    x0 = {c: a[c] - 0.5 for c in ("x", "y", "z")}
    a["vx"] = -0.8 * x0["x"] + 0.5 * x0["y"] + rng.normal(0.0, 0.05, len(a["x"]))
    a["vy"] = -0.8 * x0["y"] + rng.normal(0.0, 0.05, len(a["x"]))
    a["vz"] = 0.3 * x0["z"] + rng.normal(0.0, 0.05, len(a["x"]))
    a["u"] = np.full(len(a["x"]), 1e-3)  # a cold gas: alpha_loc is not swamped by the sound speed
    a["alpha"] = rng.uniform(0.02, 0.8, len(a["x"]))
    a["dalpha"] = rng.normal(-0.5, 1.0, len(a["x"]))  # the previous div v
    return a, p


def _cd_oracle_state(O, a):
    s = O.State(**{k: v for k, v in a.items() if k != "dalpha"})
    s.cd_divv[:] = a["dalpha"]
    return s


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cullen_dehnen_evaluation_matches_oracle(S, oracle_mod, prec):
    """One density/h solve and force evaluation: the accelerations and rates
    with alpha_ij = (alpha_i + alpha_j)/2, and the new div v (written to
    state.dalpha), against the oracle's (its cd_divv)."""
    O = oracle_mod
    a, p = _cd_inputs()
    P = O.Params(**p, use_grid=True, **CD)
    ref = _cd_oracle_state(O, a)
    assert O.density(P, ref) == O.OK and O.forces(P, ref) == O.OK
    fp64 = prec == "fp64"
    g = _gpu(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, **CD).numpy()
    tol = 1e-12 if fp64 else 1e-4
    ra = np.stack([ref.ax, ref.ay, ref.az], 1)
    arms = np.sqrt(np.mean(np.sum(ra ** 2, 1)))
    assert np.max(np.linalg.norm(_acc(g) - ra, axis=1)) < tol * arms
    assert _rms_err(g["du"], ref.du) < tol
    assert _rms_err(g["dalpha"], ref.cd_divv) < tol
    # alpha is only read by an evaluation
    assert np.array_equal(g["alpha"], a["alpha"])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cullen_dehnen_steps_match_oracle(S, oracle_mod, prec):
    """Three KDK steps with the oracle's time-steps: alpha from the switch's
    update (A = xi max(-dD/dt, 0), alpha_loc, decay), div v and the state
    against the oracle; the limiter xi and the rise and decay branches are
    all exercised by the mixed compression and shear."""
    O = oracle_mod
    a, p = _cd_inputs(seed=62)
    P = O.Params(**p, use_grid=True, **CD)
    ref = _cd_oracle_state(O, a)
    assert O.density(P, ref) == O.OK and O.forces(P, ref) == O.OK
    fp64 = prec == "fp64"
    prob = _gpu(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, **CD)
    for _ in range(3):
        dt = O.cfl_dt(P, ref)
        assert O.step(P, ref, dt) == O.OK
        prob.step(dt)
    g = prob.numpy()
    tol = 1e-10 if fp64 else 1e-4
    assert np.max(np.abs(g["alpha"] - ref.alpha)) < tol * np.max(ref.alpha)
    assert np.any(ref.alpha > a["alpha"]) and np.any(ref.alpha < a["alpha"])  # both branches taken
    assert _rms_err(g["dalpha"], ref.cd_divv) < tol
    ra = np.stack([ref.ax, ref.ay, ref.az], 1)
    assert np.max(np.linalg.norm(_acc(g) - ra, axis=1)) < tol * np.sqrt(np.mean(np.sum(ra ** 2, 1)))
    assert np.max(np.abs(g["rho"] / ref.rho - 1.0)) < (1e-10 if fp64 else 1e-5)
