"""Pins of the oracle's hierarchical block time-steps (Sec. 2.1.4) with the
Saitoh & Makino limiter (Sec. 2.1.4, predictive and reactive parts):

- one level (L = 0) is the global kick-drift-kick step with the CFL step,
  bit for bit;
- a Sedov blast (the paper's block time-step test) on 6 levels needs far
  fewer particle force evaluations than global steps of the finest level and
  tracks that global integration closely;
- the limiter only shortens steps: it adds force evaluations and lifts the
  levels of particles next to fast ones."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics


def _ready(O, a, p, **kw):
    P = O.Params(**p, use_grid=True, **kw)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    return P, s


def _block(O, P, s, L, dl=2):
    lv = np.zeros(s.n, np.int32)
    nm = np.zeros(s.n, np.int32)
    rc, dtmax, passes, evals = O.block_step(P, s, lv, nm, L, dl)
    assert rc == O.OK
    return lv, dtmax, passes, evals


@pytest.mark.parametrize("kw", [{}, dict(av_switch=1), dict(gravity=1, G=1.0)])
def test_one_level_is_the_global_step(oracle_mod, kw):
    O = oracle_mod
    if kw.get("gravity"):
        a, p = ics.cloud(1500, seed=9)
    else:
        a, p = ics.sod(left=(32, 16, 16), right=(16, 8, 8), width=0.25)
    if kw.get("av_switch"):
        a["alpha"] = np.full(len(a["x"]), 0.3)
    P, s = _ready(O, a, p, **kw)
    g = s.copy()
    dt = O.cfl_dt(P, g)
    assert O.step(P, g, dt) == O.OK
    lv, dtmax, passes, evals = _block(O, P, s, 0)
    assert dtmax == dt and passes == 1 and evals == s.n and np.all(lv == 0)
    for f in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "ax", "du", "vsig") + (("alpha",) if "av_switch" in kw else ()):
        assert np.array_equal(getattr(s, f), getattr(g, f)), f


def _sedov(O):
    a, p = ics.sedov(16)
    return _ready(O, a, p)


def test_sedov_saves_evaluations_and_tracks_global_steps(oracle_mod):
    O = oracle_mod
    P, s = _sedov(O)
    g = s.copy()
    L = 6
    lv, dtmax, passes, evals = _block(O, P, s, L)
    assert evals < s.n * 2 ** L / 4  # the point of the scheme
    assert lv.max() >= 4 and lv.min() == 0  # the blast and the cold gas on different levels
    for _ in range(2 ** L):  # global steps of the finest level over the same time
        assert O.step(P, g, dtmax / 2 ** L) == O.OK
    vmax = np.max(np.abs(np.stack([g.vx, g.vy, g.vz])))
    for f in ("vx", "vy", "vz"):
        assert np.max(np.abs(getattr(s, f) - getattr(g, f))) < 3e-3 * vmax, f
    assert np.max(np.abs(s.u - g.u)) < 1e-3 * np.max(g.u)
    assert np.max(np.abs(s.rho / g.rho - 1.0)) < 5e-3


def test_limiter_shortens_steps(oracle_mod):
    O = oracle_mod
    P, s = _sedov(O)
    t = s.copy()
    lv2, _, _, ev2 = _block(O, P, s, 6, dl=2)
    lv30, _, _, ev30 = _block(O, P, t, 6, dl=30)  # gap of 30 levels: no limiting
    assert ev2 > ev30
    assert np.sum(lv2 == 0) < np.sum(lv30 == 0)
    assert np.all(lv2 >= lv30)


def test_block_step_rejects_bad_levels(oracle_mod):
    O = oracle_mod
    a, p = ics.lattice(6, seed=2)
    P, s = _ready(O, a, p)
    lv = np.zeros(s.n, np.int32)
    nm = np.zeros(s.n, np.int32)
    assert O.block_step(P, s, lv, nm, -1)[0] == O.EINVAL
    assert O.block_step(P, s, lv, nm, 3, 0)[0] == O.EINVAL


def test_reactively_cut_steps_keep_second_order_accuracy(oracle_mod):
    """A step that the reactive limiter cuts short has its opening half kick
    corrected to the shortened step.  Constructed case: a periodic lattice
    with a pressure wave (u = 1 + 0.5 sin 2 pi x, accelerations of order 2
    everywhere), and a spread of particles whose neighbours' levels are given
    as L on entry, so the predictive limiter puts them L - dl levels up; at
    their first force pass they lift their slower neighbours, whose steps
    (up to Delta t_MAX long) end early.  Every particle then still follows
    the global integration with the finest step to second order: within
    0.03 |a|_rms Delta t_MAX.  Without the correction a cut particle keeps
    the extra half kick a (t1 - t1') / 2, at least a Delta t_MAX / 8 for
    the smallest cut (measured: 0.27 |a|_rms Delta t_MAX, 30x the bound's
    left side with the correction, 0.009)."""
    O = oracle_mod
    a, p = ics.lattice(14, seed=3)
    a["u"] = 1.0 + 0.5 * np.sin(2 * np.pi * a["x"])
    P, s = _ready(O, a, p)
    g = s.copy()
    L, dl = 6, 2
    lv = np.zeros(s.n, np.int32)
    nm = np.zeros(s.n, np.int32)
    nm[np.arange(0, s.n, 97)] = L
    rc, dtmax, passes, evals = O.block_step(P, s, lv, nm, L, dl)
    assert rc == O.OK and passes > 2
    for _ in range(2 ** L):
        assert O.step(P, g, dtmax / 2 ** L) == O.OK
    dv = np.sqrt((s.vx - g.vx) ** 2 + (s.vy - g.vy) ** 2 + (s.vz - g.vz) ** 2)
    arms = np.sqrt(np.mean(g.ax ** 2 + g.ay ** 2 + g.az ** 2))
    assert dv.max() < 0.03 * arms * dtmax
    # the heating follows likewise (du/dt ~ P div v)
    assert np.max(np.abs(s.u - g.u)) < 0.03 * np.max(np.abs(g.du)) * dtmax
