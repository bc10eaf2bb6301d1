"""Pins of the oracle's Cullen & Dehnen (2010) viscosity switch (Sec. 2.1.1
names it; the equations are the published ones, stated in oracle/sph_oracle.c
with its two readings: R from the previous evaluation's signs of div v, and
d(div v)/dt by finite differences between force evaluations).

On the interior of a perfect isolated lattice the SPH velocity gradient of a
linear field v = M r is exact: the neighbour tensor sum_j m_j r W' r_hat r_hat
is isotropic by cubic symmetry and its trace is -3 rho Omega by the grad-h
definition of Omega (which alone makes div v of M = -k I exact at every
particle, edges included).  So for M = -k I + (shear s along x of y):
- div v = -3k;
- tr(S S^T) = s^2 / 2, the shear of the traceless symmetric part;
- R = -1 once every particle's previous div v is negative (R is the
  signed density over the density), so xi = q^2 / (q^2 + s^2/2) with
  q = 2 (1 - R)^4 div v = -96 k;
- before any previous evaluation (div v = 0 taken as positive) R = +1, xi = 0.
A pure shear gives xi = 0.  The alpha update follows its closed forms, and
pair forces stay antisymmetric (exact momentum and energy balance)."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

K, SH = 0.6, 0.9


def _lattice_flow(O, k, s, n_side=14, alpha=0.5):
    a, p = ics.lattice(n_side, jitter=0.0, seed=1)
    p = dict(p, periodic=False)
    x0 = {c: a[c] - 0.5 for c in ("x", "y", "z")}
    a["vx"] = -k * x0["x"] + s * x0["y"]
    a["vy"] = -k * x0["y"]
    a["vz"] = -k * x0["z"]
    a["alpha"] = np.full(len(a["x"]), alpha)
    P = O.Params(**p, use_grid=True, av_switch=2, av_decay=0.05)
    st = O.State(**a)
    assert O.density(P, st) == O.OK
    return P, st, a


def _interior(a, h):
    m = np.ones(len(a["x"]), bool)
    for c in ("x", "y", "z"):
        m &= (a[c] > 2.5 * h.max()) & (a[c] < 1.0 - 2.5 * h.max())
    return m


def test_divergence_shear_and_limiter_on_a_lattice(oracle_mod):
    O = oracle_mod
    P, st, a = _lattice_flow(O, K, SH)
    assert O.forces(P, st) == O.OK
    inner = _interior(a, st.h)
    assert inner.sum() > 50
    assert np.max(np.abs(st.cd_divv[inner] + 3 * K)) < 1e-11
    assert np.max(st.cd_xi) < 1e-40  # no previous div v: R = +1 (to rounding)
    assert O.forces(P, st) == O.OK  # the previous div v now negative everywhere
    q2 = (96.0 * K) ** 2
    want = q2 / (q2 + SH ** 2 / 2)
    assert np.max(np.abs(st.cd_xi[inner] - want)) < 1e-10
    # pure compression: div v = -3k at every particle, edges included (only
    # the trace identity of Omega is used)
    P1, st1, _ = _lattice_flow(O, K, 0.0)
    assert O.forces(P1, st1) == O.OK
    assert np.max(np.abs(st1.cd_divv + 3 * K)) < 1e-11
    # pure shear: no divergence, no switch
    P2, st2, a2 = _lattice_flow(O, 0.0, SH)
    assert O.forces(P2, st2) == O.OK and O.forces(P2, st2) == O.OK
    in2 = _interior(a2, st2.h)
    assert np.max(np.abs(st2.cd_divv[in2])) < 1e-11
    assert np.max(st2.cd_xi[in2]) < 1e-20


def test_alpha_update_closed_forms(oracle_mod):
    O = oracle_mod
    P, st, a = _lattice_flow(O, K, SH)
    assert O.forces(P, st) == O.OK and O.forces(P, st) == O.OK
    dt = 1e-3
    alpha0 = st.alpha.copy()
    # steady divergence: no source, alpha decays on tau = h / (2 l v_sig)
    O.cd_update(P, st, st.cd_divv.copy(), dt)
    assert np.allclose(st.alpha, alpha0 * np.exp(-dt * 2 * 0.05 * st.vsig / st.h), rtol=1e-14, atol=0)
    # divergence falling (compression growing): alpha rises to alpha_loc < alpha_max
    st.alpha[:] = 0.01
    d_old = st.cd_divv + 50.0 * dt  # d(div v)/dt = -50
    O.cd_update(P, st, d_old, dt)
    A = st.cd_xi * 50.0
    aloc = P.alpha_av * st.h ** 2 * A / (st.vsig ** 2 + st.h ** 2 * A)
    up = aloc > 0.01
    assert up.sum() > 0
    assert np.allclose(st.alpha[up], aloc[up], rtol=1e-13)
    assert np.all(st.alpha <= P.alpha_av)


def test_conservation_with_the_cd_switch(oracle_mod):
    O = oracle_mod
    a, p = ics.random_cloud(1500, seed=45, mass_spread=0.4, vel=1.0, u_spread=0.6)
    a["alpha"] = np.random.default_rng(45).uniform(0.0, 1.0, 1500)
    P = O.Params(**p, use_grid=True, av_switch=2)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    ma = s.m[:, None] * np.stack([s.ax, s.ay, s.az], 1)
    assert np.all(np.abs(ma.sum(0)) < 1e-13 * np.abs(ma).sum(0))
    terms = s.m * (s.vx * s.ax + s.vy * s.ay + s.vz * s.az) + s.m * s.du
    assert abs(terms.sum()) < 1e-12 * np.abs(terms).sum()


def test_cd_steps_keep_alpha_bounded_and_block_steps_refuse_it(oracle_mod):
    O = oracle_mod
    a, p = ics.sod(left=(32, 16, 16), right=(16, 8, 8), width=0.25)
    a["alpha"] = np.zeros(len(a["x"]))
    P = O.Params(**p, use_grid=True, av_switch=2)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    for _ in range(4):
        assert O.step(P, s, O.cfl_dt(P, s)) == O.OK
    assert np.all(s.alpha >= 0) and np.all(s.alpha <= P.alpha_av)
    assert np.max(s.alpha) > 0.05  # the shock switched it on
    lv = np.zeros(s.n, np.int32)
    assert O.block_step(P, s, lv, lv.copy(), 2)[0] == O.EINVAL
