"""Pins of the oracle's Price (2008) conductivity option (Sec. 2.1.1: the
conductivity signal speed sqrt(|P_i - P_j| / rho_bar_ij) in place of
Wadsley's |v_ij . r_hat_ij|).  With the particles at rest only conduction
changes u, so the pins isolate it: energy conservation, no flux without a
pressure difference, heat flowing from hot to cold, and the exact scaling of
the rate with u (the signal speed grows as sqrt(u), the difference as u)."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics


def _rates(O, a, p, **kw):
    P = O.Params(**p, use_grid=True, **kw)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    return s


def _hot_slab(n_side=12, seed=3, jitter=0.1):
    a, p = ics.lattice(n_side, jitter=jitter, seed=seed)
    a["u"] = np.where(a["x"] < 0.5, 2.0, 1.0)
    return a, p


def test_at_rest_wadsley_conducts_nothing_price_conserves(oracle_mod):
    O = oracle_mod
    a, p = _hot_slab()
    s0 = _rates(O, a, p, ac_signal=0)
    assert np.all(s0.du == 0.0)  # no velocity: no compression, no Wadsley flux
    s1 = _rates(O, a, p, ac_signal=1)
    flux = s1.m * s1.du
    assert np.abs(flux).sum() > 0
    assert abs(flux.sum()) < 1e-13 * np.abs(flux).sum()


def test_price_no_flux_without_pressure_difference(oracle_mod):
    """Perfect lattice, uniform u: equal pressures, so no conduction even
    though the signal speed form would allow it."""
    O = oracle_mod
    a, p = ics.lattice(10, jitter=0.0, seed=1)
    s = _rates(O, a, p, ac_signal=1)
    assert np.max(np.abs(s.du)) < 1e-12 * np.max(np.abs(s.u))


def test_price_no_flux_at_pressure_equilibrium(oracle_mod):
    """u_i = 1/rho_i on a jittered lattice: u varies by the density
    scatter but P = (gamma-1) rho u is uniform, so Price's signal speed (and
    the flux) vanishes -- unlike a signal speed built from the pressures'
    sum or the velocities."""
    O = oracle_mod
    a, p = ics.lattice(12, jitter=0.15, seed=5)
    P = O.Params(**p, use_grid=True, ac_signal=1)
    s = O.State(**a)
    assert O.density(P, s) == O.OK
    b = dict(a, u=1.0 / s.rho, h=s.h.copy())
    s = O.State(**b)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    assert np.std(b["u"]) > 1e-3 * np.mean(b["u"])
    hot = _rates(O, *_hot_slab(), ac_signal=1)
    assert np.max(np.abs(s.du)) < 1e-6 * np.max(np.abs(hot.du))


def test_price_heat_flows_from_hot_to_cold(oracle_mod):
    O = oracle_mod
    a, p = _hot_slab(jitter=0.0)
    s = _rates(O, a, p, ac_signal=1)
    hot = a["x"] < 0.5
    assert np.sum(s.m[hot] * s.du[hot]) < 0 < np.sum(s.m[~hot] * s.du[~hot])
    # the flux is confined to the two interfaces (x = 0.5 and x = 0 = 1)
    far = np.minimum(np.abs(a["x"] - 0.5), np.minimum(a["x"], 1.0 - a["x"])) > 2.5 * np.max(s.h)
    assert np.all(s.du[far] == 0.0)


def test_price_rate_scales_as_u_to_three_halves(oracle_mod):
    """Scaling every u by lam leaves rho (positions, masses) unchanged and
    multiplies P_i - P_j and u_i - u_j by lam: the rate goes as lam^1.5."""
    O = oracle_mod
    a, p = _hot_slab()
    s1 = _rates(O, a, p, ac_signal=1)
    b = dict(a, u=4.0 * a["u"])
    s4 = _rates(O, b, p, ac_signal=1)
    nz = np.abs(s1.du) > 1e-8 * np.max(np.abs(s1.du))
    assert nz.sum() > 50
    assert np.max(np.abs(s4.du[nz] / s1.du[nz] - 8.0)) < 1e-10


@pytest.mark.parametrize("sig", [0, 1])
def test_energy_rate_vanishes_with_either_signal_speed(oracle_mod, sig):
    O = oracle_mod
    a, p = ics.random_cloud(1500, seed=37, mass_spread=0.4, vel=1.0, u_spread=0.7)
    s = _rates(O, a, p, ac_signal=sig)
    terms = s.m * (s.vx * s.ax + s.vy * s.ay + s.vz * s.az) + s.m * s.du
    assert abs(terms.sum()) < 1e-12 * np.abs(terms).sum()


def test_rejects_unknown_signal_speed(oracle_mod):
    O = oracle_mod
    a, p = ics.lattice(6, seed=2)
    s = O.State(**a)
    assert O.density(O.Params(**p, ac_signal=2), s) == O.EINVAL
