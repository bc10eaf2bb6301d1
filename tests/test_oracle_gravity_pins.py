"""Pins of the oracle's self-gravity (Sec. 2.1.2, Eqs. SPHSELFGRAV,
GRAVFORCEKERNEL, GRADHZETA) with the M4 kernel, isolated problems:

- the force kernel phi'(r,h) against its definition 4 pi/r^2 int_0^r W r'^2 dr'
  by quadrature, Newtonian 1/r^2 beyond the support;
- the potential phi consistent with phi' (phi' = dphi/dr), -1/r beyond 2h,
  and dphi/dh against finite differences;
- exact momentum conservation (pairwise antisymmetric terms);
- the accelerations of a cold, static distribution (P = 0, v = 0: gravity
  only) equal -(1/m_i) dE_pot/dr_i, E_pot = (G/2) sum_ij m_i m_j phi_ij with
  h from a fresh density solve: this checks the direct term, the zeta term
  that carries dh/dr, and the self terms together."""
import numpy as np
import pytest
from scipy.integrate import quad

from paper_1709_04488_gb300 import ics

GR = dict(gravity=1, G=1.0, eos="adiabatic", gamma=5.0 / 3.0)


def test_force_kernel_is_the_enclosed_mass(oracle_mod):
    O = oracle_mod
    h = 0.7
    for r in np.linspace(0.02, 2.4, 37):
        enc, _ = quad(lambda rp: 4 * np.pi * rp * rp * O.kernel_W(rp, h), 0.0, r,
                      points=[p for p in (h, 2 * h) if p < r], epsabs=1e-14, epsrel=1e-13)
        assert abs(O.grav_force(r, h) - enc / r ** 2) < 1e-11 * max(1.0, enc / r ** 2), r
    assert O.grav_force(1.5, 0.7) == pytest.approx(1.0 / 1.5 ** 2, rel=1e-15)


def test_potential_and_its_derivatives(oracle_mod):
    O = oracle_mod
    h, e = 0.6, 1e-6
    for r in np.linspace(0.05, 1.5, 30):
        dr = (O.grav_pot(r + e, h) - O.grav_pot(r - e, h)) / (2 * e)
        assert abs(dr - O.grav_force(r, h)) < 1e-7 * max(1.0, abs(dr)), r
        dh = (O.grav_pot(r, h + e) - O.grav_pot(r, h - e)) / (2 * e)
        assert abs(dh - O.grav_dphidh(r, h)) < 1e-7 * max(1.0, abs(dh)), r
    assert O.grav_pot(1.3, 0.6) == pytest.approx(-1.0 / 1.3, rel=1e-15)
    assert O.grav_pot(0.0, 0.6) == pytest.approx(-1.4 / 0.6, rel=1e-15)  # finite at the centre
    for q in (1.0, 2.0):  # continuous where the spline's pieces join
        assert abs(O.grav_pot(q * h * (1 - 1e-12), h) - O.grav_pot(q * h * (1 + 1e-12), h)) < 1e-10


def _cold_clump(n=600, seed=61):
    a, p = ics.cloud(n, seed=seed)
    a["u"][:] = 0.0
    for c in ("vx", "vy", "vz"):
        a[c][:] = 0.0
    return a, dict(p, **GR)


def test_momentum_conserved_with_gravity(oracle_mod):
    O = oracle_mod
    a, p = ics.cloud(800, seed=62)
    rng = np.random.default_rng(62)
    a["m"] = a["m"] * rng.uniform(0.5, 1.5, 800)
    P = O.Params(**dict(p, gravity=1, G=0.7), use_grid=True)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    ma = s.m[:, None] * np.stack([s.ax, s.ay, s.az], 1)
    assert np.all(np.abs(ma.sum(0)) < 1e-13 * np.abs(ma).sum(0))


def test_gravity_is_the_potential_energy_gradient(oracle_mod):
    O = oracle_mod
    a, p = _cold_clump()
    P = O.Params(**p, use_grid=True)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    assert np.all(s.P == 0.0)  # cold: gravity alone moves the particles

    def epot(b):
        t = O.State(**b)
        assert O.density(P, t) == O.OK
        return O.gravity_energy(P, t)

    eps = 1e-6
    scale = np.sqrt(np.mean(s.m ** 2 * (s.ax ** 2 + s.ay ** 2 + s.az ** 2)))
    for i in (0, 17, 300):
        for c, acc in (("x", s.ax), ("y", s.ay), ("z", s.az)):
            e2 = []
            for sign in (+1, -1):
                b = {k: v.copy() for k, v in a.items()}
                b["h"] = s.h.copy()
                b[c][i] += sign * eps
                e2.append(epot(b))
            grad = (e2[0] - e2[1]) / (2 * eps)
            assert abs(s.m[i] * acc[i] + grad) < 1e-6 * scale, (i, c, s.m[i] * acc[i], -grad)


def test_gravity_needs_an_isolated_m4_problem(oracle_mod):
    O = oracle_mod
    a, p = ics.lattice(6, seed=2)
    s = O.State(**a)
    assert O.density(O.Params(**dict(p, gravity=1)), s) == O.EINVAL  # periodic: no Ewald sums here
    b, q = ics.cloud(200, seed=3)
    t = O.State(**b)
    assert O.density(O.Params(**dict(q, gravity=1, kernel=1)), t) == O.EINVAL
    assert O.density(O.Params(**dict(q, gravity=1, G=0.0)), t) == O.EINVAL


def test_acceleration_condition_sets_the_step_of_a_cold_clump(oracle_mod):
    """Eq. SPH_DTACCEL: with no pressure (u = 0, so c = 0 and the CFL step is
    unbounded) the step is C_GRAV min sqrt(h/|a|): every acceleration of a
    cold static clump is proportional to G, so 4G halves the step, and
    C_CFL plays no part; hot gas under weak gravity keeps the CFL step."""
    O = oracle_mod
    a, p = _cold_clump(500, seed=63)
    dts = {}
    for G, ccfl in ((1.0, 0.2), (4.0, 0.2), (1.0, 0.05)):
        P = O.Params(**dict(p, G=G), use_grid=True, c_cfl=ccfl)
        s = O.State(**a)
        assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
        dts[(G, ccfl)] = O.cfl_dt(P, s)
    assert np.isfinite(dts[(1.0, 0.2)])
    assert dts[(4.0, 0.2)] == pytest.approx(dts[(1.0, 0.2)] / 2, rel=1e-12)
    assert dts[(1.0, 0.05)] == dts[(1.0, 0.2)]
    b, q = ics.cloud(500, seed=64)
    P0 = O.Params(**q, use_grid=True)
    P1 = O.Params(**dict(q, gravity=1, G=1e-6), use_grid=True)
    s0, s1 = O.State(**b), O.State(**b)
    for P, s in ((P0, s0), (P1, s1)):
        assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    assert O.cfl_dt(P1, s1) == pytest.approx(O.cfl_dt(P0, s0), rel=1e-9)
    assert O.density(O.Params(**dict(q, gravity=1, c_grav=0.0)), O.State(**b)) == O.EINVAL
