"""Pins for the Sedov-Taylor blast wave (Sec. 6.3): the similarity solution
derived in oracle/sedov.py, and an oracle SPH blast checked against it.

The similarity solution is pinned by laws it must obey that its integration
does not impose:
  - the energy-flux first integral: the energy inside any sphere moving with
    the similarity variable is constant (its total scales as Rdot^2 R^nu,
    which is constant in time), so the flux through that sphere vanishes,
    (psi phi^2/2 + pi/(gamma-1)) (lam - phi) = pi phi at every lam;
  - mass: the gas inside the front is exactly the gas swept up,
    int_0^1 psi lam^(nu-1) dlam = 1/nu;
  - the strong-shock density jump (gamma+1)/(gamma-1), i.e. 4 for gamma = 5/3;
  - the front constant xi0 ~ 1.15 for gamma = 5/3 in 3D (quoted for the
    paper's blast test).
Then the oracle's SPH blast (the generator of the Sedov configuration on a
20^3 lattice, E = 1 on the 64 central particles) must put its density peak at
the similarity front, at two times (so the R ~ t^(2/5) law is checked too),
within half a smoothing length (the stated bound is 2h), and its peak density
must stay below the jump 4 (the paper's 2D peak is just under 3).
"""
import math

import numpy as np
import pytest

from oracle import sedov
from paper_1709_04488_gb300 import ics

CASES = [(5.0 / 3.0, 3), (1.4, 3), (5.0 / 3.0, 2), (1.4, 1)]


@pytest.mark.parametrize("gamma,nu", CASES)
def test_energy_flux_first_integral(gamma, nu):
    lam, psi, phi, pi = sedov.profile(gamma, nu)
    sel = lam >= 0.02  # (below, psi < 1e-7 and phi carries the integration's noise)
    lhs = (0.5 * psi * phi ** 2 + pi / (gamma - 1.0)) * (lam - phi)
    rhs = pi * phi
    assert np.max(np.abs(lhs - rhs)[sel]) < 1e-8 * np.max(rhs)


@pytest.mark.parametrize("gamma,nu", CASES)
def test_swept_up_mass(gamma, nu):
    mass, _ = sedov.integrals(gamma, nu)
    assert abs(mass * nu - 1.0) < 1e-9


@pytest.mark.parametrize("gamma,nu", CASES)
def test_front_values_and_profile_shape(gamma, nu):
    lam, psi, phi, pi = sedov.profile(gamma, nu)
    assert lam[0] == 1.0
    assert abs(psi[0] - (gamma + 1.0) / (gamma - 1.0)) < 1e-14
    assert abs(phi[0] - 2.0 / (gamma + 1.0)) < 1e-14 and abs(pi[0] - 2.0 / (gamma + 1.0)) < 1e-14
    # density falls monotonically to zero at the centre; pressure to a
    # positive floor; the gas moves outwards behind the front
    assert np.all(np.diff(psi) < 0) and psi[-1] < 1e-6
    assert np.all(phi > 0) and pi[-1] > 0.1 * pi[0]


def test_xi0_of_the_blast_test():
    x = sedov.xi0(5.0 / 3.0, 3)
    assert abs(x - 1.15) < 0.005
    assert sedov.density(0.999 * sedov.shock_radius(1.0), 1.0) > 3.9  # jump of 4 just behind the front
    assert sedov.density(1.001 * sedov.shock_radius(1.0), 1.0) == 1.0


def _front(s):
    # radius of the density peak: the median radius of the densest 1 % of
    # particles, and the smoothing length there
    r = np.sqrt((s.x - 0.5) ** 2 + (s.y - 0.5) ** 2 + (s.z - 0.5) ** 2)
    top = np.argsort(s.rho)[-max(20, s.n // 100):]
    return float(np.median(r[top])), float(np.median(s.h[top]))


def test_oracle_blast_follows_the_similarity_front(oracle_mod):
    O = oracle_mod
    a, p = ics.sedov(20)
    P = O.Params(**p, use_grid=True)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    t = 0.0
    checks = []
    for R_target in (0.22, 0.32):
        while sedov.shock_radius(t) < R_target:
            dt = O.cfl_dt(P, s)
            assert O.step(P, s, dt) == O.OK
            t += dt
        Rs, h = _front(s)
        R_an = sedov.shock_radius(t)
        checks.append((t, Rs, h, R_an))
        assert abs(Rs - R_an) < 2.0 * h       # the stated bound
        assert abs(Rs - R_an) < 0.5 * h       # and the tighter one this set-up meets
        assert s.rho.max() < 4.0               # below the strong-shock jump
    # energy: the deposit plus the background is conserved by the KDK steps
    E0 = float(np.sum(a["m"] * a["u"]))
    E1 = float(np.sum(s.m * (s.u + 0.5 * (s.vx ** 2 + s.vy ** 2 + s.vz ** 2))))
    assert abs(E1 / E0 - 1.0) < 2e-3
    (t1, R1, _, _), (t2, R2, _, _) = checks
    assert abs(math.log(R2 / R1) / math.log(t2 / t1) - 0.4) < 0.05
