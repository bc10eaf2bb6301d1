"""Pin of the artificial viscosity's strength (Sec. 2.1.1, Eqs. MON97ARTVISC
and MON97ENERGYDISS) by its continuum limit, independent of the oracle's
pair loop.

Take a cold gas (u = 0, so P = 0 and c = 0) on an isolated perfect cubic
lattice in homologous compression, v = -k (r - r_c).  Every pair then has
v_ij . r_hat_ij = -k r_ij < 0, so mu_ij = -k r_ij and v_sig = beta_AV k r_ij,
and the viscous heating of an interior particle is

    du_i/dt = -(1/2) alpha sum_j (m_j / rho_bar) v_sig mu_ij^2 r_hat . grad W
            = -(1/2) alpha beta k^3 sum_j (m_j / rho) r^3 W'(r).

The sum over a lattice tends, as the kernel covers more particles, to the
integral int r^3 W'(r) d^3r = -5 int r^2 W d^3r = -5 h^2 <q^2> (integration
by parts; <q^2> is the kernel's second moment, a quadrature of the pinned
kernel), so du/dt -> (5/2) alpha beta k^3 h^2 <q^2>.  The oracle's heating
approaches this limit as eta grows (more neighbours), within 1 % at eta = 2.
A factor 1/2 on alpha, mu formed from r instead of r_hat (the garbled form
printed beside Eq. MON97ARTVISC), a missing beta or a wrong power of v_sig
each moves the result far outside that.  The interior acceleration vanishes
by the lattice's inversion symmetry.  The acceleration's magnitude is tied to
the heating by the energy balance pinned in test_oracle_pins.py."""
import math

import numpy as np
import pytest
from scipy import integrate


def _compressed_lattice(O, n, eta, k=0.7):
    d = 1.0 / n
    g = (np.arange(n) + 0.5) * d
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    N = len(x)
    a = dict(x=x, y=y, z=z, vx=-k * (x - 0.5), vy=-k * (y - 0.5), vz=-k * (z - 0.5), u=np.zeros(N),
             m=np.full(N, d ** 3), h=np.full(N, eta * d))
    P = O.Params(periodic=False, box_len=(0.0, 0.0, 0.0), eos="adiabatic", gamma=5.0 / 3.0, alpha_ac=0.0,
                 eta=eta, use_grid=True)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    return P, s, x, y, z, k


def _second_moment(O):
    return integrate.quad(lambda q: q * q * O.kernel_W(q, 1.0) * 4.0 * math.pi * q * q, 0.0, 2.0,
                          points=[1.0], epsabs=1e-14)[0]


@pytest.mark.parametrize("eta,n,tol_lo,tol_hi", [(1.2, 20, 0.93, 0.97), (1.6, 24, 0.975, 1.0), (2.0, 28, 0.99, 1.01)])
def test_viscous_heating_tends_to_its_continuum_limit(oracle_mod, eta, n, tol_lo, tol_hi):
    O = oracle_mod
    P, s, x, y, z, k = _compressed_lattice(O, n, eta)
    dface = np.minimum.reduce([x, y, z, 1 - x, 1 - y, 1 - z])
    hc = s.h[np.argmin((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)]
    inner = dface > 4.2 * hc  # every force neighbour has the lattice's h
    assert inner.sum() >= 500
    h = s.h[inner]
    assert np.ptp(h) < 1e-14 * h[0]
    limit = 2.5 * P.alpha_av * P.beta_av * k ** 3 * h[0] ** 2 * _second_moment(O)
    ratio = s.du[inner] / limit
    assert np.ptp(ratio) < 1e-10
    assert tol_lo < ratio[0] < tol_hi
    # no net viscous acceleration on a symmetric neighbourhood
    acc = np.sqrt(s.ax[inner] ** 2 + s.ay[inner] ** 2 + s.az[inner] ** 2)
    assert acc.max() < 1e-12 * limit / (k * h[0])


def test_viscous_heating_scales_as_alpha_beta_and_k_cubed(oracle_mod):
    """Doubling alpha (beta = 2 alpha) quadruples the heating of a cold gas,
    and doubling k multiplies it by 8 (v_sig mu^2 ~ k^3): the AV term is
    linear in alpha and in v_sig."""
    O = oracle_mod
    P, s, x, y, z, k = _compressed_lattice(O, 16, 1.2)
    i = np.argmin((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    base = s.du[i]
    s2 = O.State(**{f: getattr(s, f) for f in ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h")})
    P2 = O.Params(**{**P.__dict__, "alpha_av": 2.0, "beta_av": 4.0})
    assert O.density(P2, s2) == O.OK and O.forces(P2, s2) == O.OK
    assert abs(s2.du[i] / base - 4.0) < 1e-12
    s3 = O.State(**{f: getattr(s, f) for f in ("x", "y", "z", "u", "m", "h")},
                 vx=2 * s.vx, vy=2 * s.vy, vz=2 * s.vz)
    assert O.density(P, s3) == O.OK and O.forces(P, s3) == O.OK
    assert abs(s3.du[i] / base - 8.0) < 1e-12
