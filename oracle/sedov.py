"""Similarity solution of the point blast wave in a uniform gas (Sedov-Taylor)
for an ideal gas (test infrastructure; the analytic pin of the Sedov blast
test, Sec. 6.3).  Only ``tests/`` import it.

Derived here from the Euler equations, not taken from a table.  With the
shock radius R(t) = xi0 (E t^2 / rho0)^(1/5), its speed Rdot = (2/5) R / t
and the similarity variable lam = r / R, write

    u = Rdot phi(lam),   rho = rho0 psi(lam),   p = rho0 Rdot^2 pi(lam).

Substituting into mass, momentum and entropy conservation in nu dimensions
(nu = 3: spherical), and using Rddot = -(3/2) Rdot^2 / R, gives

    (phi - lam) psi' + psi phi' = -(nu - 1) psi phi / lam
    (phi - lam) phi' + pi' / psi = (3/2) phi                 [nu = 3 exponent]
    (phi - lam) (pi'/pi - gamma psi'/psi) = 3

(the last: p rho^-gamma is constant along particle paths; its similarity
form scales as Rdot^2, whose time derivative supplies the 3 = -2 Rddot R /
Rdot^2).  The general form for the blast in nu dimensions has R ~ t^(2/(nu+2)),
which changes the right-hand sides: written out for any nu below.

The strong-shock jump conditions give the values just behind the front,
psi(1) = (gamma+1)/(gamma-1), phi(1) = pi(1) = 2/(gamma+1).  The system is
integrated inwards from lam = 1.  The energy between the centre and the
front, E = rho0 Rdot^2 R^nu S_nu int_0^1 (psi phi^2/2 + pi/(gamma-1))
lam^(nu-1) dlam, fixes xi0 (S_nu: 4 pi, 2 pi, 2 for nu = 3, 2, 1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _exponents(nu):
    # R ~ t^a with a = 2/(nu+2); Rddot R / Rdot^2 = (a - 1)/a
    a = 2.0 / (nu + 2.0)
    return a, (a - 1.0) / a


def _rhs(lam, y, gamma, nu):
    """d(psi, phi, pi, m, e)/dlam: the three conservation laws (a 3x3 linear
    system in the derivatives) and the mass and energy integrands, which are
    integrated alongside (m, e accumulate from the front inwards)."""
    psi, phi, pi = y[0], y[1], y[2]
    a, k = _exponents(nu)
    d = phi - lam
    # (1) mass:      d psi' + psi phi'                 = -(nu-1) psi phi / lam
    # (2) momentum:  d phi' + pi'/psi                  = -k phi
    # (3) entropy:   -gamma d psi'/psi + d pi'/pi      = -2 k
    M = np.array([[d, psi, 0.0],
                  [0.0, d, 1.0 / psi],
                  [-gamma * d / psi, 0.0, d / pi]])
    b = np.array([-(nu - 1.0) * psi * phi / lam, -k * phi, -2.0 * k])
    dpsi, dphi, dpi = np.linalg.solve(M, b)
    w = lam ** (nu - 1)
    return [dpsi, dphi, dpi, -psi * w, -(0.5 * psi * phi * phi + pi / (gamma - 1.0)) * w]


def _solve(gamma, nu, lam_min, npts):
    y0 = [(gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0), 2.0 / (gamma + 1.0), 0.0, 0.0]
    lam = np.geomspace(1.0, lam_min, npts)
    sol = solve_ivp(_rhs, (1.0, lam_min), y0, t_eval=lam, args=(gamma, nu), method="LSODA",
                    rtol=1e-11, atol=1e-14)
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol


def profile(gamma: float = 5.0 / 3.0, nu: int = 3, lam_min: float = 1e-3, npts: int = 2000):
    """(lam, psi, phi, pi) from the front (lam = 1) inwards to lam_min."""
    sol = _solve(gamma, nu, lam_min, npts)
    return sol.t, sol.y[0], sol.y[1], sol.y[2]


def _surface(nu):
    return {1: 2.0, 2: 2.0 * math.pi, 3: 4.0 * math.pi}[nu]


def integrals(gamma: float = 5.0 / 3.0, nu: int = 3):
    """(int_0^1 psi lam^(nu-1) dlam, int_0^1 (psi phi^2/2 + pi/(gamma-1))
    lam^(nu-1) dlam), integrated with the profile; the part below lam = 1e-3
    (where psi ~ lam^(nu/(gamma-1)) and the energy integrand ~ lam^(nu-1))
    is below 1e-9 and left out."""
    sol = _solve(gamma, nu, 1e-3, 2)
    return float(sol.y[3][-1]), float(sol.y[4][-1])


def energy_integral(gamma: float = 5.0 / 3.0, nu: int = 3) -> float:
    """I = S_nu int_0^1 (psi phi^2 / 2 + pi / (gamma - 1)) lam^(nu-1) dlam."""
    return _surface(nu) * integrals(gamma, nu)[1]


def xi0(gamma: float = 5.0 / 3.0, nu: int = 3) -> float:
    """Dimensionless front constant: R = xi0 (E t^2 / rho0)^(1/(nu+2)).
    From E = rho0 Rdot^2 R^nu I with Rdot = a R / t, a = 2/(nu+2):
    E = a^2 rho0 R^(nu+2) t^-2 I, so xi0 = (1 / (a^2 I))^(1/(nu+2))."""
    a, _ = _exponents(nu)
    return (1.0 / (a * a * energy_integral(gamma, nu))) ** (1.0 / (nu + 2.0))


def shock_radius(t: float, E: float = 1.0, rho0: float = 1.0, gamma: float = 5.0 / 3.0, nu: int = 3) -> float:
    """R(t) = xi0 (E t^2 / rho0)^(1/(nu+2))."""
    return xi0(gamma, nu) * (E * t * t / rho0) ** (1.0 / (nu + 2.0))


def density(r, t: float, E: float = 1.0, rho0: float = 1.0, gamma: float = 5.0 / 3.0, nu: int = 3):
    """rho(r, t) of the similarity solution (rho0 outside the front)."""
    R = shock_radius(t, E, rho0, gamma, nu)
    lam, psi, _, _ = profile(gamma, nu)
    x = np.asarray(r, dtype=np.float64) / R
    out = np.interp(x, lam[::-1], psi[::-1], left=0.0, right=rho0)
    return np.where(x < 1.0, rho0 * out, rho0)
