"""Pins for the analytic shock-tube solutions (Sec. 6.2) and an oracle SPH
shock tube checked against them.

The exact Riemann solver is pinned by the conservation laws it must satisfy
(Rankine-Hugoniot jumps across shocks, isentropy and the Riemann invariant
across rarefactions) and by the star state of the classic Sod problem quoted
in the textbook literature (p* = 0.30313, u* = 0.92745; Toro, Riemann Solvers
and Numerical Methods for Fluid Dynamics, test 1)."""
import math

import numpy as np
import pytest

from oracle import riemann
from paper_1709_04488_gb300 import ics

SOD = (1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)


def test_sod_star_state_textbook():
    p, u, rl, rr = riemann.star_state(*SOD)
    assert abs(p - 0.30313) < 1e-5 and abs(u - 0.92745) < 1e-5
    assert abs(rl - 0.42632) < 1e-5 and abs(rr - 0.26557) < 1e-5


def test_shock_satisfies_rankine_hugoniot():
    g = 1.4
    ws = riemann.wave_speeds(*SOD)
    S = ws["right"][0]
    r1, u1, p1 = 0.125, 0.0, 0.1
    r2, u2, p2 = ws["rho_star_R"], ws["u_star"], ws["p_star"]
    m1, m2 = r1 * (u1 - S), r2 * (u2 - S)
    assert abs(m1 - m2) < 1e-12
    assert abs((r1 * (u1 - S) ** 2 + p1) - (r2 * (u2 - S) ** 2 + p2)) < 1e-12
    e1 = p1 / ((g - 1) * r1) + 0.5 * (u1 - S) ** 2 + p1 / r1
    e2 = p2 / ((g - 1) * r2) + 0.5 * (u2 - S) ** 2 + p2 / r2
    assert abs(e1 - e2) < 1e-12


def test_rarefaction_is_isentropic_with_constant_invariant():
    g = 1.4
    head, tail = riemann.wave_speeds(*SOD)["left"]
    xi = np.linspace(head, tail, 50)
    rho, u, p = riemann.sample(xi, *SOD)
    assert np.allclose(p / rho ** g, 1.0, rtol=1e-12)
    c = np.sqrt(g * p / rho)
    assert np.allclose(u + 2 * c / (g - 1), 2 * math.sqrt(1.4) / 0.4, rtol=1e-12)
    # the fan is self-similar: u - c = xi inside it
    assert np.allclose(u - c, xi, atol=1e-12)


def test_isothermal_shock_jump():
    cs = 1.0
    r, u = riemann.isothermal_star(1.0, 0.0, 0.25, 0.0, cs)
    # right shock: mass and momentum flux continuous
    # shock speed from mass flux: S = (r u - 0) / (r - 0.25)
    S = r * u / (r - 0.25)
    assert abs(0.25 * (0 - S) ** 2 + cs ** 2 * 0.25 - (r * (u - S) ** 2 + cs ** 2 * r)) < 1e-12
    # left rarefaction: u + cs ln rho constant
    assert abs(u + cs * math.log(r) - 0.0) < 1e-12


def _binned(x, q, edges):
    k = np.digitize(x, edges) - 1
    return np.array([q[k == b].mean() if np.any(k == b) else np.nan for b in range(len(edges) - 1)])


@pytest.mark.slow
def test_oracle_sod_wave_positions(oracle_mod):
    """3D Sod tube (Sec. 6.2 set-up in 3D: left rho=1, P=1 on 32x16x16, right
    rho=0.125, P=0.1 on 16x8x8, periodic [0,1) x [0,1/4)^2, gamma=1.4), run with
    the oracle to t = 0.1, before the mirrored interface at x = 0 interacts.
    The rarefaction head, the contact and the shock must sit where the exact
    solution puts them (0.3817, 0.5927, 0.6752) to within two smoothing
    lengths; the fan must be isentropic (P/rho^gamma = 1); momentum stays zero
    and energy is conserved to the integration error.  The plateau values
    themselves are not pinned: planar expansion of a 3D lattice makes it
    anisotropic, which biases the SPH density sum there by up to ~20 %."""
    O = oracle_mod
    a, p = ics.sod(left=(32, 16, 16), right=(16, 8, 8), width=0.25)
    P = O.Params(**p, use_grid=True)
    s = O.State(**a)
    assert O.density(P, s) == O.OK
    assert O.forces(P, s) == O.OK
    e0 = O.diagnostics(P, s)["energy"]
    t, tend = 0.0, 0.1
    while t < tend - 1e-12:
        dt = min(O.cfl_dt(P, s), tend - t)
        assert O.step(P, s, dt) == O.OK
        t += dt
    ws = riemann.wave_speeds(*SOD)
    head = 0.5 + ws["left"][0] * t
    contact = 0.5 + ws["contact"] * t
    shock = 0.5 + ws["right"][0] * t
    edges = np.linspace(0.25, 0.75, 201)
    xc = 0.5 * (edges[1:] + edges[:-1])
    vx = _binned(s.x, s.vx, edges)
    rho = _binned(s.x, s.rho, edges)
    hL = np.median(s.h[s.x < 0.3])
    x_head = xc[np.argmax(vx > 0.05 * ws["u_star"])]
    assert abs(x_head - head) < 2 * hL
    rc = 0.5 * (ws["rho_star_L"] + ws["rho_star_R"])
    sel = (xc > 0.5) & (xc < shock + 0.05)
    x_contact = xc[sel][np.argmax(rho[sel] < rc)]
    assert abs(x_contact - contact) < 2 * hL
    rs = 0.5 * (ws["rho_star_R"] + 0.125)
    x_shock = xc[sel][np.where(rho[sel] > rs)[0].max()]
    hR = np.median(s.h[(s.x > 0.8) & (s.x < 0.9)])
    assert abs(x_shock - shock) < 2 * hR
    fan = (s.x > head + 2 * hL) & (s.x < 0.5 + ws["left"][1] * t - 2 * hL)
    assert np.allclose(s.P[fan] / s.rho[fan] ** 1.4, 1.0, rtol=0.02)
    d = O.diagnostics(P, s)
    assert np.all(np.abs(d["momentum"]) < 1e-13)
    assert abs(d["energy"] - e0) < 1e-4 * e0
