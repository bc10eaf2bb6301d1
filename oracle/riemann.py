"""Exact solution of the 1D Riemann problem for an ideal gas and for an
isothermal gas (test infrastructure; used as the analytic pin for the
shock-tube tests of Sec. 6.2, Figs. ADSOD/ISOSOD).

Written from the textbook mathematics of the Riemann problem (pressure
function across shocks and rarefactions, Newton iteration for the star
pressure, self-similar sampling in x/t).  Only ``tests/`` import it.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho_k, p_k, c_k, gamma):
    """Velocity jump across the wave k as a function of the star pressure, and
    its derivative (shock branch for p > p_k, rarefaction otherwise)."""
    if p > p_k:
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        q = math.sqrt(A / (p + B))
        return (p - p_k) * q, q * (1.0 - 0.5 * (p - p_k) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * c_k / (gamma - 1.0) * ((p / p_k) ** e - 1.0)
    df = (p / p_k) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho_k * c_k)
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma):
    """Star-region pressure and velocity (Newton iteration on the pressure
    function), plus the star densities on either side of the contact."""
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    p = max(1e-12, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = _fk(p, rhoL, pL, cL, gamma)
        fR, dR = _fk(p, rhoR, pR, cR, gamma)
        g = fL + fR + (uR - uL)
        pn = p - g / (dL + dR)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fk(p, rhoL, pL, cL, gamma)
    fR, _ = _fk(p, rhoR, pR, cR, gamma)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    gm = (gamma - 1.0) / (gamma + 1.0)

    def rho_star(rho_k, p_k):
        if p > p_k:  # shock: Rankine-Hugoniot
            return rho_k * ((p / p_k + gm) / (gm * p / p_k + 1.0))
        return rho_k * (p / p_k) ** (1.0 / gamma)  # isentropic

    return p, u, rho_star(rhoL, pL), rho_star(rhoR, pR)


def wave_speeds(rhoL, uL, pL, rhoR, uR, pR, gamma):
    """Speeds of the left-wave head and tail, contact and right-wave head and
    tail (a shock has head == tail)."""
    p, u, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    if p > pL:
        sL = uL - cL * math.sqrt((gamma + 1) / (2 * gamma) * p / pL + (gamma - 1) / (2 * gamma))
        left = (sL, sL)
    else:
        csL = cL * (p / pL) ** ((gamma - 1) / (2 * gamma))
        left = (uL - cL, u - csL)
    if p > pR:
        sR = uR + cR * math.sqrt((gamma + 1) / (2 * gamma) * p / pR + (gamma - 1) / (2 * gamma))
        right = (sR, sR)
    else:
        csR = cR * (p / pR) ** ((gamma - 1) / (2 * gamma))
        right = (u + csR, uR + cR)
    return {"left": left, "contact": u, "right": right, "p_star": p, "u_star": u,
            "rho_star_L": rsL, "rho_star_R": rsR}


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    p, u, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    ws = wave_speeds(rhoL, uL, pL, rhoR, uR, pR, gamma)
    out = np.zeros((3, xi.size))
    g1 = 2.0 / (gamma + 1.0)
    g2 = (gamma - 1.0) / (gamma + 1.0)
    for k, s in enumerate(xi):
        if s <= u:  # left of contact
            if p > pL:
                st = (rhoL, uL, pL) if s < ws["left"][0] else (rsL, u, p)
            else:
                head, tail = ws["left"]
                if s <= head:
                    st = (rhoL, uL, pL)
                elif s >= tail:
                    st = (rsL, u, p)
                else:  # inside the left rarefaction fan
                    r = (g1 + g2 / cL * (uL - s)) ** (2.0 / (gamma - 1.0))
                    st = (rhoL * r, g1 * (cL + 0.5 * (gamma - 1.0) * uL + s),
                          pL * (g1 + g2 / cL * (uL - s)) ** (2.0 * gamma / (gamma - 1.0)))
        else:
            if p > pR:
                st = (rhoR, uR, pR) if s > ws["right"][0] else (rsR, u, p)
            else:
                head, tail = ws["right"][1], ws["right"][0]
                if s >= head:
                    st = (rhoR, uR, pR)
                elif s <= tail:
                    st = (rsR, u, p)
                else:
                    r = (g1 - g2 / cR * (uR - s)) ** (2.0 / (gamma - 1.0))
                    st = (rhoR * r, g1 * (-cR + 0.5 * (gamma - 1.0) * uR + s),
                          pR * (g1 - g2 / cR * (uR - s)) ** (2.0 * gamma / (gamma - 1.0)))
        out[:, k] = st
    return out[0], out[1], out[2]


def isothermal_star(rhoL, uL, rhoR, uR, cs):
    """Star density and velocity of the isothermal Riemann problem.  Shock
    branch (rho* > rho_k): u jump = cs (rho*-rho_k)/sqrt(rho* rho_k);
    rarefaction: cs ln(rho*/rho_k)."""
    def fk(r, rk):
        if r > rk:
            s = math.sqrt(r * rk)
            return cs * (r - rk) / s, cs * (r + rk) / (2.0 * r * s)
        return cs * math.log(r / rk), cs / r

    r = math.sqrt(rhoL * rhoR)
    for _ in range(200):
        fL, dL = fk(r, rhoL)
        fR, dR = fk(r, rhoR)
        g = fL + fR + (uR - uL)
        rn = r - g / (dL + dR)
        if rn <= 0:
            rn = 0.5 * r
        if abs(rn - r) < 1e-15 * r:
            r = rn
            break
        r = rn
    fL, _ = fk(r, rhoL)
    fR, _ = fk(r, rhoR)
    return r, 0.5 * (uL + uR) + 0.5 * (fR - fL)


# the classic Sod states of the shock-tube configuration (rho, u, P | rho, u, P, gamma)
SOD = (1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)


def sod_window(t: float, hmax: float):
    """Stretch of the periodic Sod tube where the solution at time t is the
    single Riemann problem at x0 = 0.5: right of the mirror problem's
    rarefaction head (the box's second discontinuity at x = 0 sends it to
    x = c_L t) and left of the contact, each edge moved inwards by 2 hmax."""
    ws = wave_speeds(*SOD)
    lo = max(0.25, -ws["left"][0] * t) + 2.0 * hmax
    hi = min(0.67, 0.5 + ws["contact"] * t) - 2.0 * hmax
    return lo, hi


def sod_l1(x, rho, vx, P, t: float, hmax: float):
    """L1 errors (1/N) sum_i |q_i - q(x_i, t)| of rho, v_x and P against the
    exact solution over the particles inside sod_window(t, hmax) (the L1
    form of the paper's shock-tube comparison, Sec. 6.2)."""
    lo, hi = sod_window(t, hmax)
    sel = (x >= lo) & (x <= hi)
    r, u, p = sample((x[sel] - 0.5) / t, *SOD)
    return (float(np.mean(np.abs(rho[sel] - r))), float(np.mean(np.abs(vx[sel] - u))),
            float(np.mean(np.abs(P[sel] - p))), int(np.sum(sel)))
