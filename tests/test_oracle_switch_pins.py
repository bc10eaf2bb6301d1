"""Pins of the oracle's Morris & Monaghan (1997) viscosity switch (Sec. 2.1.1
names it; the equations are the published ones): each particle carries
alpha_i with d alpha/dt = -(alpha - alpha_min)/tau + max(-div v, 0)(alpha_max
- alpha), tau = h/(l c), and pair (i,j) uses alpha_ij = (alpha_i + alpha_j)/2
(beta_ij = beta/alpha_max alpha_ij).

The divergence estimate -(1/(Omega rho)) sum_j m_j v_ij . grad W(h_i) is exact
for a linear velocity field v = -k r: with the grad-h Omega of the same h,
sum_j m_j r_ij W'(r_ij) = -3 rho Omega, so div v = -3k at every particle of
any distribution (isolated, so that the field stays linear)."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

SW = dict(av_switch=1, alpha_min=0.1, av_decay=0.1)


def _run(O, a, p, **kw):
    P = O.Params(**p, use_grid=True, **kw)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    return P, s


def _homologous(k, n=3000, seed=3):
    a, p = ics.cloud(n, seed=seed)
    for c, x in (("vx", "x"), ("vy", "y"), ("vz", "z")):
        a[c] = -k * a[x]
    rng = np.random.default_rng(seed)
    a["alpha"] = rng.uniform(0.1, 1.0, n)
    return a, p


@pytest.mark.parametrize("k", [0.7, -0.4])
def test_rate_under_homologous_flow(oracle_mod, k):
    """Compression (k > 0): decay plus the source 3k (alpha_max - alpha);
    expansion (k < 0): decay alone."""
    O = oracle_mod
    a, p = _homologous(k)
    P, s = _run(O, a, p, **SW)
    decay = -(s.alpha - P.alpha_min) * P.av_decay * s.c / s.h
    src = 3.0 * k * (P.alpha_av - s.alpha) if k > 0 else 0.0
    want = decay + src
    assert np.max(np.abs(s.dalpha - want)) < 1e-11 * np.max(np.abs(want))


def test_decay_at_rest_follows_the_exponential(oracle_mod):
    """At rest on a perfect lattice (no forces, div v = 0) alpha relaxes to
    alpha_min as exp(-t/tau).  Kicked and predicted like u, the decaying part
    e = alpha - alpha_min follows the kick-drift-kick recurrence with the rate
    g of the last (predicted) evaluation: e_hat = e + dt g, g' = -e_hat/tau,
    e' = e + dt (g + g')/2 -- exactly -- and stays within the scheme's
    second-order error of the exponential."""
    O = oracle_mod
    a, p = ics.lattice(8, jitter=0.0, seed=1)
    a["alpha"] = np.ones(len(a["x"]))
    P, s = _run(O, a, p, **SW)
    tau = s.h[0] / (P.av_decay * s.c[0])
    assert np.allclose(s.h, s.h[0]) and np.allclose(s.c, s.c[0])
    dt = tau / 20
    for _ in range(20):
        assert O.step(P, s, dt) == O.OK
    e, g = 1.0 - P.alpha_min, -(1.0 - P.alpha_min) / tau
    for _ in range(20):
        g_new = -(e + dt * g) / tau
        e, g = e + 0.5 * dt * (g + g_new), g_new
    assert np.max(np.abs(s.alpha - (P.alpha_min + e))) < 1e-12
    exact = P.alpha_min + (1.0 - P.alpha_min) * np.exp(-1.0)
    assert np.max(np.abs(s.alpha - exact)) < 2e-3 * exact


def test_conservation_with_alpha_per_particle(oracle_mod):
    O = oracle_mod
    a, p = ics.random_cloud(1500, seed=41, mass_spread=0.4, vel=1.0, u_spread=0.6)
    a["alpha"] = np.random.default_rng(41).uniform(0.1, 1.0, 1500)
    P, s = _run(O, a, p, **SW)
    ma = s.m[:, None] * np.stack([s.ax, s.ay, s.az], 1)
    assert np.all(np.abs(ma.sum(0)) < 1e-13 * np.abs(ma).sum(0))
    terms = s.m * (s.vx * s.ax + s.vy * s.ay + s.vz * s.az) + s.m * s.du
    assert abs(terms.sum()) < 1e-12 * np.abs(terms).sum()


@pytest.mark.parametrize("frac", [1.0, 0.5])
def test_uniform_alpha_equals_constant_viscosity(oracle_mod, frac):
    """Every alpha_i = frac alpha_max gives the forces of the constant
    scheme with alpha_AV = frac alpha_max and beta_AV = frac beta."""
    O = oracle_mod
    a, p = ics.random_cloud(1500, seed=43, vel=1.0, u_spread=0.5)
    a["alpha"] = np.full(1500, frac * 1.0)
    _, s = _run(O, a, p, **SW)
    _, r = _run(O, a, p, alpha_av=frac * 1.0, beta_av=frac * 2.0)
    for f in ("ax", "ay", "az", "du", "vsig"):
        assert np.allclose(getattr(s, f), getattr(r, f), rtol=1e-13, atol=1e-13 * np.abs(getattr(r, f)).max()), f


def test_switch_needs_alpha_arrays_and_valid_bounds(oracle_mod):
    O = oracle_mod
    a, p = ics.lattice(6, seed=2)
    s = O.State(**a)
    assert O.density(O.Params(**p, av_switch=1, alpha_min=2.0), s) == O.EINVAL  # alpha_min > alpha_max
    assert O.density(O.Params(**p, av_switch=1, av_decay=0.0), s) == O.EINVAL
