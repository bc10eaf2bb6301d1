"""Pins of the oracle's gravity tree walk (Sec. 4.2): a KD tree split at the
median along each cell's most elongated axis, cells used through their
monopole and quadrupole moments when |r_i - r_c|^2 >= l_c^2 / theta^2 and
no pair with the cell is softened.

- The multipole field of a dumbbell (masses m at +-a on the z axis) equals
  the closed-form series through second order, on the axis
  -(2Gm/d^2)(1 + 3a^2/d^2) and in the equatorial plane
  -(2Gm/d^2)(1 - 3a^2/(2d^2)); the monopole alone is -2Gm/d^2.
- For any cluster, the error against the exact sum falls as (l/d)^3 with the
  quadrupole (as (l/d)^2 without), so doubling d divides it by ~8 (~4).
- theta -> 0 opens every cell: the walk then visits each particle once and
  equals the direct sum to rounding.
- A ball in which every pair is softened leaves no cell usable: the walk
  equals the direct sum at any theta.
- The error against the direct sum shrinks with theta.
- In the force pass only the long-range part changes with theta."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

GR = dict(gravity=1, G=1.0)


def _direct_field(x, y, z, m, pt):
    d = np.stack([pt[0] - x, pt[1] - y, pt[2] - z], 1)
    r = np.linalg.norm(d, axis=1)
    return -(m[:, None] * d / r[:, None] ** 3).sum(0)


@pytest.mark.parametrize("d", [0.8, 1.5, 3.0])
def test_dumbbell_equals_the_second_order_series(oracle_mod, d):
    O = oracle_mod
    m, a = 0.7, 0.1
    x, y, z, ms = [0.0, 0.0], [0.0, 0.0], [-a, a], [m, m]
    axis = O.multipole_accel(x, y, z, ms, (0.0, 0.0, d))
    assert axis[0] == 0.0 and axis[1] == 0.0
    assert axis[2] == pytest.approx(-(2 * m / d ** 2) * (1 + 3 * a ** 2 / d ** 2), rel=1e-14)
    eq = O.multipole_accel(x, y, z, ms, (d, 0.0, 0.0))
    assert eq[0] == pytest.approx(-(2 * m / d ** 2) * (1 - 1.5 * a ** 2 / d ** 2), rel=1e-14)
    assert abs(eq[1]) < 1e-16 and abs(eq[2]) < 1e-16
    mono = O.multipole_accel(x, y, z, ms, (0.0, 0.0, d), quad=False)
    assert mono[2] == pytest.approx(-2 * m / d ** 2, rel=1e-15)


def test_multipole_error_order(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(3)
    x, y, z = rng.normal(0.0, 0.1, (3, 40))
    m = rng.uniform(0.5, 1.5, 40)
    for _ in range(4):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        for quad, lo, hi in ((True, 6.5, 9.5), (False, 3.0, 5.0)):
            err = []
            for d in (5.0, 10.0):
                ex = _direct_field(x, y, z, m, u * d)
                err.append(np.linalg.norm(O.multipole_accel(x, y, z, m, u * d, quad) - ex) / np.linalg.norm(ex))
            assert lo < err[0] / err[1] < hi, (quad, err)


def _solved(O, a, p, **kw):
    P = O.Params(**p, use_grid=True, **GR, **kw)
    s = O.State(**a)
    assert O.density(P, s) == O.OK
    return s


def _g(O, p, s, theta, leaf=8):
    P = O.Params(**p, use_grid=True, **GR, grav_theta=theta, grav_leaf=leaf)
    return np.stack(O.gravity_accel(P, s), 1)


@pytest.mark.parametrize("leaf", [1, 8, 33])
def test_tiny_theta_is_the_direct_sum(oracle_mod, leaf):
    O = oracle_mod
    a, p = ics.cloud(1500, seed=81)
    a["m"] = a["m"] * np.random.default_rng(81).uniform(0.5, 1.5, 1500)
    s = _solved(O, a, p)
    g0 = _g(O, p, s, 0.0)
    rms = np.sqrt(np.mean(np.sum(g0 ** 2, 1)))
    assert np.max(np.abs(_g(O, p, s, 1e-9, leaf) - g0)) < 1e-13 * rms


def test_softened_ball_is_never_approximated(oracle_mod):
    """All particles within 2h of one another: no cell is usable."""
    O = oracle_mod
    a, p = ics.cloud(300, seed=82)
    s = _solved(O, a, p)
    s.h[:] = 2.0 * np.max(np.ptp(np.stack([s.x, s.y, s.z]), axis=1))
    g0 = _g(O, p, s, 0.0)
    g1 = _g(O, p, s, 1.0, leaf=4)
    assert np.max(np.abs(g1 - g0)) < 1e-13 * np.sqrt(np.mean(np.sum(g0 ** 2, 1)))


def test_error_shrinks_with_theta(oracle_mod):
    O = oracle_mod
    a, p = ics.cloud(3000, seed=5)
    s = _solved(O, a, p)
    g0 = _g(O, p, s, 0.0)
    rms = np.sqrt(np.mean(np.sum(g0 ** 2, 1)))
    errs = [np.sqrt(np.mean(np.sum((_g(O, p, s, t) - g0) ** 2, 1))) / rms for t in (0.2, 0.4, 0.7, 1.0)]
    assert all(e1 < e2 for e1, e2 in zip(errs, errs[1:])), errs
    assert 0 < errs[0] < 2e-4 and errs[-1] < 2e-2, errs


def test_force_pass_changes_only_by_the_long_range_part(oracle_mod):
    O = oracle_mod
    a, p = ics.cloud(1200, seed=83)
    for c in ("vx", "vy", "vz"):
        a[c] = 0.3 * a[c]
    out = {}
    for th in (0.0, 0.6):
        P = O.Params(**p, use_grid=True, **GR, grav_theta=th)
        s = O.State(**a)
        assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
        out[th] = (np.stack([s.ax, s.ay, s.az], 1), s.du.copy(), _g(O, p, s, th))
    (a0, du0, g0), (a1, du1, g1) = out[0.0], out[0.6]
    rms = np.sqrt(np.mean(np.sum(a0 ** 2, 1)))
    assert np.array_equal(du0, du1)
    assert np.max(np.abs((a1 - a0) - (g1 - g0))) < 1e-12 * rms
    assert np.max(np.abs(g1 - g0)) > 1e-6 * rms  # the walk did approximate


def test_theta_out_of_range_is_rejected(oracle_mod):
    O = oracle_mod
    a, p = ics.cloud(100, seed=84)
    s = O.State(**a)
    assert O.density(O.Params(**p, **GR, grav_theta=1.5), s) == O.EINVAL
    assert O.density(O.Params(**p, **GR, grav_theta=0.5, grav_leaf=0), s) == O.EINVAL
