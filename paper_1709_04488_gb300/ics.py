"""Seeded synthetic initial conditions shaped like the paper's test problems.

This module holds no step of the SPH method itself: it only places particles
and assigns their masses, velocities and internal energies.  Both the CUDA path
(through ``bench.py``, the tests and the request-stream driver ``serve.py``) and
the CPU oracle (through the tests) are fed from here; it imports nothing from
the rest of the package, and nothing on the compute path imports it.

Every generator returns ``(arrays, params)``: ``arrays`` maps x, y, z, vx, vy,
vz, u, m, h to float64 NumPy arrays; ``params`` holds the problem's physical
parameters (box, EOS, gamma).  ``h`` is only a starting guess for the
smoothing-length iteration (1.2 times the local mean inter-particle spacing
implied by the set-up); converged results do not depend on it.

Recipes (seeds fixed; same bits on any host):
  lattice  periodic unit cube, n^3 particles at cell centres plus a uniform
           jitter of +-0.1 spacing per axis, total mass 1, v = 0, u = 1.5,
           gamma = 5/3 (the paper's uniform-density set-ups, Sec. 6.1).
  sod      3D shock tube in the periodic box [0,1) x [0,1/8) x [0,1/8):
           left x < 0.5 rho = 1, P = 1 on a 128x16x16 lattice, right rho = 0.125,
           P = 0.1 on a 64x8x8 lattice (equal masses), gamma = 1.4, v = 0
           (Sec. 6.2 shock tubes, in 3D with the classic Sod states).
  sedov    n^3 jittered lattice in the periodic unit cube, rho = 1, u = 1e-5,
           energy E deposited into the 64 particles nearest the centre with
           weights of the M4 shape at h_c = half the distance of the 65th
           nearest particle (Sec. 6.3, in 3D).
  cloud    isolated sphere of radius 1 and mass 1 with rho ~ 1/(1 + r^2/a^2),
           a = 0.1; isothermal, c_s = 1; Gaussian random velocity field with
           |v_k|^2 ~ k^-4 for 2 <= |k| <= 64 on a 128^3 grid over [-1,1]^3,
           interpolated trilinearly, mean removed, rms |v| = 5 c_s.
"""
from __future__ import annotations

import math

import numpy as np


def _guess_h(m, rho_est):
    # starting guess only: 1.2 x (volume per particle)^(1/3)
    return 1.2 * np.cbrt(m / rho_est)


def lattice(n_side: int = 16, jitter: float = 0.1, seed: int = 1, u: float = 1.5,
            gamma: float = 5.0 / 3.0):
    rng = np.random.default_rng(seed)
    d = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * d
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    pos += rng.uniform(-jitter, jitter, size=pos.shape) * d
    pos %= 1.0
    n = pos.shape[0]
    m = np.full(n, 1.0 / n)
    arrays = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                  vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n),
                  u=np.full(n, float(u)), m=m, h=_guess_h(m, 1.0))
    params = dict(periodic=True, box_lo=(0.0, 0.0, 0.0), box_len=(1.0, 1.0, 1.0),
                  eos="adiabatic", gamma=gamma)
    return arrays, params


def _block(nx, ny, nz, lo, hi):
    gx = lo[0] + (np.arange(nx) + 0.5) * (hi[0] - lo[0]) / nx
    gy = lo[1] + (np.arange(ny) + 0.5) * (hi[1] - lo[1]) / ny
    gz = lo[2] + (np.arange(nz) + 0.5) * (hi[2] - lo[2]) / nz
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def sod(left=(128, 16, 16), right=(64, 8, 8), rho=(1.0, 0.125), P=(1.0, 0.1),
        gamma: float = 1.4, length: float = 1.0, width: float = 0.125, jitter: float = 0.0, seed: int = 1):
    """Shock tube split at x = length/2 in a periodic box length x width x width.
    jitter > 0 moves every particle by a uniform random offset of up to
    jitter x its lattice spacing per axis (seeded; none by default)."""
    Lb = (length, width, width)
    pl = _block(*left, (0.0, 0.0, 0.0), (0.5 * length, width, width))
    pr = _block(*right, (0.5 * length, 0.0, 0.0), (length, width, width))
    if jitter > 0:
        rng = np.random.default_rng(seed)
        dl = np.array([0.5 * length / left[0], width / left[1], width / left[2]])
        dr = np.array([0.5 * length / right[0], width / right[1], width / right[2]])
        pl = pl + rng.uniform(-jitter, jitter, pl.shape) * dl
        pr = pr + rng.uniform(-jitter, jitter, pr.shape) * dr
    vol = 0.5 * length * width * width
    ml = rho[0] * vol / pl.shape[0]
    mr = rho[1] * vol / pr.shape[0]
    pos = np.concatenate([pl, pr])
    n = pos.shape[0]
    m = np.concatenate([np.full(len(pl), ml), np.full(len(pr), mr)])
    u = np.concatenate([np.full(len(pl), P[0] / ((gamma - 1.0) * rho[0])),
                        np.full(len(pr), P[1] / ((gamma - 1.0) * rho[1]))])
    rho_est = np.concatenate([np.full(len(pl), rho[0]), np.full(len(pr), rho[1])])
    arrays = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                  vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n), u=u, m=m,
                  h=_guess_h(m, rho_est))
    params = dict(periodic=True, box_lo=(0.0, 0.0, 0.0), box_len=Lb, eos="adiabatic",
                  gamma=gamma)
    return arrays, params


def _m4_shape(q):
    # initial-condition weights for the energy deposit (cubic-spline shape)
    q = np.asarray(q, dtype=np.float64)
    w = np.where(q < 1.0, 1.0 - 1.5 * q ** 2 + 0.75 * q ** 3, 0.25 * np.clip(2.0 - q, 0, None) ** 3)
    return np.where(q < 2.0, w, 0.0)


def sedov(n_side: int = 100, seed: int = 3, E: float = 1.0, u0: float = 1e-5,
          gamma: float = 5.0 / 3.0, jitter: float = 0.1, n_hot: int = 64):
    arrays, params = lattice(n_side=n_side, jitter=jitter, seed=seed, u=u0, gamma=gamma)
    x, y, z = arrays["x"], arrays["y"], arrays["z"]
    d2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    order = np.lexsort((np.arange(len(d2)), d2))  # nearest first, ties by id
    hot = order[:n_hot]
    hc = 0.5 * math.sqrt(d2[order[n_hot]])
    w = _m4_shape(np.sqrt(d2[hot]) / hc)
    m = arrays["m"]
    arrays["u"][hot] += E * w / (m[hot] * w.sum())
    return arrays, params


def _cloud_radii(n, a, R, rng):
    # invert M(<r)/M = (r - a atan(r/a)) / (R - a atan(R/a)) by bisection
    # (in cache-sized chunks; every element takes the same 60 halvings)
    target = rng.uniform(0.0, 1.0, n) * (R - a * math.atan(R / a))
    out = np.empty(n)
    chunk = 1 << 16
    mid = np.empty(chunk)
    f = np.empty(chunk)
    below = np.empty(chunk, dtype=bool)
    for c0 in range(0, n, chunk):
        t = target[c0:c0 + chunk]
        m = len(t)
        lo = np.zeros(m)
        hi = np.full(m, R)
        md, fm, bl = mid[:m], f[:m], below[:m]
        for _ in range(60):
            np.add(lo, hi, out=md)
            md *= 0.5
            np.divide(md, a, out=fm)
            np.arctan(fm, out=fm)
            fm *= a
            np.subtract(md, fm, out=fm)
            np.less(fm, t, out=bl)
            np.copyto(lo, md, where=bl)
            np.copyto(hi, md, where=~bl)
        out[c0:c0 + m] = 0.5 * (lo + hi)
    return out


def _random_field(ngrid, kmin, kmax, rng):
    k = np.fft.fftfreq(ngrid, d=1.0 / ngrid)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    amp = np.zeros_like(kk)
    sel = (kk >= kmin) & (kk <= kmax)
    amp[sel] = kk[sel] ** -2.0  # |v_k|^2 ~ k^-4
    comps = []
    for _ in range(3):
        noise = rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape)
        comps.append(np.real(np.fft.ifftn(noise * amp)))
    return comps


def _trilinear(fields, pos, lo, L):
    # the same weights and cells serve every field; one gather per corner
    # fetches the values of all fields at that node
    ng = fields[0].shape[0]
    F = np.stack([fd.ravel() for fd in fields], axis=1)
    out = np.zeros((len(pos), len(fields)))
    chunk = 1 << 18
    for c0 in range(0, len(pos), chunk):
        s = (pos[c0:c0 + chunk] - lo) / L * ng - 0.5
        i0 = np.floor(s).astype(np.int64)
        f = s - i0
        o = out[c0:c0 + chunk]
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) *
                         (f[:, 2] if dz else 1 - f[:, 2]))
                    ix = (i0[:, 0] + dx) % ng
                    iy = (i0[:, 1] + dy) % ng
                    iz = (i0[:, 2] + dz) % ng
                    o += w[:, None] * F[(iz * ng + iy) * ng + ix]
    return [out[:, k].copy() for k in range(len(fields))]


def cloud(n: int = 8_000_000, seed: int = 4, a: float = 0.1, R: float = 1.0, mach: float = 5.0,
          cs: float = 1.0, ngrid: int = 128, kmin: float = 2.0, kmax: float = 64.0):
    rng = np.random.default_rng(seed)
    r = _cloud_radii(n, a, R, rng)
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(1.0 - mu ** 2)
    pos = np.stack([r * st * np.cos(phi), r * st * np.sin(phi), r * mu], axis=1)
    vf = _random_field(ngrid, kmin, kmax, rng)
    v = np.stack(_trilinear(vf, pos, -1.0, 2.0), axis=1)
    v -= v.mean(axis=0)
    v *= mach * cs / math.sqrt(np.mean(np.sum(v ** 2, axis=1)))
    m = np.full(n, 1.0 / n)
    rho0 = 1.0 / (4.0 * math.pi * a * a * (R - a * math.atan(R / a)))
    rho_est = rho0 / (1.0 + (r / a) ** 2)
    arrays = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                  vx=v[:, 0].copy(), vy=v[:, 1].copy(), vz=v[:, 2].copy(),
                  u=np.zeros(n), m=m, h=_guess_h(m, rho_est))
    params = dict(periodic=False, box_lo=(0.0, 0.0, 0.0), box_len=(0.0, 0.0, 0.0),
                  eos="isothermal", cs_iso=cs, gamma=1.0)
    return arrays, params


def random_cloud(n: int, seed: int, periodic: bool = True, mass_spread: float = 0.0,
                 vel: float = 0.0, u_spread: float = 0.0):
    """Uniform random positions (a stress case, not a paper set-up) with
    optional unequal masses, random velocities and internal energies."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(n, 3))
    m = np.full(n, 1.0 / n) * (1.0 + mass_spread * rng.uniform(-1, 1, n))
    v = rng.normal(0.0, vel, size=(n, 3)) if vel > 0 else np.zeros((n, 3))
    u = 1.0 + u_spread * rng.uniform(-1, 1, n)
    arrays = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                  vx=v[:, 0].copy(), vy=v[:, 1].copy(), vz=v[:, 2].copy(), u=u, m=m,
                  h=_guess_h(m, np.sum(m)))
    params = dict(periodic=periodic, box_lo=(0.0, 0.0, 0.0),
                  box_len=(1.0, 1.0, 1.0) if periodic else (0.0, 0.0, 0.0),
                  eos="adiabatic", gamma=5.0 / 3.0)
    return arrays, params
