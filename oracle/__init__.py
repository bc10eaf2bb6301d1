"""FP64 CPU oracle for the grad-h SPH neighbour loop (GANDALF, arXiv:1709.04488).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library ``paper_1709_04488_gb300`` and its binding) never imports, links or
calls it, and it imports nothing from the product package.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, brute-force O(N^2)
neighbour search, each function citing the paper's equation).  This module is
the ctypes marshalling around it plus the analytic reference solutions used as
pins (``riemann.py``).

Parity status per function (see the pins in ``tests/test_oracle_pins.py``):
  kernel f, f', W, dW/dr, dW/dh ........ pinned (normalisation, finite differences)
  density / h solve / Omega ............ pinned (lattice neighbour count, <1 % lattice
                                         offset, Eq. HRHO residual, continuity-equation
                                         and energy-gradient identities)
  forces (pressure) .................... pinned (exact gradient of the thermal energy)
  forces (viscosity, conductivity) ..... pinned (pairwise antisymmetry, energy balance,
                                         v=0 and uniform-u special cases)
  KDK step ............................. pinned (free translation, Sod analytic window)
  self-gravity (direct sum, zeta) ....... pinned (enclosed mass by quadrature, phi' = dphi/dr,
                                         momentum, gravity = -grad E_pot)
  gravity tree walk (KD tree, theta) .... pinned (dumbbell fields = the closed-form series
                                         through the quadrupole; error order (l/d)^3 vs
                                         (l/d)^2; theta -> 0 is the direct sum)
  neighbour lists ...................... pinned (scipy cKDTree on the same points)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EBOX, ENOCONV, ENOMEM = 0, -1, -2, -3, -9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("periodic", C.c_int),
        ("box_lo", C.c_double * 3),
        ("box_len", C.c_double * 3),
        ("eos", C.c_int),
        ("gamma", C.c_double),
        ("cs_iso", C.c_double),
        ("eta", C.c_double),
        ("alpha_av", C.c_double),
        ("beta_av", C.c_double),
        ("alpha_ac", C.c_double),
        ("c_cfl", C.c_double),
        ("h_tol", C.c_double),
        ("h_max_iter", C.c_int),
        ("use_grid", C.c_int),
        ("kernel", C.c_int),
        ("ac_signal", C.c_int),
        ("av_switch", C.c_int),
        ("alpha_min", C.c_double),
        ("av_decay", C.c_double),
        ("gravity", C.c_int),
        ("G", C.c_double),
        ("grav_theta", C.c_double),
        ("grav_leaf", C.c_int),
        ("c_grav", C.c_double),
    ]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)

_FIELDS_D = ["x", "y", "z", "vx", "vy", "vz", "u", "m", "h",
             "rho", "omega", "P", "c", "ax", "ay", "az", "du", "vsig"]
_FIELDS_I = ["nngb", "iters"]
# viscosity switch: alpha and its rate (Morris & Monaghan); gravity: zeta;
# Cullen & Dehnen: div v of the last force evaluation and the limiter xi
_FIELDS_A = ["alpha", "dalpha", "zeta", "cd_divv", "cd_xi"]


class _State(C.Structure):
    _fields_ = [(f, _DP) for f in _FIELDS_D] + [(f, _IP) for f in _FIELDS_I] + [(f, _DP) for f in _FIELDS_A]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        for name in ("orc_f", "orc_df"):
            fn = getattr(L, name)
            fn.restype = C.c_double
            fn.argtypes = [C.c_double]
        for name in ("orc_W", "orc_dWdr", "orc_dWdh"):
            fn = getattr(L, name)
            fn.restype = C.c_double
            fn.argtypes = [C.c_double, C.c_double]
        for name in ("orc_g6", "orc_dg6"):
            fn = getattr(L, name)
            fn.restype = C.c_double
            fn.argtypes = [C.c_double]
        for name in ("orc_Wk", "orc_dWdrk", "orc_dWdhk"):
            fn = getattr(L, name)
            fn.restype = C.c_double
            fn.argtypes = [C.c_int, C.c_double, C.c_double]
        for name in ("orc_gmass", "orc_gpsi"):
            fn = getattr(L, name)
            fn.restype = C.c_double
            fn.argtypes = [C.c_double]
        for name in ("orc_gforce", "orc_gpot", "orc_gdphidh"):
            fn = getattr(L, name)
            fn.restype = C.c_double
            fn.argtypes = [C.c_double, C.c_double]
        PP, SP = C.POINTER(_Params), C.POINTER(_State)
        L.orc_density.restype = C.c_int
        L.orc_density.argtypes = [PP, C.c_int64, SP]
        L.orc_forces.restype = C.c_int
        L.orc_forces.argtypes = [PP, C.c_int64, SP]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [PP, C.c_int64, SP, C.c_double]
        L.orc_gravity_energy.restype = C.c_double
        L.orc_gravity_energy.argtypes = [PP, C.c_int64, SP]
        L.orc_cfl_dt.restype = C.c_double
        L.orc_cfl_dt.argtypes = [PP, C.c_int64, SP]
        L.orc_neighbours.restype = C.c_int64
        L.orc_neighbours.argtypes = [PP, C.c_int64, SP, C.c_int, C.POINTER(C.c_int64), _IP, C.c_int64]
        L.orc_density_at_h.restype = C.c_int
        L.orc_density_at_h.argtypes = [PP, C.c_int64, SP, C.c_int64, C.c_double, _DP, _DP]
        L.orc_density_subset.restype = C.c_int
        L.orc_density_subset.argtypes = [PP, C.c_int64, SP, C.c_int64, C.POINTER(C.c_int64)]
        L.orc_forces_subset.restype = C.c_int
        L.orc_forces_subset.argtypes = [PP, C.c_int64, SP, C.c_int64, C.POINTER(C.c_int64), C.c_double]
        L.orc_block_step.restype = C.c_int
        L.orc_block_step.argtypes = [PP, C.c_int64, SP, _IP, _IP, C.c_int, C.c_int, _DP, C.POINTER(C.c_int64)]
        L.orc_cd_update.restype = None
        L.orc_cd_update.argtypes = [PP, C.c_int64, SP, _DP, C.c_double]
        L.orc_gravity_accel.restype = C.c_int
        L.orc_gravity_accel.argtypes = [PP, C.c_int64, SP, _DP, _DP, _DP]
        L.orc_multipole_accel.restype = None
        L.orc_multipole_accel.argtypes = [C.c_int64, _DP, _DP, _DP, _DP, C.c_double, C.c_double, C.c_double,
                                          C.c_int, _DP]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


@dataclass
class Params:
    """Run-time parameters of the method (defaults from the paper: eta = 1.2,
    alpha_AV = 1, beta_AV = 2 alpha_AV, C_CFL = 0.2)."""
    periodic: bool = True
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_len: tuple = (1.0, 1.0, 1.0)
    eos: str = "adiabatic"          # or "isothermal"
    gamma: float = 5.0 / 3.0
    cs_iso: float = 1.0
    eta: float = 1.2
    alpha_av: float = 1.0
    beta_av: float = 2.0
    alpha_ac: float = 1.0
    c_cfl: float = 0.2
    h_tol: float = 1e-13
    h_max_iter: int = 50
    use_grid: bool = False
    kernel: int = 0                 # 0 = M4 cubic spline (support 2h), 1 = M6 quintic (3h)
    ac_signal: int = 0              # conductivity signal speed: 0 Wadsley |v.r_hat|, 1 Price sqrt(|dP|/rho_bar)
    av_switch: int = 0              # 1: Morris & Monaghan, 2: Cullen & Dehnen viscosity switch (alpha per particle)
    alpha_min: float = 0.1          # switch: floor of alpha
    av_decay: float = 0.1           # switch: tau = h / (av_decay c)
    gravity: int = 0                # 1: self-gravity (isolated, M4), Eq. SPHSELFGRAV
    G: float = 1.0                  # gravitational constant
    grav_theta: float = 0.0         # gravity: tree opening angle theta_MAX (0: direct summation)
    grav_leaf: int = 8              # gravity tree: N_LEAF
    c_grav: float = 0.5             # gravity: acceleration time-step condition multiplier

    def _c(self) -> _Params:
        p = _Params()
        p.periodic = int(bool(self.periodic))
        p.box_lo = (C.c_double * 3)(*self.box_lo)
        p.box_len = (C.c_double * 3)(*self.box_len)
        p.eos = 0 if self.eos == "adiabatic" else 1
        p.gamma, p.cs_iso, p.eta = self.gamma, self.cs_iso, self.eta
        p.alpha_av, p.beta_av, p.alpha_ac = self.alpha_av, self.beta_av, self.alpha_ac
        p.c_cfl, p.h_tol, p.h_max_iter = self.c_cfl, self.h_tol, int(self.h_max_iter)
        p.use_grid = int(bool(self.use_grid))
        p.kernel = int(self.kernel)
        p.ac_signal = int(self.ac_signal)
        p.av_switch = int(self.av_switch)
        p.alpha_min, p.av_decay = self.alpha_min, self.av_decay
        p.gravity, p.G = int(self.gravity), self.G
        p.grav_theta, p.grav_leaf = float(self.grav_theta), int(self.grav_leaf)
        p.c_grav = float(self.c_grav)
        return p


class State:
    """SoA particle state, all FP64 (plus int32 neighbour counts and iteration
    counts).  Construct from the inputs x, y, z, vx, vy, vz, u, m and h (h <= 0
    asks for a default starting guess)."""

    def __init__(self, **arrays):
        n = len(arrays["x"])
        self.n = n
        for f in _FIELDS_D + _FIELDS_A:
            a = arrays.get(f)
            a = np.zeros(n) if a is None else np.array(a, dtype=np.float64, copy=True)
            setattr(self, f, np.ascontiguousarray(a, dtype=np.float64))
        for f in _FIELDS_I:
            setattr(self, f, np.zeros(n, dtype=np.int32))

    def copy(self) -> "State":
        s = State(**{f: getattr(self, f) for f in _FIELDS_D + _FIELDS_A})
        for f in _FIELDS_I:
            setattr(s, f, getattr(self, f).copy())
        return s

    def _c(self) -> _State:
        st = _State()
        for f in _FIELDS_D + _FIELDS_A:
            a = getattr(self, f)
            assert a.flags.c_contiguous and a.dtype == np.float64 and len(a) == self.n
            setattr(st, f, a.ctypes.data_as(_DP))
        for f in _FIELDS_I:
            setattr(st, f, getattr(self, f).ctypes.data_as(_IP))
        return st


def density(p: Params, s: State) -> int:
    """h, rho, Omega, P, c for every particle (Eqs. SPHRHO, HRHO, OMEGA)."""
    return lib().orc_density(C.byref(p._c()), s.n, C.byref(s._c()))


def forces(p: Params, s: State) -> int:
    """a, du/dt and v_sig (Eqs. GRADHMOMEQN, GRADHENEQN, MON97ARTVISC, MON97ENERGYDISS, SPH_DT)."""
    return lib().orc_forces(C.byref(p._c()), s.n, C.byref(s._c()))


def step(p: Params, s: State, dt: float) -> int:
    """One KDK step (Eqs. LFKDK1/2) with the predictor reading of the paper."""
    return lib().orc_step(C.byref(p._c()), s.n, C.byref(s._c()), float(dt))


def density_subset(p: Params, s: State, idx) -> int:
    """Density / h solve for the listed particles only (others untouched)."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    return lib().orc_density_subset(C.byref(p._c()), s.n, C.byref(s._c()), len(idx),
                                    idx.ctypes.data_as(C.POINTER(C.c_int64)))


def forces_subset(p: Params, s: State, idx, hmax: float) -> int:
    """Forces for the listed particles; their neighbours' h, rho, Omega, P, c
    must be valid; hmax bounds the h of any particle that can reach them."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    return lib().orc_forces_subset(C.byref(p._c()), s.n, C.byref(s._c()), len(idx),
                                   idx.ctypes.data_as(C.POINTER(C.c_int64)), float(hmax))


def cfl_dt(p: Params, s: State) -> float:
    """C_CFL min_i h_i / v_sig,i (Eq. SPH_DT)."""
    return lib().orc_cfl_dt(C.byref(p._c()), s.n, C.byref(s._c()))


def density_at_h(p: Params, s: State, i: int, h: float):
    """(rho_i(h), drho_i/dh) at fixed positions, Eq. SPHRHO and its h-derivative."""
    r, d = C.c_double(), C.c_double()
    rc = lib().orc_density_at_h(C.byref(p._c()), s.n, C.byref(s._c()), int(i), float(h),
                                C.byref(r), C.byref(d))
    if rc:
        raise ValueError(f"orc_density_at_h failed: {rc}")
    return r.value, d.value


def neighbours(p: Params, s: State, kind: int):
    """CSR neighbour lists (ids ascending). kind 0: r < 2 h_i (incl. self);
    kind 1: j != i, r < 2 max(h_i, h_j)."""
    off = np.zeros(s.n + 1, dtype=np.int64)
    cap = max(1, s.n * 80)
    while True:
        idx = np.zeros(cap, dtype=np.int32)
        tot = lib().orc_neighbours(C.byref(p._c()), s.n, C.byref(s._c()), int(kind),
                                   off.ctypes.data_as(C.POINTER(C.c_int64)),
                                   idx.ctypes.data_as(_IP), cap)
        if tot < 0:
            raise ValueError(f"orc_neighbours failed: {tot}")
        if tot <= cap:
            return off, idx[:tot].copy()
        cap = int(tot)


def kernel_f(q):
    return np.vectorize(lib().orc_f, otypes=[np.float64])(q)


def kernel_df(q):
    return np.vectorize(lib().orc_df, otypes=[np.float64])(q)


def kernel_W(r, h):
    return np.vectorize(lib().orc_W, otypes=[np.float64])(r, h)


def kernel_dWdr(r, h):
    return np.vectorize(lib().orc_dWdr, otypes=[np.float64])(r, h)


def kernel_dWdh(r, h):
    return np.vectorize(lib().orc_dWdh, otypes=[np.float64])(r, h)


def kernel_g6(q):
    """Quintic M6 shape g(q) (W = g / (120 pi h^3), support 3h)."""
    return np.vectorize(lib().orc_g6, otypes=[np.float64])(q)


def kernel_dg6(q):
    return np.vectorize(lib().orc_dg6, otypes=[np.float64])(q)


def grav_mass(q):
    """Enclosed mass fraction M(q) of the M4 kernel (phi' = M / r^2)."""
    return np.vectorize(lib().orc_gmass, otypes=[np.float64])(q)


def grav_force(r, h):
    """Softened gravitational force kernel phi'(r, h), Eq. GRAVFORCEKERNEL (G = 1)."""
    return np.vectorize(lib().orc_gforce, otypes=[np.float64])(r, h)


def grav_pot(r, h):
    """Softened potential phi(r, h) (-> -1/r beyond 2h)."""
    return np.vectorize(lib().orc_gpot, otypes=[np.float64])(r, h)


def grav_dphidh(r, h):
    return np.vectorize(lib().orc_gdphidh, otypes=[np.float64])(r, h)


def gravity_energy(p: Params, s: State) -> float:
    """(G/2) sum_i sum_j m_i m_j (phi(r_ij,h_i) + phi(r_ij,h_j))/2 with the state's h."""
    return lib().orc_gravity_energy(C.byref(p._c()), s.n, C.byref(s._c()))


def block_step(p: Params, s: State, level, ngb_maxlev, L: int, dl: int = 2):
    """One block step (Sec. 2.1.4) from one synchronisation to the next:
    returns (status, Delta t_MAX, force passes, particle force evaluations).
    `level` and `ngb_maxlev` (int32, length n, zeros before the first call)
    are updated in place."""
    for a in (level, ngb_maxlev):
        assert a.dtype == np.int32 and a.flags.c_contiguous and len(a) == s.n
    dtmax = C.c_double(0.0)
    counts = (C.c_int64 * 2)()
    rc = lib().orc_block_step(C.byref(p._c()), s.n, C.byref(s._c()), level.ctypes.data_as(_IP),
                              ngb_maxlev.ctypes.data_as(_IP), int(L), int(dl), C.byref(dtmax), counts)
    return rc, dtmax.value, counts[0], counts[1]


def cd_update(p: Params, s: State, d_old, dt: float) -> None:
    """The Cullen & Dehnen alpha update after a step of dt, d_old being div v
    at the step's start (the state holds the new div v, xi, h and v_sig)."""
    d = np.ascontiguousarray(d_old, dtype=np.float64)
    lib().orc_cd_update(C.byref(p._c()), s.n, C.byref(s._c()), d.ctypes.data_as(_DP), float(dt))


def gravity_accel(p: Params, s: State):
    """Long-range gravitational accelerations alone (tree walk when
    p.grav_theta > 0, else the direct sum) with the state's h: (gx, gy, gz)."""
    g = [np.zeros(s.n) for _ in range(3)]
    rc = lib().orc_gravity_accel(C.byref(p._c()), s.n, C.byref(s._c()),
                                 *[a.ctypes.data_as(_DP) for a in g])
    if rc != OK:
        raise ValueError(f"orc_gravity_accel: {rc}")
    return tuple(g)


def multipole_accel(x, y, z, m, point, quad=True):
    """Acceleration (G = 1) at `point` from the points' multipole expansion
    about their centre of mass: monopole, plus the quadrupole if `quad`."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, m)]
    out = np.zeros(3)
    lib().orc_multipole_accel(len(arrs[0]), *[a.ctypes.data_as(_DP) for a in arrs],
                              float(point[0]), float(point[1]), float(point[2]), int(bool(quad)),
                              out.ctypes.data_as(_DP))
    return out


def kernel_Wk(k, r, h):
    return np.vectorize(lambda rr, hh: lib().orc_Wk(int(k), rr, hh), otypes=[np.float64])(r, h)


def kernel_dWdrk(k, r, h):
    return np.vectorize(lambda rr, hh: lib().orc_dWdrk(int(k), rr, hh), otypes=[np.float64])(r, h)


def kernel_dWdhk(k, r, h):
    return np.vectorize(lambda rr, hh: lib().orc_dWdhk(int(k), rr, hh), otypes=[np.float64])(r, h)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


def diagnostics(p: Params, s: State) -> dict:
    """FP64 conserved quantities: total mass, momentum, energy, and the rates
    sum m a and sum m (v.a + du/dt)."""
    m = s.m
    mom = np.array([np.sum(m * s.vx), np.sum(m * s.vy), np.sum(m * s.vz)])
    ekin = 0.5 * np.sum(m * (s.vx ** 2 + s.vy ** 2 + s.vz ** 2))
    eth = np.sum(m * s.u) if p.eos == "adiabatic" else 0.0
    fsum = np.array([np.sum(m * s.ax), np.sum(m * s.ay), np.sum(m * s.az)])
    dedt = np.sum(m * (s.vx * s.ax + s.vy * s.ay + s.vz * s.az))
    if p.eos == "adiabatic":
        dedt += np.sum(m * s.du)
    return {"mass": float(np.sum(m)), "momentum": mom, "energy": float(ekin + eth),
            "force_sum": fsum, "dEdt": float(dedt)}
