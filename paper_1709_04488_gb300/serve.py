"""Driver for the request server (sph_server_* in include/sph.h): builds seeded
request streams shaped like the serving configuration and runs them through
the library's continuous-batching loop.

Request stream: sizes log-uniform in [n_min, n_max]; each request is a
lattice, Sod or Sedov problem (uniform choice) with seeded parameters (jitter
seed, Sedov energy in [0.5, 2], Sod density ratio in [4, 10]) asking for
`nsteps` CFL steps; arrivals are a Poisson process of rate `rate` (all at
t = 0 when rate is None).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import ics
from . import sph as S

FIELDS_IN = ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h")


def sod_request(n_target: int, ratio: float, gamma: float = 1.4):
    """Sod tube at the resolution of the 36864-particle configuration
    (left spacing 1/256 x 1/128, right 1/128 x 1/64) in a shorter, narrower
    periodic box: left 8k x k x k, right 4k x k/2 x k/2, n = 9k^3, k >= 12 and
    even.  Right density 1/ratio through the particle masses, P_R = 0.1."""
    k = max(12, int(round((n_target / 9.0) ** (1.0 / 3.0))))
    k += k % 2
    L, w = k / 16.0, k / 128.0
    a, p = ics.sod(left=(8 * k, k, k), right=(4 * k, k // 2, k // 2), gamma=gamma, length=L, width=w,
                   rho=(1.0, 1.0 / ratio), P=(1.0, 0.1))
    return a, p


def make_requests(n_req: int, seed: int = 5, n_min: float = 1e3, n_max: float = 2e5, nsteps: int = 10):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        size = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        kind = int(rng.integers(3))
        sub = int(rng.integers(1 << 30))
        if kind == 0:
            nside = max(10, int(round(size ** (1.0 / 3.0))))
            a, p = ics.lattice(nside, seed=sub)
        elif kind == 1:
            a, p = sod_request(size, ratio=float(rng.uniform(4.0, 10.0)))
        else:
            nside = max(10, int(round(size ** (1.0 / 3.0))))
            a, p = ics.sedov(nside, seed=sub, E=float(rng.uniform(0.5, 2.0)))
        reqs.append({"arrays": a, "params": p, "nsteps": nsteps, "kind": ("lattice", "sod", "sedov")[kind]})
    return reqs


def poisson_arrivals(n: int, rate: float | None, seed: int = 6):
    if not rate:
        return np.zeros(n)
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


class Server:
    """Owns the device pool (a uint8 tensor) and the sph_server handle."""

    def __init__(self, pool_bytes: int, max_slots: int = 256, max_queue: int = 1 << 16,
                 precision: int = S.PREC_MIXED, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device="cuda")
        cfg = S.ServerCfg(pool=self.pool.data_ptr(), pool_bytes=int(pool_bytes), max_slots=max_slots,
                          max_queue=max_queue, stream=self.stream.cuda_stream, precision=precision)
        self.h = C.c_void_p()
        S.check(S.lib().sph_server_create(C.byref(self.h), C.byref(cfg)), "sph_server_create")
        self._keep = {}

    def submit(self, arrays: dict, params: dict, nsteps: int, arrival: float) -> int:
        n = len(arrays["x"])
        host = {f: np.ascontiguousarray(arrays[f], dtype=np.float64) for f in FIELDS_IN}
        ptr = {f: host[f].ctypes.data_as(C.POINTER(C.c_double)) for f in FIELDS_IN}
        req = S.Request(n=n, params=S.make_params(S.PREC_MIXED, **params), nsteps=int(nsteps),
                        arrival=float(arrival), **ptr)
        t = C.c_uint64(0)
        rc = S.lib().sph_server_submit(self.h, C.byref(req), C.byref(t))
        if rc != S.OK:
            raise S.SPHError(rc, "sph_server_submit")
        return t.value

    def run(self, until: float = float("inf"), virtual_clock: bool = False):
        S.check(S.lib().sph_server_run(self.h, float(until), int(bool(virtual_clock))), "sph_server_run")

    def poll(self, ticket: int, n: int, want_state: bool = False):
        res = S.Result()
        bufs = {}
        if want_state:
            for f in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho"):
                bufs[f] = np.zeros(n)
                setattr(res, f, bufs[f].ctypes.data_as(C.POINTER(C.c_double)))
        rc = S.lib().sph_server_poll(self.h, C.c_uint64(ticket), C.byref(res))
        if rc == S.EAGAIN:
            return None
        S.check(rc, "sph_server_poll")
        out = {"status": res.status, "steps_done": res.steps_done, "arrival": res.arrival,
               "admitted": res.admitted, "completed": res.completed, "t_sim": res.t_sim}
        out.update(bufs)
        return out

    def clock(self) -> float:
        return S.lib().sph_server_clock(self.h)

    def close(self):
        if self.h and self.h.value:
            S.lib().sph_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def route(reqs, arrivals, nranks: int, rate: float = 1.0e8):
    """Multi-GPU serving (one process per GPU): each request goes to the GPU
    whose queue empties first by a cost model every rank shares (its
    particle-steps at `rate` particle-updates/s per GPU, queues taken in
    arrival order, ties to the lowest rank), so every rank computes the same
    assignment from the same request stream and nothing is exchanged on the
    data path.  Returns the rank of each request."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    arrivals = np.asarray(arrivals, dtype=np.float64)
    order = np.argsort(arrivals, kind="stable")
    free = np.zeros(nranks)  # time at which each GPU's queue empties
    out = np.zeros(len(reqs), dtype=np.int64)
    for i in order:
        start = np.maximum(free, arrivals[i])
        r = int(np.argmin(start))
        free[r] = start[r] + len(reqs[i]["arrays"]["x"]) * reqs[i]["nsteps"] / rate
        out[i] = r
    return out


def run_stream(reqs, arrivals, pool_bytes: int, max_slots: int = 256, virtual_clock: bool = False):
    """Submit every request with its arrival time, drive the loop until all are
    done; returns per-request records and the makespan on the server clock."""
    srv = Server(pool_bytes, max_slots=max_slots)
    tickets = [srv.submit(r["arrays"], r["params"], r["nsteps"], t) for r, t in zip(reqs, arrivals)]
    srv.run(virtual_clock=virtual_clock)
    recs = []
    for r, tk in zip(reqs, tickets):
        o = srv.poll(tk, len(r["arrays"]["x"]))
        o["n"] = len(r["arrays"]["x"])
        o["latency"] = o["completed"] - o["arrival"]
        recs.append(o)
    makespan = srv.clock()
    srv.close()
    return recs, makespan
