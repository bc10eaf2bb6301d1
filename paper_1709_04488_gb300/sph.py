"""ctypes binding of libsph.so (include/sph.h), plus a small helper that owns
the caller-side device memory as PyTorch tensors.

Argument marshalling only: every step of the method runs in the CUDA library.
If libsph.so is missing the import of this module fails loudly; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SPH_LIB_PATH") or os.path.join(HERE, "libsph.so")

OK, EINVAL, EBOX, ENOCONV, ENONFINITE, ETIMEOUT, ETOOBIG, EBUSY, EAGAIN, ECUDA, ENOSPACE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10)
EOS_ADIABATIC, EOS_ISOTHERMAL = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
KERNEL_M4, KERNEL_M6 = 0, 1
AC_WADSLEY, AC_PRICE = 0, 1
AV_CONSTANT, AV_MORRIS_MONAGHAN, AV_CULLEN_DEHNEN = 0, 1, 2
FLAG_ASYNC, FLAG_TIMING = 1, 2
NSTAGES = 8
STAGES = ["kick_drift", "sort", "tree", "density", "refit", "forces", "gravity", "close"]

_DP = C.POINTER(C.c_double)


class Params(C.Structure):
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
        ("precision", C.c_int),
        ("kernel", C.c_int),
        ("leaf_size", C.c_int),
        ("lanes_per_particle", C.c_int),
        ("flags", C.c_uint),
        ("tree_rebuild_every", C.c_int),
        ("ac_signal", C.c_int),
        ("av_switch", C.c_int),
        ("alpha_min", C.c_double),
        ("av_decay", C.c_double),
        ("gravity", C.c_int),
        ("G", C.c_double),
        ("grav_theta", C.c_double),
        ("c_grav", C.c_double),
        ("block_levels", C.c_int),
        ("block_gap", C.c_int),
    ]


STATE_FIELDS = ["x", "y", "z", "vx", "vy", "vz", "u", "m", "h",
                "rho", "omega", "P", "c", "ax", "ay", "az", "du", "vsig", "alpha", "dalpha"]


class State(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in STATE_FIELDS]


class Diag(C.Structure):
    _fields_ = [
        ("mass", C.c_double),
        ("momentum", C.c_double * 3),
        ("energy", C.c_double),
        ("force_sum", C.c_double * 3),
        ("dEdt", C.c_double),
        ("dt_next", C.c_double),
        ("time", C.c_double),
        ("steps", C.c_int64),
        ("nr_iterations", C.c_int64),
        ("nr_max", C.c_int32),
        ("ngb_min", C.c_int32),
        ("ngb_max", C.c_int32),
        ("ngb_mean", C.c_double),
        ("density_pairs", C.c_int64),
        ("force_pairs", C.c_int64),
        ("candidates", C.c_int64),
        ("fallback", C.c_int64),
        ("leaves", C.c_int64),
        ("status", C.c_int32),
        ("unconverged", C.c_int32),
        ("walk_reused", C.c_int32),
        ("wrap_leaves", C.c_int32),
        ("grav_pairs", C.c_int64),
        ("grav_nodes", C.c_int64),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class ServerCfg(C.Structure):
    _fields_ = [
        ("pool", C.c_void_p),
        ("pool_bytes", C.c_size_t),
        ("max_slots", C.c_int),
        ("max_queue", C.c_int),
        ("stream", C.c_void_p),
        ("precision", C.c_int),
    ]


class Request(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(f, _DP) for f in ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h")] + [
        ("params", Params),
        ("nsteps", C.c_int),
        ("arrival", C.c_double),
    ]


class Result(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("n", C.c_int64),
        ("steps_done", C.c_int),
        ("arrival", C.c_double),
        ("admitted", C.c_double),
        ("completed", C.c_double),
        ("t_sim", C.c_double),
    ] + [(f, _DP) for f in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho")]


class SPHError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where} failed with status {code}: {last_error()}")


_lib = None


def lib():
    """Load libsph.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "sph_params_default": (i, [C.POINTER(Params)]),
            "sph_workspace_bytes": (C.c_size_t, [i64, C.POINTER(Params)]),
            "sph_setup": (i, [C.POINTER(vp), C.POINTER(Params), i64, C.POINTER(State), vp, C.c_size_t, vp]),
            "sph_density_h": (i, [vp]),
            "sph_forces": (i, [vp]),
            "sph_step": (i, [vp, d, C.POINTER(d)]),
            "sph_run": (i, [vp, i]),
            "sph_block_step": (i, [vp, C.POINTER(d), C.POINTER(i64)]),
            "sph_block_levels": (i, [vp, vp]),
            "sph_block_prepare": (i, [vp]),
            "sph_sync": (i, [vp]),
            "sph_diagnostics": (i, [vp, C.POINTER(Diag)]),
            "sph_neighbours": (i, [vp, i, vp, vp, vp, i64, C.POINTER(i64)]),
            "sph_destroy": (i, [vp]),
            "sph_stage_times": (i, [vp, C.POINTER(d)]),
            "sph_step_kernel_count": (i, [vp, C.POINTER(i)]),
            "sph_batch_workspace_bytes": (C.c_size_t, [C.POINTER(vp), i]),
            "sph_batch_step": (i, [C.POINTER(vp), i, i, vp, C.c_size_t]),
            "sph_server_create": (i, [C.POINTER(vp), C.POINTER(ServerCfg)]),
            "sph_server_submit": (i, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
            "sph_server_run": (i, [vp, d, i]),
            "sph_server_poll": (i, [vp, C.c_uint64, C.POINTER(Result)]),
            "sph_server_clock": (d, [vp]),
            "sph_server_destroy": (i, [vp]),
            "sph_density_forces_noalloc": (i, [C.POINTER(Params), i64, C.POINTER(State), vp]),
            "sph_last_error": (C.c_char_p, []),
            "sph_version": (C.c_char_p, []),
            "sph_set_launch_table": (i, [C.POINTER(i64), C.POINTER(C.c_int32), i]),
            "sph_alu_peak": (i, [i, d, C.POINTER(d), C.POINTER(d), vp]),
            "sph_batch_create": (i, [C.POINTER(vp), C.POINTER(vp), i, vp, C.c_size_t, C.c_uint]),
            "sph_batch_run": (i, [vp, i]),
            "sph_batch_sync": (i, [vp, C.POINTER(i)]),
            "sph_batch_stage_times": (i, [vp, C.POINTER(d)]),
            "sph_batch_kernel_count": (i, [vp, C.POINTER(i)]),
            "sph_batch_destroy": (i, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        _install_tuning(L)
    return _lib


TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def set_launch_table(rows, L=None):
    """Install [(n_max, lanes_per_particle), ...] (see sph_set_launch_table)."""
    L = L or lib()
    n = len(rows)
    nm = (C.c_int64 * max(n, 1))(*[int(r[0]) for r in rows])
    ln = (C.c_int32 * max(n, 1))(*[int(r[1]) for r in rows])
    rc = L.sph_set_launch_table(nm, ln, n)
    if rc != OK:
        raise SPHError(rc, "sph_set_launch_table")


def _install_tuning(L):
    # the autotuner's measured table (paper_1709_04488_gb300/tuning.json), if any
    if os.environ.get("SPH_NO_TUNING") or not os.path.exists(TUNING_PATH):
        return
    import json
    with open(TUNING_PATH) as f:
        rows = json.load(f).get("lpp_table", [])
    set_launch_table(rows, L)


def last_error() -> str:
    try:
        return lib().sph_last_error().decode()
    except Exception:  # pragma: no cover
        return ""


def check(rc: int, where: str, allow=()):
    if rc != OK and rc not in allow:
        raise SPHError(rc, where)
    return rc


# ---- thin wrappers with the C names -------------------------------------------
def sph_params_default() -> Params:
    p = Params()
    check(lib().sph_params_default(C.byref(p)), "sph_params_default")
    return p


def sph_workspace_bytes(n: int, p: Params) -> int:
    return int(lib().sph_workspace_bytes(int(n), C.byref(p)))


def sph_setup(p: Params, n: int, state: State, ws_ptr: int, ws_bytes: int, stream: int):
    ctx = C.c_void_p()
    rc = lib().sph_setup(C.byref(ctx), C.byref(p), int(n), C.byref(state), C.c_void_p(ws_ptr), int(ws_bytes),
                         C.c_void_p(stream))
    return rc, ctx


def sph_density_h(ctx) -> int:
    return lib().sph_density_h(ctx)


def sph_forces(ctx) -> int:
    return lib().sph_forces(ctx)


def sph_step(ctx, dt: float):
    used = C.c_double(0.0)
    rc = lib().sph_step(ctx, float(dt), C.byref(used))
    return rc, used.value


def sph_step_nowait(ctx, dt: float) -> int:
    return lib().sph_step(ctx, float(dt), None)


def sph_run(ctx, nsteps: int) -> int:
    return lib().sph_run(ctx, int(nsteps))


def sph_block_step(ctx):
    """One block step: (status, Delta t_MAX, particle force evaluations)."""
    dtmax = C.c_double(0.0)
    evals = C.c_int64(0)
    rc = lib().sph_block_step(ctx, C.byref(dtmax), C.byref(evals))
    return rc, dtmax.value, evals.value


def sph_block_prepare(ctx) -> int:
    """Capture the block step's graph now (nothing runs)."""
    return lib().sph_block_prepare(ctx)


def sph_block_levels(ctx, levels_ptr) -> int:
    return lib().sph_block_levels(ctx, levels_ptr)


def sph_sync(ctx) -> int:
    return lib().sph_sync(ctx)


def sph_diagnostics(ctx) -> Diag:
    d = Diag()
    check(lib().sph_diagnostics(ctx, C.byref(d)), "sph_diagnostics")
    return d


def sph_neighbours(ctx, kind: int, h_ptr: int, off_ptr: int, idx_ptr: int, cap: int):
    tot = C.c_int64(0)
    rc = lib().sph_neighbours(ctx, int(kind), C.c_void_p(h_ptr) if h_ptr else None, C.c_void_p(off_ptr),
                              C.c_void_p(idx_ptr), int(cap), C.byref(tot))
    return rc, tot.value


def sph_destroy(ctx) -> int:
    return lib().sph_destroy(ctx)


def sph_stage_times(ctx) -> list:
    ms = (C.c_double * NSTAGES)()
    check(lib().sph_stage_times(ctx, ms), "sph_stage_times")
    return list(ms)


def sph_step_kernel_count(ctx) -> int:
    k = C.c_int(0)
    check(lib().sph_step_kernel_count(ctx, C.byref(k)), "sph_step_kernel_count")
    return k.value


def sph_density_forces_noalloc(p: Params, n: int, state: State, stream: int) -> int:
    """Density solve + force evaluation with the library's fixed scratch
    memory (no allocation); at most 32768 particles."""
    return lib().sph_density_forces_noalloc(C.byref(p), int(n), C.byref(state), C.c_void_p(stream))


def sph_batch_workspace_bytes(ctxs) -> int:
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    return int(lib().sph_batch_workspace_bytes(arr, len(ctxs)))


def sph_batch_step(ctxs, nsteps: int, ws_ptr: int, ws_bytes: int) -> int:
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    return lib().sph_batch_step(arr, len(ctxs), int(nsteps), C.c_void_p(ws_ptr), int(ws_bytes))


class Batch:
    """A resident batch of Problems (sph_batch_*): tables uploaded once, the
    batched step captured as a CUDA graph on the first run.  The problems
    must share precision and a non-default stream and have a force
    evaluation."""

    def __init__(self, problems, flags: int = 0):
        import torch
        self.problems = list(problems)
        self.stream = self.problems[0].stream
        self._arr = (C.c_void_p * len(self.problems))(*[p.ctx.value for p in self.problems])
        self.ws_bytes = int(lib().sph_batch_workspace_bytes(self._arr, len(self.problems)))
        if self.ws_bytes == 0:
            raise SPHError(EINVAL, "sph_batch_workspace_bytes")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.problems[0].device)
        self.h = C.c_void_p()
        check(lib().sph_batch_create(C.byref(self.h), self._arr, len(self.problems), C.c_void_p(self.ws.data_ptr()),
                                     self.ws_bytes, int(flags)), "sph_batch_create")

    def run(self, nsteps: int):
        check(lib().sph_batch_run(self.h, int(nsteps)), "sph_batch_run")

    def sync(self):
        """Per-problem statuses (list) after waiting for the batch's work."""
        st = (C.c_int * len(self.problems))()
        lib().sph_batch_sync(self.h, st)
        return list(st)

    def stage_times(self):
        ms = (C.c_double * NSTAGES)()
        check(lib().sph_batch_stage_times(self.h, ms), "sph_batch_stage_times")
        return list(ms)

    def kernel_count(self) -> int:
        k = C.c_int(0)
        check(lib().sph_batch_kernel_count(self.h, C.byref(k)), "sph_batch_kernel_count")
        return k.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sph_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- helper: problem state held in PyTorch device memory ----------------------
def sph_alu_peak(precision: int, target_ms: float, stream: int = 0):
    """Measured fused multiply-add throughput (TFLOP/s, launch ms) of the
    current device: FP32 for PREC_MIXED, FP64 for PREC_FP64."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    check(lib().sph_alu_peak(int(precision), float(target_ms), C.byref(tf), C.byref(ms), C.c_void_p(stream)),
          "sph_alu_peak")
    return tf.value, ms.value


def make_params(precision: int = PREC_MIXED, **kw) -> Params:
    """sph_params from keyword arguments (names as in sph_params; 'eos' may be
    'adiabatic'/'isothermal'; box tuples accepted)."""
    p = sph_params_default()
    p.precision = precision
    for k, v in kw.items():
        if k == "eos":
            p.eos = EOS_ISOTHERMAL if v in ("isothermal", 1) else EOS_ADIABATIC
        elif k in ("box_lo", "box_len"):
            setattr(p, k, (C.c_double * 3)(*v))
        elif k == "periodic":
            p.periodic = int(bool(v))
        else:
            setattr(p, k, v)
    return p


class Problem:
    """One SPH problem: FP64 state tensors and the workspace on the GPU, and
    the library context that points at them."""

    def __init__(self, arrays: dict, params: Params, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.n = n = len(arrays["x"])
        self.params = params
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.t = {}
        for f in STATE_FIELDS:
            a = arrays.get(f)
            if a is not None:
                self.t[f] = torch.as_tensor(a, dtype=torch.float64).to(self.device).contiguous()
            else:
                self.t[f] = torch.zeros(max(n, 1), dtype=torch.float64, device=self.device)
        if params.av_switch and arrays.get("alpha") is None:
            self.t["alpha"].fill_(params.alpha_av)  # the switch starts from the full viscosity
        self.state = State(**{f: self.t[f].data_ptr() for f in STATE_FIELDS})
        self.ws_bytes = sph_workspace_bytes(n, params)
        if self.ws_bytes == 0:
            raise SPHError(EINVAL, "sph_workspace_bytes")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        rc, self.ctx = sph_setup(params, n, self.state, self.ws.data_ptr(), self.ws_bytes, self.stream.cuda_stream)
        check(rc, "sph_setup")

    def density_h(self, allow=()):
        return check(sph_density_h(self.ctx), "sph_density_h", allow)

    def forces(self, allow=()):
        return check(sph_forces(self.ctx), "sph_forces", allow)

    def step(self, dt: float = -1.0, allow=()):
        rc, used = sph_step(self.ctx, dt)
        check(rc, "sph_step", allow)
        return used

    def run(self, nsteps: int, allow=()):
        return check(sph_run(self.ctx, nsteps), "sph_run", allow)

    def block_step(self, allow=()):
        """One hierarchical block step (needs block_levels > 0 in the
        params): returns (Delta t_MAX, particle force evaluations)."""
        rc, dtmax, evals = sph_block_step(self.ctx)
        check(rc, "sph_block_step", allow)
        return dtmax, evals

    def block_prepare(self):
        """Capture the block step's graph ahead of the first block step."""
        check(sph_block_prepare(self.ctx), "sph_block_prepare")

    def levels(self):
        """Each particle's time-step level (numpy int32, caller's order)."""
        torch = self.torch
        lv = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        check(sph_block_levels(self.ctx, lv.data_ptr()), "sph_block_levels")
        return lv.cpu().numpy()

    def sync(self, allow=()):
        return check(sph_sync(self.ctx), "sph_sync", allow)

    def diagnostics(self) -> Diag:
        return sph_diagnostics(self.ctx)

    def neighbours(self, kind: int, h=None):
        """CSR (offsets, idx) as int64/int32 tensors on the device."""
        torch = self.torch
        off = torch.zeros(self.n + 1, dtype=torch.int64, device=self.device)
        hp = 0
        if h is not None:
            ht = torch.as_tensor(h, dtype=torch.float64).to(self.device).contiguous()
            hp = ht.data_ptr()
        cap = max(1, self.n * 96)
        while True:
            idx = torch.zeros(cap, dtype=torch.int32, device=self.device)
            rc, tot = sph_neighbours(self.ctx, kind, hp, off.data_ptr(), idx.data_ptr(), cap)
            if rc == ENOSPACE and tot > cap:
                cap = int(tot)
                continue
            check(rc, "sph_neighbours")
            return off, idx[:tot]

    def numpy(self, *fields):
        self.stream.synchronize()
        return {f: self.t[f][:self.n].cpu().numpy() for f in (fields or STATE_FIELDS)}

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            sph_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
