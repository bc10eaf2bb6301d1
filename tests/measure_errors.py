"""Measures the error of every result of the GPU path against the FP64 CPU
oracle, per configuration, and prints a table (the stated per-result errors
of the mixed-precision path and the plain FP64 path).  Needs a GPU.

    python tests/measure_errors.py [--large]

Configurations: the 16^3 jittered lattice with random velocities and u (one
density/h solve and force evaluation); the Sod tube of 36864 particles (the
first evaluation, then after 5 steps with the oracle's time-steps); with
--large, the Sedov blast (1e6) and the turbulent cloud (8e6) on 300 and 200
sampled particles.  Norms: rho, h, Omega, v_sig: max relative error; a:
max |delta a_i| / rms |a|; du/dt: max |delta du_i| / rms |du|; momentum
drift: |sum_i m_i a_i| / sum_i m_i |a_i| (per component, the largest);
dE/dt residual: |sum_i m_i (v_i . a_i + du_i)| / sum_i m_i (|v_i . a_i| +
|du_i|); energy change per step: relative change of the total energy over
one step, GPU minus oracle.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle as O  # noqa: E402
from paper_1709_04488_gb300 import ics  # noqa: E402
from paper_1709_04488_gb300 import sph as S  # noqa: E402


def errors(g, r, a, sel=None):
    full = sel is None
    sel = slice(None) if full else sel
    out = {}
    for f in ("rho", "h", "omega", "vsig"):
        out[f] = float(np.max(np.abs(g[f][sel] / getattr(r, f)[sel] - 1.0)))
    ga = np.stack([g["ax"], g["ay"], g["az"]], 1)[sel]
    ra = np.stack([r.ax, r.ay, r.az], 1)[sel]
    out["a"] = float(np.max(np.linalg.norm(ga - ra, axis=1)) / np.sqrt(np.mean(np.sum(ra ** 2, 1))))
    du = r.du[sel]
    out["du"] = float(np.max(np.abs(g["du"][sel] - du)) / np.sqrt(np.mean(du ** 2))) if np.any(du != 0) else 0.0
    if full:
        m = g["m"]
        ma = m[:, None] * np.stack([g["ax"], g["ay"], g["az"]], 1)
        out["momentum_drift"] = float(np.max(np.abs(ma.sum(0)) / np.abs(ma).sum(0)))
        va = a["vx"] * g["ax"] + a["vy"] * g["ay"] + a["vz"] * g["az"]
        den = float(np.sum(m * (np.abs(va) + np.abs(g["du"]))))
        out["dEdt_residual"] = float(abs(np.sum(m * (va + g["du"]))) / den) if den > 0 else 0.0
    return out


def energy(x, m, adi=True):
    e = 0.5 * np.sum(m * (x["vx"] ** 2 + x["vy"] ** 2 + x["vz"] ** 2))
    return e + (np.sum(m * x["u"]) if adi else 0.0)


def run(prec_name, large):
    prec = S.PREC_MIXED if prec_name == "mixed" else S.PREC_FP64
    rows = {}
    a, p = ics.lattice(16, seed=1)
    rng = np.random.default_rng(101)
    for c in ("vx", "vy", "vz"):
        a[c] = rng.normal(0.0, 0.3, len(a["x"]))
    a["u"] = a["u"] * (1.0 + 0.2 * rng.uniform(-1, 1, len(a["x"])))
    P = O.Params(**p)
    r = O.State(**a)
    assert O.density(P, r) == O.OK and O.forces(P, r) == O.OK
    prob = S.Problem(a, S.make_params(prec, **p))
    prob.density_h()
    prob.forces()
    rows["lattice 4096, one evaluation"] = errors(prob.numpy(), r, a)
    prob.close()
    a, p = ics.sod()
    P = O.Params(**p, use_grid=True)
    r = O.State(**a)
    assert O.density(P, r) == O.OK and O.forces(P, r) == O.OK
    prob = S.Problem(a, S.make_params(prec, **p))
    prob.density_h()
    prob.forces()
    rows["Sod 36864, first evaluation"] = errors(prob.numpy(), r, a)
    de = []
    for _ in range(5):
        g0 = prob.numpy()
        r0 = {f: getattr(r, f).copy() for f in ("vx", "vy", "vz", "u")}
        dt = O.cfl_dt(P, r)
        assert O.step(P, r, dt) == O.OK
        prob.step(dt)
        g1 = prob.numpy()
        eg = energy(g1, g1["m"]) / energy(g0, g0["m"]) - 1.0
        eo = energy({f: getattr(r, f) for f in ("vx", "vy", "vz", "u")}, r.m) / energy(r0, r.m) - 1.0
        de.append(abs(eg - eo))
    g = prob.numpy()
    # (the step's forces act on the predicted velocities, which the state
    # does not keep: the dE/dt balance is checked on single evaluations)
    rows["Sod 36864, after 5 steps"] = errors(g, r, {"vx": g["vx"], "vy": g["vy"], "vz": g["vz"]})
    rows["Sod 36864, after 5 steps"].pop("dEdt_residual")
    rows["Sod 36864, after 5 steps"]["energy_change_per_step"] = float(max(de))
    prob.close()
    if large and prec == S.PREC_MIXED:
        from test_gpu_fullsize import _sampled
        for name, (aa, pp), ns in (("Sedov 1e6, 300 sampled", ics.sedov(), 300),
                                   ("cloud 8e6, 200 sampled", ics.cloud(), 200)):
            rec = {}

            def grab(g, ref, samp):
                rec.update(errors(g, ref, None, samp))
            _sampled(S, O, aa, pp, ns, seed=41, check=grab)
            rows[name] = rec
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--large", action="store_true")
    args = ap.parse_args()
    O.build()
    out = {"mixed": run("mixed", args.large), "fp64": run("fp64", False)}
    print(json.dumps(out, indent=1))
    keys = ["rho", "h", "omega", "a", "du", "vsig", "momentum_drift", "dEdt_residual", "energy_change_per_step"]
    for prec, rows in out.items():
        print(f"\n{prec}\n| configuration | " + " | ".join(keys) + " |")
        print("|---|" + "---:|" * len(keys))
        for name, e in rows.items():
            print(f"| {name} | " + " | ".join(f"{e[k]:.1e}" if k in e else "—" for k in keys) + " |")


if __name__ == "__main__":
    main()
