"""Autotuner for the launch shapes of the pair kernels (needs a GPU).

Two tables, both measured on the GPU it runs on:

``lanes``  lanes per particle (the leaf size is 32 / lanes) by problem size.
           For each size it times CFL steps at 1, 2, 4 and 8 lanes of a
           jittered lattice, a Sedov blast and (from 15552 particles) a Sod
           tube of about that size, scores each choice by the sum over the
           problems of its time relative to the problem's fastest, keeps the
           best, and writes ``tuning.json`` (rows ``[n_max, lanes]``, bucket
           edges at the geometric means of neighbouring sizes).  The binding
           installs the table (``sph_set_launch_table``) whenever it loads
           the library.

``build``  compile-time shapes of the pair kernels (staged candidates per
           chunk, list capacities, register budgets).  Coordinate descent:
           for each constant in turn it builds the library with each
           candidate value as a -D override, times the Sod-36864 and
           Sedov-1e6 steps in a fresh process, and keeps the value with the
           smallest sum of step times relative to the starting point.  The
           winners are written to ``csrc/sph_tuned.h``.

    python -m paper_1709_04488_gb300.autotune lanes [--steps K]
    python -m paper_1709_04488_gb300.autotune build [--workloads sod,sedov]
    python -m paper_1709_04488_gb300.autotune time --workload sod   (one timing)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
TUNED_H = os.path.join(HERE, "csrc", "sph_tuned.h")
TUNING_JSON = os.path.join(HERE, "tuning.json")

LANES = (1, 2, 4, 8)
LATTICE_SIDES = (12, 20, 33, 50, 80, 126)  # 1728 ... 2.0e6 particles (33: the Sod configuration's size)

# candidate values of the compile-time shapes, in the order they are tuned
BUILD_SPACE = {
    "SPH_FORCE_MINB": (4, 5, 6),
    "SPH_FORCE_MINB1": (4, 5, 6),
    "SPH_DENS_MINB": (3, 4, 5),
    "SPH_DENS_MINB1": (3, 4, 5),
    "SPH_FORCE_SB1": (4, 8, 16),
    "SPH_FORCE_LC1": (80, 96, 112),
    "SPH_DENS_LCAP1": (88, 96),
    "SPH_FORCE_CH": (32, 64, 128),
    "SPH_DENS_CH": (32, 64, 128),
    "SPH_FORCE_TAB": (64, 128),
}


def time_steps(arrays, params, steps=5, warmup=3, lanes=0):
    """Median device time (ms) of one CFL step of a problem, timed as the
    benchmark times it: the step replayed as a CUDA graph (sph_run), stage
    timing off, L2 flushed (a 256 MiB write) before every timed step."""
    import numpy as np
    import torch
    from . import sph as S
    st = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(st):
        prm = S.make_params(S.PREC_MIXED, lanes_per_particle=lanes, flags=S.FLAG_ASYNC, **params)
        prob = S.Problem(arrays, prm, stream=st)
        prob.density_h()
        prob.forces()
        prob.run(warmup)
        prob.sync()
        ts = []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            prob.run(1)
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        prob.sync()
        prob.close()
    return float(np.median(ts))


def _problems_of_size(side):
    """Problems of about side^3 particles: lattice, Sedov and (if large
    enough) a Sod tube with the bench configuration's resolution."""
    from . import ics
    from .serve import sod_request
    out = {"lattice": ics.lattice(side, seed=7), "sedov": ics.sedov(side, seed=8)}
    if side ** 3 >= 9 * 12 ** 3:
        out["sod"] = ics.sod() if side == 33 else sod_request(side ** 3, ratio=8.0)
    return out


def tune_lanes(steps=5):
    rows, measured = [], {}
    for side in LATTICE_SIDES:
        n = side ** 3
        score = {l: 0.0 for l in LANES}
        per = {}
        for kind, (a, p) in _problems_of_size(side).items():
            t = {l: time_steps(a, p, steps=steps, lanes=l) for l in LANES}
            per[kind] = {str(k): round(v, 4) for k, v in t.items()}
            fastest = min(t.values())
            for l in LANES:
                score[l] += t[l] / fastest
            print(f"n~{n:8d} {kind:8s} " + " ".join(f"{l}:{t[l]:.3f}ms" for l in LANES), flush=True)
        best = min(score, key=score.get)
        measured[str(n)] = {"ms": per, "score": {str(k): round(v, 4) for k, v in score.items()}, "best": best}
        rows.append((n, best))
        print(f"n~{n:8d} -> {best}", flush=True)
    table = []
    for k, (n, lanes) in enumerate(rows):
        if k + 1 < len(rows):
            edge = int(math.sqrt(n * rows[k + 1][0]))
        else:
            edge = 1 << 62
        if table and table[-1][1] == lanes:
            table[-1][0] = edge
        else:
            table.append([edge, lanes])
    out = {"lpp_table": table, "measured": measured,
           "note": "lattice, Sedov and Sod problems per size, median of CFL steps, mixed precision"}
    with open(TUNING_JSON, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", TUNING_JSON, table)
    return table


def _workload(name):
    from . import ics
    if name == "sod":
        return ics.sod()
    if name == "sedov":
        return ics.sedov()
    raise ValueError(name)


def _time_variant(flags, workloads, tmp):
    """Build the library with `flags` in `tmp` and time each workload in a
    fresh process (the build replaces no file of the package)."""
    from . import build as B
    tag = "_".join(f.split("=")[0][6:] + f.split("=")[1] for f in flags) or "base"
    out = os.path.join(tmp, tag, "libsph.so")
    B.build(extra=list(flags), out=out, build_dir=os.path.join(tmp, tag, "obj"))
    env = dict(os.environ, SPH_LIB_PATH=out, SPH_NO_TUNING="1")
    res = {}
    for w in workloads:
        r = subprocess.run([sys.executable, "-m", "paper_1709_04488_gb300.autotune", "time", "--workload", w],
                           capture_output=True, text=True, env=env, cwd=os.path.dirname(HERE))
        if r.returncode != 0:
            raise RuntimeError(f"timing {tag} {w} failed:\n{r.stderr[-2000:]}")
        res[w] = float(r.stdout.strip().splitlines()[-1])
    return res


def current_values():
    vals = {}
    with open(TUNED_H) as f:
        for m in re.finditer(r"#define (SPH_\w+) (\d+)", f.read()):
            vals[m.group(1)] = int(m.group(2))
    return vals


def write_tuned(vals):
    with open(TUNED_H) as f:
        text = f.read()
    for k, v in vals.items():
        text = re.sub(rf"#define {k} \d+", f"#define {k} {v}", text)
    with open(TUNED_H, "w") as f:
        f.write(text)


def tune_build(workloads=("sod", "sedov")):
    vals = current_values()
    with tempfile.TemporaryDirectory(prefix="sph_tune_") as tmp:
        base = _time_variant([f"-D{k}={v}" for k, v in vals.items()], workloads, tmp)
        print("start", vals, base, flush=True)
        for key, cands in BUILD_SPACE.items():
            scores = {}
            for c in cands:
                trial = dict(vals, **{key: c})
                t = _time_variant([f"-D{k}={v}" for k, v in trial.items()], workloads, tmp)
                scores[c] = sum(t[w] / base[w] for w in workloads)
                print(f"{key}={c}: " + " ".join(f"{w} {t[w]:.4f}ms" for w in workloads) + f" score {scores[c]:.4f}",
                      flush=True)
            vals[key] = min(scores, key=scores.get)
    write_tuned(vals)
    print("wrote", TUNED_H, vals)
    return vals


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["lanes", "build", "time"])
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--workloads", default="sod,sedov")
    ap.add_argument("--workload", default="sod")
    a = ap.parse_args(argv)
    if a.what == "lanes":
        tune_lanes(a.steps)
    elif a.what == "build":
        tune_build(tuple(a.workloads.split(",")))
    else:
        arrays, params = _workload(a.workload)
        print(time_steps(arrays, params, steps=a.steps))


if __name__ == "__main__":
    main()
