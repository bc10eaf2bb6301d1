"""The stepped configurations against their analytic solutions, on the GPU.

- Sod shock tube, 36864 particles (Sec. 6.2), run to t = 0.2 with the CFL
  step (the last step shortened to end at 0.2): the L1 errors of rho, v_x
  and P against the exact Riemann solution, over the window where the
  periodic tube's solution is the single Riemann problem, must equal the
  FP64 CPU oracle's own L1 errors within 1 % (the oracle's values are
  stored in tests/golden/sod_t02_oracle_l1.json by the script beside them,
  which calls only the oracle).
- Sedov blast, 100^3 particles (Sec. 6.3), mixed precision, 200 CFL steps:
  the density peak sits at the similarity solution's front within 2 h (and
  within h), the peak density stays below the strong-shock jump 4, and a
  fresh density and force evaluation of the evolved state (strong h
  contrast, uneven neighbour counts) matches the oracle on sampled particles
  at the parity tolerances.
"""
import json
import os

import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _run_to(S, prob, T):
    """CFL steps until time T, the last one shortened to land on T."""
    t, steps = 0.0, 0
    while t < T * (1 - 1e-12):
        dt = min(prob.diagnostics().dt_next, T - t)
        prob.step(dt)
        t += dt
        steps += 1
    return t, steps


@pytest.mark.parametrize("prec,case", [("fp64", "plain"), ("mixed", "jittered"), ("fp64", "jittered")])
def test_sod_to_t02_matches_riemann_like_the_oracle(S, prec, case):
    """The configuration as stated (perfect lattices) in FP64; in mixed
    precision (and FP64 again) with every particle moved by up to 1e-3 of its
    lattice spacing: on perfect lattices the L1 at t = 0.2 depends on how
    the lattices' symmetry breaks as they relax, which FP32 rounding would
    decide (a 1e-7 perturbation of the oracle's positions lowers its L1 by a
    third); the jitter sets it in the inputs for both."""
    from oracle import riemann
    ref = json.load(open(os.path.join(HERE, "golden", "sod_t02_oracle_l1.json")))[case]
    a, p = ics.sod(jitter=ref["jitter"], seed=ref["seed"]) if case == "jittered" else ics.sod()
    pr = S.PREC_MIXED if prec == "mixed" else S.PREC_FP64
    prob = S.Problem(a, S.make_params(pr, **p))
    prob.density_h()
    prob.forces()
    t, steps = _run_to(S, prob, 0.2)
    g = prob.numpy("x", "vx", "rho", "P", "h")
    d = prob.diagnostics()
    prob.close()
    assert d.status == S.OK
    assert abs(t - 0.2) < 1e-12
    l1 = riemann.sod_l1(g["x"], g["rho"], g["vx"], g["P"], 0.2, ref["hmax_window"])
    assert abs(l1[3] - ref["particles_in_window"]) <= 0.002 * ref["particles_in_window"]
    for k, name in enumerate(("l1_rho", "l1_vx", "l1_P")):
        assert abs(l1[k] / ref[name] - 1.0) < 0.01, (name, l1[k], ref[name])
    # the step count follows the same CFL condition
    assert abs(steps - ref["steps"]) <= max(2, 0.01 * ref["steps"])


def test_sedov_200_steps_follows_the_similarity_solution(S, oracle_mod):
    from oracle import sedov
    from test_gpu_fullsize import _sampled
    a, p = ics.sedov()
    prob = S.Problem(a, S.make_params(S.PREC_MIXED, **p))
    prob.density_h()
    prob.forces()
    prob.run(200)
    d = prob.diagnostics()
    assert d.status == S.OK and d.steps == 200
    g = prob.numpy()
    prob.close()
    r = np.sqrt((g["x"] - 0.5) ** 2 + (g["y"] - 0.5) ** 2 + (g["z"] - 0.5) ** 2)
    top = np.argsort(g["rho"])[-500:]  # (the shell behind the front holds ~10^3 particles)
    Rs, h = float(np.median(r[top])), float(np.median(g["h"][top]))
    R_an = sedov.shock_radius(d.time)
    assert abs(Rs - R_an) < 2.0 * h
    assert abs(Rs - R_an) < 1.0 * h
    assert g["rho"].max() < 4.0
    # energy is conserved by the global steps to the KDK scheme's accuracy
    E0 = float(np.sum(a["m"] * a["u"]))
    E1 = float(np.sum(g["m"] * (g["u"] + 0.5 * (g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2))))
    assert abs(E1 / E0 - 1.0) < 2e-3
    # the evolved state, evaluated afresh, against the oracle on a sample
    evolved = {f: g[f] for f in ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h")}
    _sampled(S, oracle_mod, evolved, p, 300, seed=37)
