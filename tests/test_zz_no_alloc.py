"""The allocation-free entry point (sph_density_forces_noalloc) against the
regular path (sph_setup + sph_density_h + sph_forces with a caller-allocated
workspace), through the C ABI, on two calls in a row.

It exists for callers that must not create device allocations themselves
(for instance a host that keeps all device memory in its own pool); its
scratch memory is a fixed array inside the library, shared by every call.
This file is collected last so that a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

pytestmark = pytest.mark.gpu

FIELDS = ["x", "y", "z", "vx", "vy", "vz", "u", "m", "h", "rho", "omega", "P", "c",
          "ax", "ay", "az", "du", "vsig"]


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _inputs(seed, side=16):
    a, p = ics.lattice(side, seed=seed)
    rng = np.random.default_rng(seed + 7)
    for c in ("vx", "vy", "vz"):
        a[c] = rng.normal(0.0, 0.3, len(a["x"]))
    a["u"] = a["u"] * (1.0 + 0.2 * rng.uniform(-1, 1, len(a["x"])))
    return a, p


def _regular(S, a, prm):
    prob = S.Problem(a, prm)
    prob.density_h()
    prob.forces()
    out = prob.numpy()
    prob.close()
    return out


def _noalloc(S, a, prm):
    import torch
    n = len(a["x"])
    t = {}
    for f in FIELDS:
        v = a.get(f)
        t[f] = (torch.as_tensor(v, dtype=torch.float64).cuda().contiguous() if v is not None
                else torch.zeros(n, dtype=torch.float64, device="cuda"))
    st = S.State(**{f: t[f].data_ptr() for f in FIELDS})
    stream = torch.cuda.current_stream().cuda_stream
    S.check(S.sph_density_forces_noalloc(prm, n, st, stream), "sph_density_forces_noalloc")
    torch.cuda.synchronize()
    return {f: t[f].cpu().numpy() for f in FIELDS}


def _same(g, r):
    # the same kernels on the same inputs: identical bits, whichever memory
    # holds the scratch
    for f in ("h", "rho", "omega", "P", "c", "ax", "ay", "az", "du", "vsig"):
        assert np.array_equal(g[f], r[f]), f


def test_noalloc_matches_regular_path_twice(S):
    """Two calls in a row with different inputs: each matches the regular
    path, so nothing left in the shared scratch from the first call leaks
    into the second."""
    for seed in (3, 4):
        a, p = _inputs(seed)
        prm = S.make_params(S.PREC_MIXED, **p)
        _same(_noalloc(S, a, prm), _regular(S, a, prm))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_at_its_size_limit(S, prec):
    """32768 particles (the largest problem without self-gravity) in either
    precision, then a small call, both equal to the regular path."""
    pr = S.PREC_MIXED if prec == "mixed" else S.PREC_FP64
    for side, seed in ((32, 5), (12, 6)):
        a, p = _inputs(seed, side)
        prm = S.make_params(pr, **p)
        _same(_noalloc(S, a, prm), _regular(S, a, prm))


def test_noalloc_self_gravity(S):
    """An isolated self-gravitating cloud (direct sum and tree walk): the
    long-range sum's buffers also live in the fixed scratch."""
    a, p = ics.cloud(3000, seed=81)
    for theta in (0.0, 0.5):
        prm = S.make_params(S.PREC_MIXED, **p, gravity=1, G=1.0, grav_theta=theta)
        _same(_noalloc(S, a, prm), _regular(S, a, prm))


def test_noalloc_rejects_too_many_particles(S):
    import torch
    n = 32769
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = S.State(**{f: t.data_ptr() for f in FIELDS})
    rc = S.sph_density_forces_noalloc(S.make_params(S.PREC_MIXED), n, st, 0)
    assert rc == S.EINVAL
    assert "32768" in S.last_error()
