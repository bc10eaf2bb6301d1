"""GPU parity of hierarchical block time-steps (Sec. 2.1.4) with the Saitoh &
Makino limiter against the FP64 oracle's block step: the same levels and
force evaluations (every decision is taken on integer levels from the same
step lengths), and the state after a block step within the norms of one
evaluation: mixed rho 1e-5 relative, a 1e-4 of rms |a|, v and u 1e-5 of
their largest magnitude; FP64 1e-12 relative.  Measured on the Sedov blast
of 16^3 (mixed / FP64, largest over the particles): after one block of 1
level (2 ticks) rho 3.4e-7 / 1.9e-14, a 7.0e-6 / 2.5e-13 of rms; after 5
levels (32 ticks) rho 3.4e-7 / 5.5e-14, a 6.8e-6 / 1.4e-12, v 2.8e-7 /
8.7e-14, u 9.9e-8 / 6.8e-14 -- the error does not grow with the ticks
beyond the FP64 force sums' 1e-12 (bounded at 1e-11 after 32 ticks)."""
import numpy as np
import pytest

from paper_1709_04488_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _oracle_block(O, a, p, L, dl=2, blocks=1):
    P = O.Params(**p, use_grid=True)
    s = O.State(**a)
    assert O.density(P, s) == O.OK and O.forces(P, s) == O.OK
    lv = np.zeros(s.n, np.int32)
    nm = np.zeros(s.n, np.int32)
    out = []
    for _ in range(blocks):
        rc, dtmax, passes, evals = O.block_step(P, s, lv, nm, L, dl)
        assert rc == O.OK
        out.append((dtmax, evals))
    return s, lv, out


def _gpu_block(S, a, p, prec, L, dl=2, blocks=1):
    prob = S.Problem(a, S.make_params(prec, **p, block_levels=L, block_gap=dl))
    prob.density_h()
    prob.forces()
    out = [prob.block_step() for _ in range(blocks)]
    return prob, out


def _scale_err(g, ref, f):
    r = getattr(ref, f)
    return np.max(np.abs(g[f] - r)) / max(np.max(np.abs(r)), 1e-300)


def _a_err(g, ref):
    ra = np.stack([ref.ax, ref.ay, ref.az], 1)
    ga = np.stack([g["ax"], g["ay"], g["az"]], 1)
    return np.max(np.linalg.norm(ga - ra, axis=1)) / np.sqrt(np.mean(np.sum(ra ** 2, 1)))


@pytest.mark.parametrize("prec,L", [("fp64", 1), ("mixed", 1), ("fp64", 5), ("mixed", 5)])
def test_sedov_block_step_matches_oracle(S, oracle_mod, prec, L):
    """One level (two ticks) and five levels (32 ticks) at the norms of one
    evaluation (FP64 forces after 32 ticks: 1e-11, see the module notes)."""
    O = oracle_mod
    a, p = ics.sedov(16)
    ref, lv_ref, oo = _oracle_block(O, a, p, L)
    fp64 = prec == "fp64"
    prob, go = _gpu_block(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, L)
    lv = prob.levels()
    assert np.array_equal(lv, lv_ref)
    assert go[0][0] == pytest.approx(oo[0][0], rel=1e-12 if fp64 else 1e-5)
    assert go[0][1] == oo[0][1]  # the same particle force evaluations
    if L == 5:
        assert lv.max() >= 3 and go[0][1] < len(a["x"]) * 2 ** L / 4
    g = prob.numpy()
    tol = 1e-12 if fp64 else 1e-5
    for f in ("vx", "vy", "vz", "u"):
        assert _scale_err(g, ref, f) < tol, f
    L_box = np.asarray(p["box_len"])
    for k, f in enumerate(("x", "y", "z")):
        d = np.abs(g[f] - getattr(ref, f))
        d = np.minimum(d, L_box[k] - d)
        assert np.max(d) < (1e-12 if fp64 else 1e-6), f
    assert np.max(np.abs(g["rho"] / ref.rho - 1.0)) < (1e-12 if fp64 else 1e-5)
    assert _a_err(g, ref) < ((1e-12 if L == 1 else 1e-11) if fp64 else 1e-4)


def test_block_step_with_tree_reuse_matches_oracle(S, oracle_mod):
    """Leaves kept and refitted between ticks (tree_rebuild_every = 4): the
    same neighbour sets, so the same levels and evaluations as the oracle."""
    O = oracle_mod
    a, p = ics.sedov(16)
    ref, lv_ref, oo = _oracle_block(O, a, p, 5)
    prob = S.Problem(a, S.make_params(S.PREC_FP64, **p, block_levels=5, tree_rebuild_every=4))
    prob.density_h()
    prob.forces()
    dtmax, evals = prob.block_step()
    assert np.array_equal(prob.levels(), lv_ref) and evals == oo[0][1]
    g = prob.numpy()
    for f in ("vx", "vy", "vz", "u"):
        assert _scale_err(g, ref, f) < 1e-10, f
    prob.step(-1.0)  # a global step after the block (it rebuilds the leaves)


def test_two_block_steps_and_limiter_history(S, oracle_mod):
    """The neighbours' largest levels carry from one block step to the next
    (the predictive limiter at the second block's start)."""
    O = oracle_mod
    a, p = ics.sedov(14, seed=5)
    ref, lv_ref, oo = _oracle_block(O, a, p, 4, blocks=2)
    prob, go = _gpu_block(S, a, p, S.PREC_FP64, 4, blocks=2)
    assert np.array_equal(prob.levels(), lv_ref)
    assert [e for _, e in go] == [e for _, e in oo]
    g = prob.numpy()
    for f in ("vx", "u"):
        assert _scale_err(g, ref, f) < 1e-9, f


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_m6_block_step_matches_oracle(S, oracle_mod, prec):
    """The M6 kernel (support 3h, eta = 1) in block steps: in mixed precision
    its tasks are up to 4 particles with 8 lanes each (the M4 kernel's take a
    whole warp per particle); the same levels and evaluations as the oracle
    and the state at the norms of one evaluation."""
    O = oracle_mod
    a, p = ics.sedov(14, seed=3)
    a["h"] = a["h"] / 1.2  # (the M6 lattice spacing guess)
    p = dict(p, kernel=1, eta=1.0)
    L = 4
    ref, lv_ref, oo = _oracle_block(O, a, p, L)
    fp64 = prec == "fp64"
    prob, go = _gpu_block(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, L)
    assert np.array_equal(prob.levels(), lv_ref)
    assert go[0][1] == oo[0][1] and go[0][1] < len(a["x"]) * 2 ** L
    g = prob.numpy()
    tol = 1e-12 if fp64 else 1e-5
    for f in ("vx", "vy", "vz", "u"):
        assert _scale_err(g, ref, f) < tol, f
    assert np.max(np.abs(g["rho"] / ref.rho - 1.0)) < tol
    assert _a_err(g, ref) < (1e-11 if fp64 else 1e-4)


def _gravity_block_case(n=3000, seed=93):
    a, p = ics.cloud(n, seed=seed)
    rng = np.random.default_rng(seed)
    a["m"] = a["m"] * rng.uniform(0.7, 1.3, n)
    return a, dict(p, gravity=1, G=3.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gravity_block_step_matches_oracle(S, oracle_mod, prec):
    """Self-gravity inside block steps: the acceleration condition enters the
    levels, the long-range sum and the zeta term follow the active set."""
    O = oracle_mod
    a, p = _gravity_block_case()
    L = 4
    ref, lv_ref, oo = _oracle_block(O, a, p, L)
    fp64 = prec == "fp64"
    prob, go = _gpu_block(S, a, p, S.PREC_FP64 if fp64 else S.PREC_MIXED, L)
    lv = prob.levels()
    assert np.array_equal(lv, lv_ref)
    assert go[0][1] == oo[0][1] and lv.max() > lv.min()
    g = prob.numpy()
    tol = 1e-10 if fp64 else 5e-4
    for f in ("vx", "vy", "vz"):
        assert _scale_err(g, ref, f) < tol, f
    for f in ("x", "y", "z"):
        assert np.max(np.abs(g[f] - getattr(ref, f))) < (1e-10 if fp64 else 1e-6), f


def _stepped(S, a, p, stream, blocks, **kw):
    prob = S.Problem(a, S.make_params(S.PREC_MIXED, **p, **kw), stream=stream)
    prob.density_h()
    prob.forces()
    if stream is not None:
        prob.block_prepare()  # the graph captured ahead of the first block
    out = [prob.block_step() for _ in range(blocks)]
    g = prob.numpy()
    g["levels"] = prob.levels()
    d = prob.diagnostics()
    prob.close()
    return out, g, d


@pytest.mark.parametrize("case", ["sedov", "sedov_reuse", "gravity"])
def test_graph_loop_equals_host_driven_ticks(S, case):
    """On a capturable stream the ticks of a block step run as the loop of
    one captured graph (a conditional while node; with tree reuse a
    conditional branch picks rebuild or refit), with no host round trip
    between them; on the legacy default stream the host reads the loop flag
    after every tick.  Both enqueue the same kernels in the same order, so
    two consecutive blocks (the second replays the graph) agree bit for
    bit: levels, evaluations, Delta t_MAX and the whole state."""
    import torch
    if case == "gravity":
        a, p = _gravity_block_case(2000, seed=95)
        kw = dict(block_levels=4)
    else:
        a, p = ics.sedov(14, seed=5)
        kw = dict(block_levels=5, tree_rebuild_every=3 if case == "sedov_reuse" else 1)
    host, gh, dh = _stepped(S, a, p, None, 2, **kw)
    graph, gg, dg = _stepped(S, a, p, torch.cuda.Stream(), 2, **kw)
    assert host == graph
    assert host[0][1] < len(a["x"]) * 2 ** kw["block_levels"]  # fewer evaluations than global steps
    assert dh.steps == dg.steps and dh.time == dg.time and dh.status == dg.status == S.OK
    for f in gh:
        assert np.array_equal(gh[f], gg[f]), f


def test_graph_loop_reports_a_failed_block(S):
    """A block that cannot start (four isolated particles: no finite
    positive time-step) ends on the device in both forms: the same error,
    and the clock does not advance."""
    import torch
    rng = np.random.default_rng(0)
    bad = {k: rng.uniform(0, 1, 4) for k in ("x", "y", "z")}
    bad.update(vx=np.zeros(4), vy=np.zeros(4), vz=np.zeros(4), u=np.ones(4), m=np.ones(4), h=np.full(4, 0.1))
    codes = []
    for stream in (None, torch.cuda.Stream()):
        prob = S.Problem(bad, S.make_params(S.PREC_MIXED, periodic=False, block_levels=3, flags=S.FLAG_ASYNC),
                         stream=stream)
        prob.density_h()
        prob.forces()
        prob.sync(allow=(S.ENOCONV,))
        rc, _, _ = S.sph_block_step(prob.ctx)
        codes.append(rc)
        assert prob.diagnostics().steps == 0 and prob.diagnostics().time == 0.0
        prob.close()
    assert codes[0] == codes[1] and codes[0] in (S.ENONFINITE, S.ENOCONV), codes


def test_block_step_rejections(S):
    import torch
    a, p = ics.lattice(6, seed=2)
    prob = S.Problem(a, S.make_params(S.PREC_MIXED, **p))
    prob.density_h()
    prob.forces()
    rc, _, _ = S.sph_block_step(prob.ctx)
    assert rc == S.EINVAL  # set up without block_levels
    b, q = ics.cloud(500, seed=3)
    assert S.sph_workspace_bytes(500, S.make_params(S.PREC_MIXED, **q, gravity=1, G=1.0, block_levels=3)) > 0
    assert S.sph_workspace_bytes(500, S.make_params(S.PREC_MIXED, **q, block_levels=21)) == 0
    assert S.sph_workspace_bytes(500, S.make_params(S.PREC_MIXED, **q, block_levels=3, block_gap=0)) == 0
