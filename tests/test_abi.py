"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point include/sph.h declares, validates
parameters and sizes workspaces without touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    from paper_1709_04488_gb300 import build as b
    b.build()
    from paper_1709_04488_gb300 import sph
    return sph


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(S):
    lib = S.lib()
    names = _declared("sph.h")
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(S, tmp_path):
    """The ctypes mirrors of the public structs have the C layout (compiled
    with gcc against include/sph.h)."""
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sph.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(sph_params),sizeof(sph_state),sizeof(sph_diag),sizeof(sph_server_cfg),"
        "sizeof(sph_request),sizeof(sph_result),offsetof(sph_params,flags),offsetof(sph_diag,status),"
        "offsetof(sph_params,tree_rebuild_every),offsetof(sph_params,ac_signal),offsetof(sph_params,av_decay),"
        "offsetof(sph_state,dalpha));return 0;}\n")
    exe = tmp_path / "sizes"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(S.Params), C.sizeof(S.State), C.sizeof(S.Diag), C.sizeof(S.ServerCfg),
            C.sizeof(S.Request), C.sizeof(S.Result), S.Params.flags.offset, S.Diag.status.offset,
            S.Params.tree_rebuild_every.offset, S.Params.ac_signal.offset, S.Params.av_decay.offset,
            S.State.dalpha.offset]
    assert got == want


def test_defaults_are_the_papers(S):
    p = S.sph_params_default()
    assert p.eta == 1.2 and p.alpha_av == 1.0 and p.beta_av == 2.0 and p.c_cfl == 0.2
    assert p.kernel == S.KERNEL_M4


def test_constants_match_header(S):
    txt = open(os.path.join(ROOT, "include", "sph.h")).read()
    defs = dict(re.findall(r"#define (SPH_[A-Z0-9_]+)\s+(-?\d+)u?\b", txt))
    for name in ("KERNEL_M4", "KERNEL_M6", "AC_WADSLEY", "AC_PRICE", "AV_CONSTANT", "AV_MORRIS_MONAGHAN", "EOS_ADIABATIC", "EOS_ISOTHERMAL", "PREC_FP64", "PREC_MIXED",
                 "FLAG_ASYNC", "FLAG_TIMING"):
        assert int(defs["SPH_" + name]) == getattr(S, name), name


def test_workspace_bytes_and_validation(S):
    p = S.sph_params_default()
    w1 = S.sph_workspace_bytes(1000, p)
    w2 = S.sph_workspace_bytes(100000, p)
    assert 0 < w1 < w2
    assert w2 / 100000 < 600  # bytes per particle of scratch
    assert S.sph_workspace_bytes(-1, p) == 0
    bad = S.sph_params_default()
    bad.eta = -1.0
    assert S.sph_workspace_bytes(10, bad) == 0
    m6 = S.sph_params_default()
    m6.kernel = S.KERNEL_M6
    assert S.sph_workspace_bytes(1000, m6) > 0
    bad = S.sph_params_default()
    bad.kernel = 2
    assert S.sph_workspace_bytes(10, bad) == 0
    bad = S.sph_params_default()
    bad.ac_signal = 2
    assert S.sph_workspace_bytes(10, bad) == 0
    sw = S.sph_params_default()
    sw.av_switch = S.AV_MORRIS_MONAGHAN
    assert sw.alpha_min == 0.1 and sw.av_decay == 0.1
    assert S.sph_workspace_bytes(10, sw) > 0
    sw.alpha_min = 2.0  # above alpha_av
    assert S.sph_workspace_bytes(10, sw) == 0
    bad = S.sph_params_default()
    bad.lanes_per_particle = 3
    assert S.sph_workspace_bytes(10, bad) == 0


def test_gravity_and_block_step_parameters(S):
    """Defaults (direct summation, c_grav 0.5, no block steps, gap 2) and the
    host-side validation of the self-gravity and block-step parameters; the
    workspace grows by the tree walk's and the block steps' arrays."""
    p = S.sph_params_default()
    assert p.gravity == 0 and p.grav_theta == 0.0 and p.c_grav == 0.5
    assert p.block_levels == 0 and p.block_gap == 2

    def iso(**kw):
        q = S.make_params(S.PREC_MIXED, periodic=False, **kw)
        return S.sph_workspace_bytes(20000, q)

    direct = iso(gravity=1, G=1.0)
    tree = iso(gravity=1, G=1.0, grav_theta=0.5)
    assert 0 < direct and 0 < tree and tree != direct
    assert iso(gravity=1, G=0.0) == 0
    assert iso(gravity=1, G=1.0, grav_theta=1.01) == 0
    assert iso(gravity=1, G=1.0, grav_theta=-0.5) == 0
    assert iso(gravity=1, G=1.0, c_grav=0.0) == 0
    assert iso(gravity=1, G=1.0, kernel=S.KERNEL_M6) == 0
    assert S.sph_workspace_bytes(20000, S.make_params(S.PREC_MIXED, gravity=1, G=1.0)) == 0  # periodic
    plain = iso()
    blk = iso(block_levels=6)
    assert blk > plain
    assert iso(block_levels=21) == 0 and iso(block_levels=-1) == 0
    assert iso(block_levels=4, block_gap=0) == 0
    assert iso(block_levels=4, gravity=1, G=1.0, grav_theta=0.5) > 0


def test_setup_rejects_bad_arguments_without_a_gpu(S):
    p = S.sph_params_default()
    st = S.State()
    rc, ctx = S.sph_setup(p, 10, st, 0, 0, 0)
    assert rc in (S.EINVAL, S.ENOSPACE)
    assert S.last_error() != ""
    p.gamma = 1.0
    rc, ctx = S.sph_setup(p, 10, st, 0, 0, 0)
    assert rc == S.EINVAL


def test_launch_table_validation(S):
    """sph_set_launch_table accepts increasing rows of 1/2/4/8 lanes and
    rejects the rest without changing the installed table."""
    lib = S.lib()

    def call(rows):
        n = len(rows)
        nm = (C.c_int64 * max(n, 1))(*[r[0] for r in rows])
        ln = (C.c_int32 * max(n, 1))(*[r[1] for r in rows])
        return lib.sph_set_launch_table(nm, ln, n)

    assert call([(1000, 8), (100000, 4), (1 << 40, 1)]) == S.OK
    assert call([(1000, 3)]) == S.EINVAL
    assert call([(1000, 4), (1000, 2)]) == S.EINVAL
    assert call([(k + 1, 4) for k in range(33)]) == S.EINVAL
    assert lib.sph_set_launch_table(None, None, 1) == S.EINVAL
    assert call([]) == S.OK  # back to the built-in rule
    if os.path.exists(S.TUNING_PATH):  # the autotuned table the binding installs
        import json
        rows = json.load(open(S.TUNING_PATH))["lpp_table"]
        assert call(rows) == S.OK


def test_noalloc_limits_per_option_without_a_gpu(S):
    """The allocation-free entry point rejects, before touching the device,
    n > 32768 with SPH_EINVAL; at n = 32768 every option's layout (either
    precision, either kernel, either viscosity switch, self-gravity by
    direct sum or tree walk) fits its fixed scratch, so the call passes the
    size checks and stops at the NULL state arrays."""
    import ctypes as C
    st = S.State()  # NULL arrays: a call that passes the size checks stops at SPH_EINVAL

    def call(n, prec, **kw):
        p = S.make_params(prec, **kw)
        return S.lib().sph_density_forces_noalloc(C.byref(p), n, C.byref(st), None)

    assert call(32769, S.PREC_MIXED) == S.EINVAL and "32768" in S.last_error()
    grav = dict(periodic=False, gravity=1, G=1.0)
    for prec in (S.PREC_MIXED, S.PREC_FP64):
        for kw in (dict(), dict(kernel=S.KERNEL_M6, eta=1.0), dict(av_switch=2), grav, dict(grav, grav_theta=0.5)):
            assert call(32768, prec, **kw) == S.EINVAL and "NULL" in S.last_error(), (prec, kw)


def test_cullen_dehnen_switch_parameters(S):
    """av_switch = 2 (Cullen & Dehnen) is accepted with alpha_av > 0 and
    av_decay > 0, and refused with block time-steps or an unknown value."""
    def ws(**kw):
        return S.sph_workspace_bytes(4096, S.make_params(S.PREC_MIXED, **kw))
    assert S.AV_CULLEN_DEHNEN == 2
    assert ws(av_switch=2) > 0
    assert ws(av_switch=2, av_decay=0.0) == 0
    assert ws(av_switch=2, alpha_av=0.0) == 0
    assert ws(av_switch=2, block_levels=3) == 0
    assert ws(av_switch=3) == 0
