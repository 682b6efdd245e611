"""The C ABI library builds for sm_103a, loads, and exports every function include/ecmg.h
declares (no GPU needed: nothing is called that touches the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ecmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ecmg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1506_02983_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ecmg_create", "ecmg_solve", "ecmg_extrapolate", "ecmg_get_level", "ecmg_destroy",
              "ecmg_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1506_02983_gb300 import ecmg
    assert sorted(ecmg.EXPORTED) == _declared()


def test_host_side_validation_without_gpu(libpath):
    """Argument checks run before any CUDA call."""
    from paper_1506_02983_gb300 import ecmg
    p = ecmg.ecmg_problem()
    p.n0[:] = [2, 2, 2]
    p.levels = 2  # < 3
    p.lo[:] = [0, 0, 0]
    p.hi[:] = [1, 1, 1]
    o = ecmg.default_options()
    h = ctypes.c_void_p()
    assert ecmg.ecmg_create(ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    p.levels = 3
    p.beta = 16
    p.f = 16
    p.face_bc[:] = [1] * 6
    p.robin_alpha[:] = [0.0] * 6
    assert ecmg.ecmg_create(ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_SINGULAR
    p.face_bc[0] = 0
    o.rtol = 2.0
    assert ecmg.ecmg_create(ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    o.rtol = 1e-9
    nbytes = ctypes.c_uint64()
    assert ecmg.ecmg_workspace_bytes(ctypes.byref(p), ctypes.byref(o), ctypes.byref(nbytes)) == 0
    assert nbytes.value > 0
    assert b"singular" in ecmg.ecmg_status_string(ecmg.ECMG_ERR_SINGULAR)


def test_batched_validation_without_gpu(libpath):
    """ecmg_create_batched rejects bad batch sizes and non-MIXED precision before any CUDA call."""
    from paper_1506_02983_gb300 import ecmg
    arr = (ecmg.ecmg_problem * 2)()
    for p in arr:
        p.n0[:] = [2, 2, 2]
        p.levels = 3
        p.lo[:] = [0, 0, 0]
        p.hi[:] = [1, 1, 1]
        p.beta = 16
        p.f = 16
    o = ecmg.default_options(precision=ecmg.ECMG_MIXED)
    h = ctypes.c_void_p()
    assert ecmg.ecmg_create_batched(arr, 0, ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    assert ecmg.ecmg_create_batched(arr, 129, ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    o64 = ecmg.default_options(precision=ecmg.ECMG_FP64)
    assert ecmg.ecmg_create_batched(arr, 2, ctypes.byref(o64), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    arr[1].levels = 2
    assert ecmg.ecmg_create_batched(arr, 2, ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    assert ecmg.ecmg_solve_batched(None, None, None) == ecmg.ECMG_ERR_INVALID_ARG


def test_solver_variant_options_validation_without_gpu(libpath):
    """Preconditioner and schedule options are checked before any CUDA call."""
    from paper_1506_02983_gb300 import ecmg
    p = ecmg.ecmg_problem()
    p.n0[:] = [2, 2, 2]
    p.levels = 4
    p.lo[:] = [0, 0, 0]
    p.hi[:] = [1, 1, 1]
    p.beta = 16
    p.f = 16
    h = ctypes.c_void_p()
    for bad in (dict(preconditioner=2), dict(schedule=3), dict(schedule=1, sched_mL=0),
                dict(schedule=1, sched_beta=0.5), dict(schedule=1, sched_beta=65.0),
                dict(schedule=1, sched_mL=2000000, sched_beta=64.0)):
        o = ecmg.default_options(**bad)
        assert ecmg.ecmg_create(ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG, bad
    o = ecmg.default_options(cg_form=3)
    assert ecmg.ecmg_create(ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    # the batched entry point takes a bad step form as an invalid argument too
    o = ecmg.default_options(precision=ecmg.ECMG_MIXED, cg_form=3)
    assert ecmg.ecmg_create_batched(ctypes.byref(p), 1, ctypes.byref(o), None, ctypes.byref(h)) == \
        ecmg.ECMG_ERR_INVALID_ARG
    o = ecmg.default_options()
    assert o.preconditioner == ecmg.ECMG_PREC_JACOBI and o.schedule == ecmg.ECMG_SCHED_TOLERANCE
    assert o.sched_mL == 4 and o.sched_beta == 4.0 and o.inner_rtol == 1e-3
    assert o.cg_form == ecmg.ECMG_CG_AUTO


def test_compact_input_validation_without_gpu(libpath):
    """Separable f, separable g_D and beta_const are checked before any CUDA call; the batched
    entry point rejects them."""
    from paper_1506_02983_gb300 import ecmg

    def prob():
        p = ecmg.ecmg_problem()
        p.n0[:] = [2, 2, 2]
        p.levels = 3
        p.lo[:] = [0, 0, 0]
        p.hi[:] = [1, 1, 1]
        p.f = 16
        p.f_mode = ecmg.ECMG_F_SEPARABLE
        p.f_terms = 1
        p.beta_const = 1.0
        return p

    o = ecmg.default_options()
    h = ctypes.c_void_p()
    nbytes = ctypes.c_uint64()
    good = prob()
    assert ecmg.ecmg_workspace_bytes(ctypes.byref(good), ctypes.byref(o), ctypes.byref(nbytes)) == 0
    dense = prob()
    dense.f_mode, dense.beta = ecmg.ECMG_F_LOAD, 16
    dense_bytes = ctypes.c_uint64()
    assert ecmg.ecmg_workspace_bytes(ctypes.byref(dense), ctypes.byref(o), ctypes.byref(dense_bytes)) == 0
    assert nbytes.value > dense_bytes.value  # the 1D factor arrays of every level
    bad = []
    for field, value in (("beta_const", 0.0), ("beta_const", float("inf")), ("f_terms", 0), ("f_terms", 65),
                         ("g_R", 16), ("gD_terms", 1), ("gD_terms", -1), ("f_mode", 3)):
        p = prob()
        setattr(p, field, value)
        bad.append((field, value, p))
    for field, value, p in bad:
        assert ecmg.ecmg_create(ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG, (field, value)
    arr = (ecmg.ecmg_problem * 1)(prob())
    om = ecmg.default_options(precision=ecmg.ECMG_MIXED)
    assert ecmg.ecmg_create_batched(arr, 1, ctypes.byref(om), None, ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG


def test_problem_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of ecmg_problem and ecmg_options has the C layout (gcc on the header)."""
    import shutil
    import subprocess
    from paper_1506_02983_gb300 import ecmg
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    fields = {"ecmg_problem": [f[0] for f in ecmg.ecmg_problem._fields_],
              "ecmg_options": [f[0] for f in ecmg.ecmg_options._fields_]}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ecmg.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st, st))
        for n in names:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st, n, st, n))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for st, names in fields.items():
        cls = getattr(ecmg, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for n in names:
            assert int(got["%s.%s" % (st, n)]) == getattr(cls, n).offset, (st, n)


def test_create_with_allocator_validation_without_gpu(libpath):
    """alloc and free come together; the problem is validated before any allocation."""
    from paper_1506_02983_gb300 import ecmg
    p = ecmg.ecmg_problem()
    p.n0[:] = [2, 2, 2]
    p.levels = 3
    p.lo[:] = [0, 0, 0]
    p.hi[:] = [1, 1, 1]
    p.beta = 16
    p.f = 16
    o = ecmg.default_options()
    h = ctypes.c_void_p()
    calls = []
    alloc = ecmg.ALLOC_FN(lambda n, s, c: calls.append(n) or None)
    free = ecmg.FREE_FN(lambda ptr, n, s, c: calls.append(-n))
    assert ecmg.ecmg_create_with_allocator(ctypes.byref(p), ctypes.byref(o), None, alloc, ecmg.FREE_FN(), None,
                                           ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    p.levels = 2  # invalid: at least 3 levels
    assert ecmg.ecmg_create_with_allocator(ctypes.byref(p), ctypes.byref(o), None, alloc, free, None,
                                           ctypes.byref(h)) == ecmg.ECMG_ERR_INVALID_ARG
    assert calls == [] and not h.value


def test_binding_constants_match_the_header():
    """Every enum value and #define constant of include/ecmg.h that the binding names has the
    header's value."""
    import re
    from paper_1506_02983_gb300 import ecmg
    text = open(os.path.join(ROOT, "include", "ecmg.h")).read()
    consts = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", text):
        for name, val in re.findall(r"(ECMG_\w+)\s*=\s*(\d+)", body):
            consts[name] = int(val)
    for name, expr in re.findall(r"#define\s+(ECMG_\w+)\s+\(?([0-9 <<]+)\)?", text):
        consts[name] = eval(expr)
    named = {k: v for k, v in consts.items() if hasattr(ecmg, k)}
    assert len(named) >= 20, sorted(named)
    for k, v in named.items():
        assert getattr(ecmg, k) == v, (k, getattr(ecmg, k), v)


def test_workspace_of_the_step_forms_without_gpu(libpath):
    """Host logic of the MIXED step form: the single-pass form adds a second FP32 r and q on
    every level >= 2, ECMG_CG_AUTO only on the levels of fewer than 2^22 nodes, and both widen
    the per-block partials from 3 to 8 doubles (ecmg_workspace_bytes, no CUDA call)."""
    from paper_1506_02983_gb300 import ecmg
    p = ecmg.ecmg_problem()
    p.n0[:] = [8, 8, 8]
    p.levels = 7
    p.lo[:] = [0, 0, 0]
    p.hi[:] = [1, 1, 1]
    p.beta = 16
    p.f = 16

    def ws(form, ring_slots=0):
        o = ecmg.default_options(precision=ecmg.ECMG_MIXED, cg_form=form, ring_slots=ring_slots)
        n = ctypes.c_uint64()
        assert ecmg.ecmg_workspace_bytes(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == 0
        return n.value

    def total(l):  # padded nodes of level l (ghost layers and the 16-byte left pad)
        nx = 8 << l
        pitch = (nx + 1 + 4 + 2 + 7) // 8 * 8
        return pitch * (nx + 3) * (nx + 3)

    two, single, auto = ws(ecmg.ECMG_CG_TWO_PASS), ws(ecmg.ECMG_CG_SINGLE_PASS), ws(ecmg.ECMG_CG_AUTO)
    small = [l for l in range(2, 7) if ((8 << l) + 1) ** 3 < ecmg.ECMG_AUTO_SINGLE_PASS_NODES]
    assert small == [2, 3, 4]
    # the partials (3 -> 8 doubles per block) are the same for both forms that use them
    assert single - auto == sum(8 * total(l) for l in range(2, 7) if l not in small)
    extra = single - two - sum(8 * total(l) for l in range(2, 7))
    assert extra > 0 and extra % (5 * 8) == 0  # 5 more doubles per block of the largest grid
    # the ring of search directions: 4 bytes per stored node (slots 256-byte aligned) and 8 bytes
    # of alpha per slot on every two-pass level >= 2, nothing on single-pass levels
    def slot(l):
        return 4 * ((total(l) + 63) // 64 * 64) + 8

    for slots in (4, 34, 64):
        assert ws(ecmg.ECMG_CG_TWO_PASS, slots) - two == sum(slot(l) * slots for l in range(2, 7))
        assert ws(ecmg.ECMG_CG_AUTO, slots) - auto == sum(slot(l) * slots for l in (5, 6))
        assert ws(ecmg.ECMG_CG_SINGLE_PASS, slots) == single
    o = ecmg.default_options()
    assert o.ring_slots == ecmg.ECMG_RING_AUTO
    for bad in (1, 3, 65, -2):
        o = ecmg.default_options(precision=ecmg.ECMG_MIXED, ring_slots=bad)
        n = ctypes.c_uint64()
        assert ecmg.ecmg_workspace_bytes(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == \
            ecmg.ECMG_ERR_INVALID_ARG, bad


def test_binding_fails_loudly_without_the_library(tmp_path):
    """The binding has no fallback: imported from a tree where libecmg.so was never built, it
    raises ImportError instead of running anything on the CPU."""
    import importlib.util
    import shutil
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1506_02983_gb300", "ecmg.py"), pkg / "ecmg.py")
    spec = importlib.util.spec_from_file_location("ecmg_unbuilt", pkg / "ecmg.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError, match="no fallback"):
        spec.loader.exec_module(mod)


def test_ring_auto_resolves_to_none_without_a_device(libpath):
    """ECMG_RING_AUTO sizes the ring from the device's memory; with no device it keeps the
    correction vector (0 slots)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present (tests/test_gpu_ring.py covers the choice there)")
    from paper_1506_02983_gb300 import ecmg
    p = ecmg.ecmg_problem()
    p.n0[:] = [8, 8, 8]
    p.levels = 6
    p.lo[:] = [0, 0, 0]
    p.hi[:] = [1, 1, 1]
    p.beta = 16
    p.f = 16
    n = {}
    for slots in (ecmg.ECMG_RING_AUTO, 0):
        o = ecmg.default_options(precision=ecmg.ECMG_MIXED, cg_form=ecmg.ECMG_CG_TWO_PASS, ring_slots=slots)
        b = ctypes.c_uint64()
        assert ecmg.ecmg_workspace_bytes(ctypes.byref(p), ctypes.byref(o), ctypes.byref(b)) == 0
        n[slots] = b.value
    assert n[ecmg.ECMG_RING_AUTO] == n[0]
