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
    o = ecmg.default_options()
    assert o.preconditioner == ecmg.ECMG_PREC_JACOBI and o.schedule == ecmg.ECMG_SCHED_TOLERANCE
    assert o.sched_mL == 4 and o.sched_beta == 4.0 and o.inner_rtol == 1e-3
