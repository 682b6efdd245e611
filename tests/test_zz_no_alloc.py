"""ecmg_error_norms_noalloc: the error norms for callers that may not allocate device memory
(for example code inside a latency-critical loop or under a framework that owns every device
allocation, where the device-wide synchronisation of cudaMalloc/cudaFree is not allowed).

Its scratch is a fixed array inside the library, so this file checks it through the C ABI
against the handle-based ecmg_error_norms on the same vectors, twice in a row (the second
call reuses the array the first one left behind). The file name makes pytest collect it
last; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_02983_gb300 import build
    build.build()
    from paper_1506_02983_gb300 import ecmg
    return ecmg


def _noalloc(E, a, b):
    import torch
    mx, rms = ctypes.c_double(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = E.ecmg_error_norms_noalloc(ctypes.c_void_p(a.data_ptr()), None if b is None else ctypes.c_void_p(b.data_ptr()),
                                    a.numel(), stream, ctypes.byref(mx), ctypes.byref(rms))
    return st, mx.value, rms.value


def test_noalloc_norms_match_handle_norms_on_two_calls(E):
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    s = E.solver_from_problem(p)
    s.solve()
    U = s.get(E.ECMG_VEC_U)
    ue = torch.tensor(np.asarray(p["u_exact"]), device="cuda")
    ref_diff = s.norms(U, ue)
    ref_one = s.norms(U)
    for _ in range(2):
        st, mx, rms = _noalloc(E, U, ue)
        assert st == E.ECMG_OK
        assert mx == ref_diff[0]                      # a max does not depend on the order
        assert rms == pytest.approx(ref_diff[1], rel=1e-12)
        st, mx, rms = _noalloc(E, U, None)
        assert st == E.ECMG_OK
        assert mx == ref_one[0]
        assert rms == pytest.approx(ref_one[1], rel=1e-12)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(E):
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    mx, rms = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    st = E.ecmg_error_norms_noalloc(ctypes.c_void_p(x.data_ptr()), None, E.ECMG_NOALLOC_MAX_ELEMS + 1, None,
                                    ctypes.byref(mx), ctypes.byref(rms))
    assert st == E.ECMG_ERR_INVALID_ARG
    assert mx.value == -1.0 and rms.value == -1.0     # nothing was written
