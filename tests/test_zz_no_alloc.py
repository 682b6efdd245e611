"""ecmg_error_norms_noalloc: the error norms for callers that may not allocate device memory
(for example code inside a latency-critical loop or under a framework that owns every device
allocation, where the device-wide synchronisation of cudaMalloc/cudaFree is not allowed).

Its scratch is a fixed array inside the library, so this file checks it through the C ABI
against the handle-based ecmg_error_norms on the same vectors, twice in a row (the second
call reuses the array the first one left behind), and against the oracle's norms and numpy
on lengths that do not fill its blocks. The file name makes pytest collect it last; it also
passes when run alone in a fresh process.
"""
import ctypes
import math

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


def _noalloc(E, a, b, n=None):
    import torch
    mx, rms = ctypes.c_double(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = E.ecmg_error_norms_noalloc(ctypes.c_void_p(a.data_ptr()), None if b is None else ctypes.c_void_p(b.data_ptr()),
                                    a.numel() if n is None else n, stream, ctypes.byref(mx), ctypes.byref(rms))
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
        # and both against torch's own max and mean of the same difference
        assert mx == (U - ue).abs().max().item()
        assert rms == pytest.approx(math.sqrt(((U - ue) ** 2).mean().item()), rel=1e-12)
        st, mx, rms = _noalloc(E, U, None)
        assert st == E.ECMG_OK
        assert mx == ref_one[0]
        assert rms == pytest.approx(ref_one[1], rel=1e-12)
        assert mx == U.abs().max().item()
        assert rms == pytest.approx(math.sqrt((U ** 2).mean().item()), rel=1e-12)
    s.close()


@pytest.mark.parametrize("n", [1, 255, 16383, 16384, 16385, 3 * 16384 + 17, 1_000_003])
def test_noalloc_norms_match_oracle_for_lengths_that_do_not_fill_a_block(E, oracle_mod, n):
    import torch
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) * 3.0
    b = rng.standard_normal(n)
    ta, tb = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    for bb, tbb in ((b, tb), (None, None)):
        want = oracle_mod.norms(a, bb)
        st, mx, rms = _noalloc(E, ta, tbb)
        assert st == E.ECMG_OK
        assert mx == want[0]
        assert rms == pytest.approx(want[1], rel=1e-12)


def test_noalloc_norms_of_a_vector_of_the_512_cube_size(E):
    """513^3 values, the nodes of the finest level of the 512^3 workload, against numpy."""
    import torch
    n = 513 ** 3
    g = torch.Generator(device="cuda")
    g.manual_seed(513)
    a = torch.rand(n, dtype=torch.float64, device="cuda", generator=g) - 0.5
    b = torch.rand(n, dtype=torch.float64, device="cuda", generator=g) - 0.5
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    d = an - bn
    st, mx, rms = _noalloc(E, a, b)
    assert st == E.ECMG_OK
    assert mx == np.abs(d).max()
    assert rms == pytest.approx(float(np.sqrt(np.mean(d * d))), rel=1e-12)


@pytest.mark.parametrize("where", [0, 40000, 99999])
def test_noalloc_a_nan_makes_both_norms_nan(E, where):
    import torch
    a = torch.linspace(-1.0, 1.0, 100000, dtype=torch.float64, device="cuda")
    a[where] = float("nan")
    b = torch.zeros_like(a)
    b[(where + 1) % a.numel()] = 1e300
    for args in ((a, None), (a, b), (b, a)):
        st, mx, rms = _noalloc(E, *args)
        assert st == E.ECMG_OK
        assert math.isnan(mx) and math.isnan(rms)
    # the next call on clean data is not affected by the NaN left in the scratch
    st, mx, rms = _noalloc(E, b, None)
    assert st == E.ECMG_OK and mx == 1e300


def test_noalloc_refuses_pageable_host_memory_and_accepts_pinned(E):
    import torch
    host = np.ones(1000)
    mx, rms = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    st = E.ecmg_error_norms_noalloc(ctypes.c_void_p(host.ctypes.data), None, host.size, None,
                                    ctypes.byref(mx), ctypes.byref(rms))
    assert st == E.ECMG_ERR_INVALID_ARG
    assert mx.value == -1.0 and rms.value == -1.0     # nothing was written
    dev = torch.zeros(1000, dtype=torch.float64, device="cuda")
    st = E.ecmg_error_norms_noalloc(ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(host.ctypes.data), host.size,
                                    None, ctypes.byref(mx), ctypes.byref(rms))
    assert st == E.ECMG_ERR_INVALID_ARG
    assert mx.value == -1.0 and rms.value == -1.0
    pinned = torch.full((1000,), -2.5, dtype=torch.float64).pin_memory()
    st, mx2, rms2 = _noalloc(E, pinned, dev)
    assert st == E.ECMG_OK and mx2 == 2.5 and rms2 == 2.5


def test_noalloc_rejects_sizes_beyond_its_scratch(E):
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    mx, rms = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    st = E.ecmg_error_norms_noalloc(ctypes.c_void_p(x.data_ptr()), None, E.ECMG_NOALLOC_MAX_ELEMS + 1, None,
                                    ctypes.byref(mx), ctypes.byref(rms))
    assert st == E.ECMG_ERR_INVALID_ARG
    assert mx.value == -1.0 and rms.value == -1.0     # nothing was written
