"""C-ABI services around the solve, on the GPU: per-level device times in ecmg_stats, and the
workspace taken from a caller-supplied allocator (PyTorch's caching allocator)."""
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


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_level_seconds_add_up_to_the_solve(E, precision, use_graph):
    import torch
    p = inputs.cos_cube(levels=5, n0=(4, 4, 4), rtol=1e-10)
    s = E.solver_from_problem(p, precision=precision, use_graph=use_graph)
    s.solve()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st, status = s.solve()
    e1.record()
    torch.cuda.synchronize()
    assert status == 0
    total = e0.elapsed_time(e1) * 1e-3
    assert st["setup_seconds"] > 0 and all(t > 0 for t in st["seconds"]), st["seconds"]
    inside = st["setup_seconds"] + sum(st["seconds"])
    assert inside <= total * 1.02 + 1e-5, (inside, total)
    if use_graph:
        assert inside >= 0.5 * total, (inside, total)
    # a solve from level 2 times levels 2.. only
    st2 = s.solve_from(2)
    assert st2["setup_seconds"] == 0 and st2["seconds"][:2] == [0.0, 0.0] and all(t > 0 for t in st2["seconds"][2:])
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_workspace_from_the_torch_caching_allocator(E, precision):
    """Every device block of the handle comes from PyTorch's allocator (its statistics grow by at
    least ecmg_workspace_bytes) and goes back at destroy; the solve is the same bit for bit."""
    import ctypes
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    ref = E.solver_from_problem(p, precision=precision)
    st_ref, _ = ref.solve()
    U_ref = ref.get(E.ECMG_VEC_U).cpu().numpy()
    ref.close()
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64).contiguous().cuda()
    beta, f, gD = t(p["beta"]), t(p["f"]), t(p["gD"])
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], beta, f, gD, None,
                 rtol=1e-10, precision=precision, torch_memory=True)
    grown = torch.cuda.memory_allocated() - before
    nbytes = ctypes.c_uint64()
    assert E.ecmg_workspace_bytes(ctypes.byref(s.problem), ctypes.byref(s.options), ctypes.byref(nbytes)) == 0
    assert grown >= nbytes.value * 0.85, (grown, nbytes.value)  # the estimate rounds up
    st, status = s.solve()
    assert status == 0 and st["iters"] == st_ref["iters"]
    assert np.array_equal(s.get(E.ECMG_VEC_U).cpu().numpy(), U_ref)
    s.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


@pytest.mark.parametrize("use_graph", [1, 0])
def test_output_array_changes_between_solves(E, use_graph):
    """The copy of the solution into the caller's array is part of the recorded solve and reads
    the array's address on the device at each launch: one graph writes a new array each time,
    and a solve without an output array writes none."""
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    s = E.solver_from_problem(p, precision=1, use_graph=use_graph)
    a = torch.full(s.level_shape(), -1.0, dtype=torch.float64, device="cuda")
    b = torch.full(s.level_shape(), -2.0, dtype=torch.float64, device="cuda")
    s.solve(a)
    want = a.clone()
    assert not torch.equal(want, torch.full_like(want, -1.0))
    s.solve(b)
    assert torch.equal(b, want)
    a.fill_(-3.0)
    b.fill_(-4.0)
    s.solve()
    assert torch.equal(a, torch.full_like(a, -3.0)) and torch.equal(b, torch.full_like(b, -4.0))
    s.solve(a)
    assert torch.equal(a, want)
    # the finest level's U, in the dense layout, is what the array receives
    U = s.get(E.ECMG_VEC_U, -1)
    assert torch.equal(U.reshape(-1), want.reshape(-1))
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_host_inputs_and_output(E, precision):
    """Inputs in page-locked host memory are read, and the solution written, by the kernels
    directly; the solve is the same bit for bit as with device arrays. Pageable host memory is
    refused before any kernel runs."""
    import ctypes
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    ref = E.solver_from_problem(p, precision=precision)
    u_dev = torch.empty(ref.level_shape(), dtype=torch.float64, device="cuda")
    st_ref, _ = ref.solve(u_dev)
    ref.close()
    pin = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64).contiguous().pin_memory()
    beta, f, gD = pin(p["beta"]), pin(p["f"]), pin(p["gD"])
    s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], beta, f, gD, None,
                 rtol=1e-10, precision=precision)
    u_host = torch.empty(s.level_shape(), dtype=torch.float64).pin_memory()
    st, status = s.solve(u_host)
    assert status == 0 and st["iters"] == st_ref["iters"]
    assert torch.equal(u_host, u_dev.cpu())
    # pageable host memory: refused, no kernel launched, the handle stays usable
    pageable = torch.empty(s.level_shape(), dtype=torch.float64)
    st2 = E.ecmg_stats()
    assert E.ecmg_solve(s.handle, ctypes.c_void_p(pageable.data_ptr()), ctypes.byref(st2)) == E.ECMG_ERR_INVALID_ARG
    st3, status = s.solve(u_host)
    assert status == 0 and torch.equal(u_host, u_dev.cpu())
    s.close()
    # and at create
    bad = torch.as_tensor(np.asarray(p["f"]), dtype=torch.float64).contiguous()
    pr = E.ecmg_problem()
    pr.n0[:] = p["n0"]
    pr.levels = p["levels"]
    pr.lo[:] = p["lo"]
    pr.hi[:] = p["hi"]
    pr.face_bc[:] = p["face_bc"]
    pr.robin_alpha[:] = p["alpha"]
    pr.beta, pr.f, pr.g_D = beta.data_ptr(), bad.data_ptr(), gD.data_ptr()
    o = E.default_options(rtol=1e-10)
    h = ctypes.c_void_p()
    assert E.ecmg_create(ctypes.byref(pr), ctypes.byref(o), None, ctypes.byref(h)) == E.ECMG_ERR_INVALID_ARG
