"""Batched solves (ecmg_create_batched) through the C ABI against the FP64 oracle, problem by
problem: the MIXED bar of the single-problem tests (true relative residual <= rtol on every
level >= 2, solution and extrapolations within 1e-7 relative of the oracle's, discretisation
error within 1 % where the exact solution is known)."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_02983_gb300 import build
    build.build()
    from paper_1506_02983_gb300 import ecmg
    return ecmg


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _device(p):
    import torch
    q = dict(p)
    for k in ("beta", "f", "gD", "gR"):
        v = p.get(k)
        q[k] = None if v is None else torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64).cuda()
    return q


def _mixed_batch():
    """Different sizes, level counts, boundary types, Robin faces, load modes and coefficients."""
    return [
        inputs.exp_cube(levels=4, rtol=RTOL),
        inputs.random_problem(0, n0=(2, 3, 2), levels=4, rtol=RTOL),
        inputs.random_problem(1, n0=(3, 2, 2), levels=3, rtol=RTOL),
        inputs.paper_problem1(levels=4, rtol=RTOL),
        inputs.variable_box(levels=3, n0=(2, 2, 4), rtol=RTOL),
        inputs.random_problem(7, n0=(2, 3, 2), levels=4, rtol=RTOL, contrast=1.0, face_bc=[1, 0, 1, 0, 1, 1],
                              alpha=[0.5, 0.0, 2.0, 0.0, 0.0, 1.0]),
        inputs.random_problem(11, n0=(5, 3, 4), levels=4, rtol=RTOL, face_bc=[1, 0, 0, 1, 1, 0],
                              alpha=[0.5, 0.0, 0.0, 2.0, 1.0, 0.0]),
    ]


def _iter_bound(p, l, fp64_iters):
    """Mixed JCG iterations of level l: the FP64 count when the residual is generic; for
    right-hand sides FP64 CG resolves in a few steps (a single eigenmode), FP32 rounding brings
    in every mode and CG needs O(n) iterations, n the elements per axis."""
    n = max(v << l for v in p["n0"])
    return max(3 * fp64_iters + 2, 4 * n)


@pytest.mark.parametrize("cg_form", [2, 1])  # the default (two-pass: K1 + K2), and the single-pass step
def test_batched_solve_matches_oracle(E, oracle_mod, cg_form):
    probs = _mixed_batch()
    dev = [_device(p) for p in probs]
    bs = E.BatchSolver(dev, rtol=RTOL, cg_form=cg_form)
    stats, status = bs.solve()
    assert status == 0, stats
    for i, p in enumerate(probs):
        lv, ost = oracle_mod.ecmg(p, RTOL)
        # the single-problem solve with the same step form on every level
        single = E.solver_from_problem(p, precision=1, rtol=RTOL,
                                       cg_form=E.ECMG_CG_SINGLE_PASS if cg_form == 1 else E.ECMG_CG_TWO_PASS)
        sst, sstatus = single.solve()
        assert sstatus == 0
        single.close()
        st = stats[i]
        L = p["levels"]
        assert st["levels"] == L
        for l in range(L):
            U = _np(bs.get(i, E.ECMG_VEC_U, l))
            if l >= 2:
                assert st["rel_res"][l] <= RTOL, (i, l, st["rel_res"])
                assert _rel(U, lv[l]["U"]) <= 1e-7, (i, l, _rel(U, lv[l]["U"]))
                W = _np(bs.get(i, E.ECMG_VEC_W, l))
                assert _rel(W, lv[l]["W"]) <= 1e-7, (i, l, _rel(W, lv[l]["W"]))
                Ut = _np(bs.get(i, E.ECMG_VEC_UTILDE, l))
                assert _rel(Ut, lv[l]["Ut"]) <= 1e-7, (i, l, _rel(Ut, lv[l]["Ut"]))
                assert st["iters"][l] <= _iter_bound(p, l, ost["iters"][l]), (i, l, st["iters"], ost["iters"])
                # the same FP32 recurrence as the single-problem MIXED solve, up to the order of
                # the partial sums of the dot products
                assert abs(st["iters"][l] - sst["iters"][l]) <= 2, (i, l, st["iters"], sst["iters"])
            else:
                assert st["rel_res"][l] <= 1e-12, (i, l, st["rel_res"])
                assert _rel(U, lv[l]["U"]) <= 1e-10, (i, l, _rel(U, lv[l]["U"]))
            B = _np(bs.get(i, E.ECMG_VEC_B, l))
            assert st["rhs_norm"][l] == pytest.approx(ost["rhs_norm"][l], rel=1e-12)
        if p.get("u_exact") is not None:
            ue = np.asarray(p["u_exact"])
            e_b = np.abs(_np(bs.get(i, E.ECMG_VEC_U)) - ue).max()
            e_o = np.abs(lv[L - 1]["U"] - ue).max()
            assert e_b == pytest.approx(e_o, rel=0.01)
    bs.close()


def test_batched_u_out_and_repeat_are_bitwise_stable(E):
    import torch
    probs = _mixed_batch()[:4]
    dev = [_device(p) for p in probs]
    bs = E.BatchSolver(dev, rtol=RTOL)
    outs = [torch.empty(bs.finest_shape(i), dtype=torch.float64, device="cuda") for i in range(len(probs))]
    s1, _ = bs.solve(outs)
    first = [_np(o).copy() for o in outs]
    for i in range(len(probs)):
        assert np.array_equal(first[i], _np(bs.get(i, E.ECMG_VEC_U)))
    s2, _ = bs.solve(outs)
    for i in range(len(probs)):
        assert np.array_equal(first[i], _np(outs[i]))
        assert s1[i]["iters"] == s2[i]["iters"]
    bs.close()


def test_batched_graph_and_eager_agree_bitwise(E):
    probs = _mixed_batch()[:3]
    dev = [_device(p) for p in probs]
    res = []
    for use_graph in (1, 0):
        bs = E.BatchSolver(dev, rtol=RTOL, use_graph=use_graph)
        st, status = bs.solve()
        assert status == 0
        res.append(([_np(bs.get(i, E.ECMG_VEC_U)) for i in range(len(probs))], [s["iters"] for s in st]))
        bs.close()
    assert res[0][1] == res[1][1]
    assert all(np.array_equal(a, b) for a, b in zip(res[0][0], res[1][0]))


def test_batched_workload_sample_matches_oracle(E, oracle_mod):
    """Problems of the batched workload's kind (lognormal beta, random f, g_D = 0) at sizes the
    oracle finishes quickly."""
    probs = inputs.batch_problems(count=6, seed=3, sizes=(16, 32, 48))
    dev = [_device(p) for p in probs]
    bs = E.BatchSolver(dev, rtol=1e-8)
    stats, status = bs.solve()
    assert status == 0
    for i, p in enumerate(probs):
        lv, ost = oracle_mod.ecmg(p, 1e-8)
        L = p["levels"]
        assert stats[i]["rel_res"][L - 1] <= 1e-8
        U = _np(bs.get(i, E.ECMG_VEC_U))
        # two solutions inside the 1e-8 residual test differ by at most ~cond * 1e-8
        assert _rel(U, lv[L - 1]["U"]) <= 1e-5, (i, _rel(U, lv[L - 1]["U"]))
    bs.close()


def test_single_problem_calls_reject_a_batched_handle(E):
    p = _device(inputs.exp_cube(levels=3, rtol=RTOL))
    bs = E.BatchSolver([p], rtol=RTOL)
    st = E.ecmg_stats()
    assert E.ecmg_solve(bs.handle, None, st) == E.ECMG_ERR_INVALID_ARG
    out = E.ecmg_get_level_batched(bs.handle, 1, -1, E.ECMG_VEC_U, None)
    assert out == E.ECMG_ERR_INVALID_ARG
    bs.close()


def test_batched_ecmg_cg_matches_oracle(E, oracle_mod):
    """A batch solved with plain CG (ECMG_cg) against the oracle's CG, problem by problem."""
    probs = _mixed_batch()[:3]
    dev = [_device(p) for p in probs]
    bs = E.BatchSolver(dev, rtol=RTOL, preconditioner=E.ECMG_PREC_NONE)
    stats, status = bs.solve()
    assert status == 0, stats
    for i, p in enumerate(probs):
        lv, ost = oracle_mod.ecmg(p, RTOL, precond=0)
        L = p["levels"]
        assert stats[i]["rel_res"][L - 1] <= RTOL
        U = _np(bs.get(i, E.ECMG_VEC_U))
        assert _rel(U, lv[L - 1]["U"]) <= 1e-7, (i, _rel(U, lv[L - 1]["U"]))
    bs.close()


def test_batched_autotuned_tiles_match_the_oracle(E, oracle_mod):
    """The autotuner of the batched FP32 stencil (per stage: rows per thread and planes per
    block, then planes per block of each size class) changes only launch geometry and the order
    of the partial sums: the MIXED bar against the oracle still holds and the step counts stay
    within 2 of the untuned batch."""
    import ctypes
    probs = _mixed_batch()
    dev = [_device(p) for p in probs]
    plain = E.BatchSolver(dev, rtol=RTOL)
    st0, status = plain.solve()
    assert status == 0
    plain.close()
    bs = E.BatchSolver(dev, rtol=RTOL, autotune=1)
    stats, status = bs.solve()
    assert status == 0, stats
    for i, p in enumerate(probs):
        lv, ost = oracle_mod.ecmg(p, RTOL)
        L = p["levels"]
        for l in range(2, L):
            assert stats[i]["rel_res"][l] <= RTOL
            assert abs(stats[i]["iters"][l] - st0[i]["iters"][l]) <= 2, (i, l, stats[i]["iters"], st0[i]["iters"])
        U = _np(bs.get(i, E.ECMG_VEC_U))
        assert _rel(U, lv[L - 1]["U"]) <= 1e-7, (i, _rel(U, lv[L - 1]["U"]))
    # the stage kernels timed alone through the C ABI (level = stage): K1 and K2 of the last stage
    # (the default step form of a batch is the two-pass step: kernels 0 and 1)
    ms, nb = ctypes.c_double(), ctypes.c_double()
    for which in (0, 1):
        assert E.ecmg_time_kernel(bs.handle, -1, which, 2, ctypes.byref(ms), ctypes.byref(nb)) == E.ECMG_OK
        assert ms.value > 0.0 and nb.value > 0.0
    for which in (11, 5):
        assert E.ecmg_time_kernel(bs.handle, -1, which, 2, ctypes.byref(ms), ctypes.byref(nb)) == E.ECMG_ERR_INVALID_ARG
    # and the batch solves again to the same result after the timing launches
    again, status = bs.solve()
    assert status == 0
    assert [s["iters"] for s in again] == [s["iters"] for s in stats]
    bs.close()
    # a single-pass batch (autotuned on its own step kernel) times that kernel, 11
    one = E.BatchSolver(dev, rtol=RTOL, cg_form=E.ECMG_CG_SINGLE_PASS, autotune=1)
    assert E.ecmg_time_kernel(one.handle, -1, 11, 2, ctypes.byref(ms), ctypes.byref(nb)) == E.ECMG_OK
    assert ms.value > 0.0 and nb.value > 0.0
    for which in (0, 1):
        assert E.ecmg_time_kernel(one.handle, -1, which, 2, ctypes.byref(ms), ctypes.byref(nb)) == E.ECMG_ERR_INVALID_ARG
    st1, status = one.solve()
    assert status == 0
    for i, p in enumerate(probs):
        for l in range(2, p["levels"]):
            assert st1[i]["rel_res"][l] <= RTOL
    one.close()
