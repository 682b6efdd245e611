"""The ring of search directions of the two-pass MIXED step (option ring_slots), through the C ABI.

With a ring, the FP32 step stores its search direction p_k in the next ring slot instead of
adding alpha_k p_k to the correction vector e; the pending directions are added, oldest first,
with the same FP32 fused multiply-adds the correction vector performs, when ring_slots - 2 are
pending (into e, by K2) and at each residual replacement (into the FP64 iterate). So the ring
solve is bit-identical to the correction-vector solve for any ring size: same iterates, same
iteration and replacement counts, same solutions."""
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


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# Every face Dirichlet and one beta: the levels run the constant-coefficient stencil kernel, the
# one that uses the ring (cubic elements, non-cubic elements, ragged tiles, compact inputs).
PROBLEMS = {
    "exp_cube": lambda: inputs.exp_cube(levels=4, rtol=1e-10),
    "cos_cube_40": lambda: inputs.cos_cube(levels=4, n0=(5, 5, 5), rtol=1e-10),
    "cube_elements_ragged": lambda: inputs.random_problem(31, n0=(5, 3, 7), levels=4, box=(1.25, 0.75, 1.75),
                                                          face_bc=[0] * 6, contrast=1.0, rtol=1e-9),
    "one_beta_box": lambda: inputs.random_problem(7, n0=(4, 3, 5), levels=4, box=(1.0, 0.9, 1.3),
                                                  face_bc=[0] * 6, contrast=1.0, rtol=1e-10),
    "cos_cube_compact": lambda: inputs.cos_cube_compact(levels=4, n0=(4, 4, 4), rtol=1e-10, with_exact=False),
}


def _solve(E, p, **kw):
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_TWO_PASS, **kw)
    st, status = s.solve()
    assert status == 0, st
    U = [_np(s.get(E.ECMG_VEC_U, l)) for l in range(p["levels"])]
    Ut = _np(s.get(E.ECMG_VEC_UTILDE))
    s.close()
    return st, U, Ut


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("slots", [4, 7, 64])
def test_ring_solve_is_bitwise_the_correction_vector_solve(E, name, use_graph, slots):
    """4 slots add the ring to e every second step, 7 every fifth, 64 only at replacements on
    these levels."""
    p = PROBLEMS[name]()
    st0, U0, Ut0 = _solve(E, p, ring_slots=0, use_graph=use_graph)
    st1, U1, Ut1 = _solve(E, p, ring_slots=slots, use_graph=use_graph)
    assert st1["iters"] == st0["iters"] and st1["updates"] == st0["updates"], (st0, st1)
    for l in range(p["levels"]):
        assert np.array_equal(U1[l], U0[l]), l
    assert np.array_equal(Ut1, Ut0)


@pytest.mark.parametrize("name", sorted(set(PROBLEMS) - {"cos_cube_compact"}))  # the oracle takes dense inputs
def test_smallest_ring_meets_the_mixed_bar(E, oracle_mod, name):
    """Against the oracle directly: the mixed bar of test_gpu_parity.py (1e-7 relative)."""
    p = PROBLEMS[name]()
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    assert ost["status"] == 0
    st, U, _ = _solve(E, p, ring_slots=4)
    for l in range(2, p["levels"]):
        assert st["rel_res"][l] <= p["rtol"], (l, st["rel_res"])
        assert _rel(U[l], lv[l]["U"]) <= 1e-7, (l, _rel(U[l], lv[l]["U"]))


def _workspace(E, n0, levels, **opts):
    import ctypes
    p = E.ecmg_problem()
    p.n0[:] = list(n0)
    p.levels = levels
    p.lo[:] = [0, 0, 0]
    p.hi[:] = [1, 1, 1]
    p.beta = 16  # any non-null pointer: ecmg_workspace_bytes reads no input
    p.f = 16
    o = E.default_options(precision=E.ECMG_MIXED, **opts)
    b = ctypes.c_uint64()
    assert E.ecmg_workspace_bytes(ctypes.byref(p), ctypes.byref(o), ctypes.byref(b)) == 0
    return b.value


def test_ring_auto_choice_follows_the_device_memory(E):
    """ECMG_RING_AUTO: 64 slots while the workspace stays within 3/4 of the device's memory, else
    the most (>= 34) that do, else none -- checked against the byte counts of explicit choices."""
    import torch
    total = torch.cuda.get_device_properties(0).total_memory
    budget = total // 4 * 3
    for n0, levels in (((8, 8, 8), 7), ((8, 8, 16), 7), ((12, 12, 12), 7), ((16, 16, 16), 7)):
        auto = _workspace(E, n0, levels)
        base = _workspace(E, n0, levels, ring_slots=0)
        per_slot = (_workspace(E, n0, levels, ring_slots=4) - base) // 4
        want = min(64, (budget - base) // per_slot) if budget > base else 0
        want = want if want >= 8 else 0
        assert auto == base + want * per_slot, (n0, auto, base, per_slot, want)
    # the benchmark's 512^3 cube takes the full ring
    assert _workspace(E, (8, 8, 8), 7) == _workspace(E, (8, 8, 8), 7, ring_slots=64)


def test_fixed_schedule_takes_exactly_m_j_steps_with_any_ring(E, oracle_mod):
    """Alg. 3's fixed step counts with and without a ring, and the same iterates."""
    p = PROBLEMS["one_beta_box"]()
    L = p["levels"]
    want = [oracle_mod.schedule_steps(L, l, 3, 2.5) for l in range(2, L)]
    out = []
    for slots in (0, 4, 64):
        m = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_TWO_PASS, schedule=E.ECMG_SCHED_FIXED,
                                  sched_mL=3, sched_beta=2.5, ring_slots=slots)
        st, status = m.solve()
        assert status == 0, (slots, st)
        assert st["iters"][2:L] == want, (slots, st["iters"], want)
        out.append(_np(m.get(E.ECMG_VEC_U)))
        m.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_ring_runs_with_the_constant_coefficient_kernel_only(E):
    """The ring's kernels run where the level has one beta and every face Dirichlet (K1 then
    moves 16 bytes per node: r and p_old in, p and q out); with a variable beta the level keeps
    the correction vector (K1 moves 20 bytes per node plus beta and D^-1) and solves as before."""
    p = PROBLEMS["one_beta_box"]()
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_TWO_PASS, ring_slots=16)
    s.solve()
    for l in range(2, p["levels"]):
        n = [(v << l) - 1 for v in p["n0"]]
        _, b = s.time_kernel(0, l, reps=1)
        assert b == 16.0 * n[0] * n[1] * n[2], (l, b)
        _, b9 = s.time_kernel(9, l, reps=1)
        nodes = np.prod([(v << l) + 1 for v in p["n0"]])
        assert b9 == (16.0 + 4.0 * 14) * nodes, (l, b9)
    s.close()
    q = inputs.random_problem(51, n0=(3, 2, 4), levels=4, box=(0.75, 0.5, 1.0), face_bc=[0] * 6, rtol=1e-10)
    outs = []
    for slots in (0, 16):
        s = E.solver_from_problem(q, precision=1, cg_form=E.ECMG_CG_TWO_PASS, ring_slots=slots)
        st, status = s.solve()
        assert status == 0
        _, b = s.time_kernel(0, -1, reps=1)
        n = [(v << 3) - 1 for v in q["n0"]]
        assert b > 16.0 * n[0] * n[1] * n[2]
        outs.append(_np(s.get(E.ECMG_VEC_U)))
        s.close()
    assert np.array_equal(outs[0], outs[1])
