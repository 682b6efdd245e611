"""The single-pass form of the MIXED step (ECMG_CG_SINGLE_PASS) against the oracle, through the
C ABI: every parity problem at the MIXED bar (residual test met, U within 1e-7 of the oracle's),
step counts next to the two-pass form's (the two are the same recurrence in exact arithmetic),
graph and eager loop control bit for bit, the variants (plain CG, fixed schedule, separable
inputs), the stale constant-coefficient path, and the error statuses."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

from test_gpu_parity import PROBLEMS, SEPARABLE, _random_case, _rel, _np

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


def _check(E, oracle_mod, p, s, st, two=None, **oracle_kw):
    lv, ost = oracle_mod.ecmg(p, p["rtol"], **oracle_kw)
    for l in range(2, p["levels"]):
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= 1e-7, (l, _rel(U, lv[l]["U"]))
        assert st["rel_res"][l] <= p["rtol"] * 1.01, (l, st["rel_res"])
        if two is not None:
            a, b = st["iters"][l], two["iters"][l]
            assert abs(a - b) <= max(2, b // 10), (l, st["iters"], two["iters"])


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_single_pass_matches_oracle(E, oracle_mod, name):
    p = PROBLEMS[name]()
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st, status = s.solve()
    assert status == 0, st
    t = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_TWO_PASS)
    two, status = t.solve()
    assert status == 0
    _check(E, oracle_mod, p, s, st, two)
    s.close()
    t.close()


@pytest.mark.parametrize("seed", range(200, 216))
def test_single_pass_random_problems(E, oracle_mod, seed):
    p = _random_case(seed)
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st, status = s.solve()
    assert status == 0, (p["n0"], p["levels"], p["face_bc"], st)
    _check(E, oracle_mod, p, s, st)
    s.close()


@pytest.mark.parametrize("name", ["exp_cube", "random_mixed_bc_0", "aniso_uniform_robin"])
def test_single_pass_graph_and_eager_agree_bitwise(E, name):
    p = PROBLEMS[name]()
    outs = []
    for use_graph in (1, 0):
        s = E.solver_from_problem(p, precision=1, use_graph=use_graph, cg_form=E.ECMG_CG_SINGLE_PASS)
        st, status = s.solve()
        assert status == 0
        outs.append((_np(s.get(E.ECMG_VEC_U)), st["iters"]))
        st2, _ = s.solve()  # a second solve of the same handle repeats the first bit for bit
        assert st2["iters"] == st["iters"] and np.array_equal(_np(s.get(E.ECMG_VEC_U)), outs[-1][0])
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("tiles", [(1, 4), (2, 4), (2, 7), (1, 64)])
def test_single_pass_tile_shapes(E, oracle_mod, tiles):
    """Ragged tiles in every direction on the constant-coefficient and the general kernel."""
    for name in ("cube_elements_ragged", "random_mixed_bc_0"):
        p = PROBLEMS[name]()
        s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
        for l in range(2, p["levels"]):
            s.set_tiles(*tiles, level=l)
        st, status = s.solve()
        assert status == 0, (name, tiles, st)
        _check(E, oracle_mod, p, s, st)
        s.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_single_pass_plain_cg_and_fixed_schedule(E, oracle_mod, precond):
    p = PROBLEMS["exp_cube"]()
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS,
                              preconditioner=E.ECMG_PREC_JACOBI if precond else E.ECMG_PREC_NONE)
    st, status = s.solve()
    assert status == 0, st
    _check(E, oracle_mod, p, s, st, precond=precond)
    s.close()
    # fixed schedule: exactly m_j steps per level, as the two-pass form runs them
    f = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS, schedule=E.ECMG_SCHED_FIXED,
                              sched_mL=3, sched_beta=2.0, preconditioner=0 if precond else 1)
    t = E.solver_from_problem(p, precision=1, schedule=E.ECMG_SCHED_FIXED, sched_mL=3, sched_beta=2.0,
                              preconditioner=0 if precond else 1, cg_form=E.ECMG_CG_TWO_PASS)
    sf, status = f.solve()
    assert status == 0
    tf, _ = t.solve()
    assert sf["iters"] == tf["iters"]
    for l in range(2, p["levels"]):
        a, b = _np(f.get(E.ECMG_VEC_U, l)), _np(t.get(E.ECMG_VEC_U, l))
        assert _rel(a, b) <= 1e-6, (l, _rel(a, b))
    f.close()
    t.close()


@pytest.mark.parametrize("name", sorted(SEPARABLE))
def test_single_pass_separable_inputs(E, oracle_mod, name):
    from test_gpu_parity import _dense_from_compact
    p = SEPARABLE[name]()
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st, status = s.solve()
    assert status == 0, st
    _check(E, oracle_mod, _dense_from_compact(oracle_mod, p), s, st)
    s.close()


def test_single_pass_beta_change_switches_the_stencil_path(E, oracle_mod):
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    q = inputs.random_problem(3, n0=(4, 4, 4), levels=4, rtol=1e-10, face_bc=[0] * 6)
    beta = torch.ones(np.asarray(p["beta"]).shape, dtype=torch.float64, device="cuda")
    f = torch.tensor(np.asarray(p["f"]), device="cuda")
    gD = torch.tensor(np.asarray(p["gD"]), device="cuda")
    s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], beta, f, gD, None,
                 rtol=1e-10, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st1, status = s.solve()
    assert status == 0, st1
    beta.copy_(torch.tensor(np.asarray(q["beta"]), device="cuda"))
    st2, status = s.solve()
    assert status == 0, st2
    d = dict(p, beta=np.asarray(q["beta"]))
    fresh = E.solver_from_problem(d, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st3, status = fresh.solve()
    assert status == 0
    assert st2["iters"] == st3["iters"]
    assert np.array_equal(_np(s.get(E.ECMG_VEC_U, -1)), _np(fresh.get(E.ECMG_VEC_U, -1)))
    _check(E, oracle_mod, d, s, st2)
    s.close()
    fresh.close()


def test_single_pass_iteration_cap_and_breakdown(E):
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-12)
    s = E.solver_from_problem(p, precision=1, max_iters=2, cg_form=E.ECMG_CG_SINGLE_PASS)
    st, status = s.solve(raise_on_error=False)
    assert status == E.ECMG_ERR_NO_CONVERGENCE, st
    assert np.all(np.isfinite(_np(s.get(E.ECMG_VEC_U, -1))))
    s.close()
    f = torch.tensor(np.asarray(p["f"]), device="cuda")
    good = f.clone()
    f[10, 11, 12] = float("nan")
    beta = torch.tensor(np.asarray(p["beta"]), device="cuda")
    gD = torch.tensor(np.asarray(p["gD"]), device="cuda")
    s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], beta, f, gD, None,
                 rtol=1e-10, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st, status = s.solve(raise_on_error=False)
    assert status == E.ECMG_ERR_BREAKDOWN, st
    f.copy_(good)
    st, status = s.solve(raise_on_error=False)
    assert status == E.ECMG_OK, st
    s.close()


def test_single_pass_kernel_timer_and_bytes(E):
    p = PROBLEMS["cube_elements_ragged"]()
    s = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    s.solve()
    ms, nb = s.time_kernel(11, level=-1, reps=3)
    ms1, nb1 = s.time_kernel(0, level=-1, reps=3)
    assert ms > 0 and nb == pytest.approx(nb1 * 32 / 24)  # 8 words per node against K1's 6
    s.close()
    t = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_TWO_PASS)
    t.solve()
    with pytest.raises(E.EcmgError):
        t.time_kernel(11, level=-1, reps=1)
    t.close()


def test_auto_form_picks_single_pass_on_small_levels(E, oracle_mod):
    """ECMG_CG_AUTO (the default): the single-pass step on levels of fewer than 2^22 nodes, the
    two-pass step above; the solve meets the residual test and equals a two-pass solve's error."""
    p = inputs.cos_cube(levels=6, n0=(8, 8, 8), rtol=1e-10)  # 256^3 finest: 16.8 M nodes
    ue = np.asarray(p["u_exact"])
    s = E.solver_from_problem(p, precision=1)
    assert s.options.cg_form == E.ECMG_CG_AUTO
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, p["levels"]):
        assert st["rel_res"][l] <= p["rtol"] * 1.0001, (l, st["rel_res"])
    for l in range(2, 5):  # 32^3 .. 128^3: single-pass buffers exist
        ms, nb = s.time_kernel(11, level=l, reps=1)
        assert ms > 0
    with pytest.raises(E.EcmgError):  # 256^3: two-pass
        s.time_kernel(11, level=5, reps=1)
    t = E.solver_from_problem(p, precision=1, cg_form=E.ECMG_CG_TWO_PASS)
    st2, status = t.solve()
    assert status == 0
    e_auto = np.abs(_np(s.get(E.ECMG_VEC_U)) - ue).max()
    e_two = np.abs(_np(t.get(E.ECMG_VEC_U)) - ue).max()
    assert e_auto == pytest.approx(e_two, rel=1e-6)
    for l in range(2, p["levels"]):
        assert abs(st["iters"][l] - st2["iters"][l]) <= max(2, st2["iters"][l] // 10), (st["iters"], st2["iters"])
    s.close()
    t.close()
