"""Error behaviour and degenerate cases of the CUDA path (through the C ABI): a solve that
runs out of iterations or meets a non-finite value returns a status instead of trapping,
keeps the context usable, and the smallest and the all-Robin problems match the oracle."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_iteration_cap_reports_no_convergence(E, precision):
    p = inputs.exp_cube(levels=4, rtol=1e-12)
    s = E.solver_from_problem(p, precision=precision, max_iters=2, cg_form=0)
    st, status = s.solve(raise_on_error=False)
    assert status == E.ECMG_ERR_NO_CONVERGENCE, st
    assert st["status"] == E.ECMG_ERR_NO_CONVERGENCE
    U = _np(s.get(E.ECMG_VEC_U, -1))
    assert np.all(np.isfinite(U))  # the best iterate stays in place
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_load_reports_breakdown_and_the_handle_recovers(E, precision):
    """A NaN in the load makes the residual or p.q non-finite: the solve returns
    ECMG_ERR_BREAKDOWN (no device trap), and after the caller repairs the input the same
    handle solves normally."""
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    f = torch.tensor(np.asarray(p["f"]), device="cuda")
    beta = torch.tensor(np.asarray(p["beta"]), device="cuda")
    gD = torch.tensor(np.asarray(p["gD"]), device="cuda")
    good = f.clone()
    f[10, 11, 12] = float("nan")
    s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], beta, f, gD, None,
                 rtol=1e-10, precision=precision, cg_form=0)
    st, status = s.solve(raise_on_error=False)
    assert status == E.ECMG_ERR_BREAKDOWN, st
    f.copy_(good)
    st, status = s.solve(raise_on_error=False)
    assert status == E.ECMG_OK, st
    fresh = E.solver_from_problem(p, precision=precision, cg_form=0)
    st2, _ = fresh.solve()
    assert st["iters"] == st2["iters"]
    assert np.array_equal(_np(s.get(E.ECMG_VEC_U, -1)), _np(fresh.get(E.ECMG_VEC_U, -1)))
    s.close()
    fresh.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_smallest_hierarchy_matches_oracle(E, oracle_mod, precision):
    """One coarsest element, three levels (1, 2, 4 elements per axis): two direct levels
    and one JCG level of 3^3 free nodes."""
    p = inputs.exp_cube(levels=3, n0=(1, 1, 1), rtol=1e-10)
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    s = E.solver_from_problem(p, precision=precision)
    st, status = s.solve()
    assert status == 0, st
    U = _np(s.get(E.ECMG_VEC_U, 2))
    assert _rel(U, lv[2]["U"]) <= (1e-10 if precision == 0 else 1e-7), _rel(U, lv[2]["U"])
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_all_robin_faces_match_oracle(E, oracle_mod, precision):
    """No Dirichlet face, every face Robin with alpha > 0 (a regular system without any
    eliminated node): every node is free, the stencil kernels visit the whole box."""
    p = inputs.random_problem(41, n0=(2, 3, 2), levels=4, face_bc=[1] * 6, alpha=[0.5, 1.0, 2.0, 0.25, 1.5, 0.75],
                              rtol=1e-10)
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    assert ost["status"] == 0
    s = E.solver_from_problem(p, precision=precision)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, p["levels"]):
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= (1e-10 if precision == 0 else 1e-7), (l, _rel(U, lv[l]["U"]))
        if precision == 0:
            assert abs(st["iters"][l] - ost["iters"][l]) <= 1, (l, st["iters"], ost["iters"])
    s.close()
