"""Pins of the oracle's solvers (DSOLVE, JCG of Alg. 4) and of the FE convergence order."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs


def _level_system(oracle_mod, p):
    n = p["n0"]
    h = [(p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    A = oracle_mod.assemble(n, h, p["beta"], p["face_bc"], p["alpha"])
    b = oracle_mod.load_nodal(n, h, p["f"], p["face_bc"], p["gR"])
    mask = oracle_mod.dirichlet_mask(n, p["face_bc"])
    gext = np.where(mask == 0, p["gD"].ravel(), 0.0)
    return n, A, b, mask, gext


def _dense_solution(A, b, mask, gext):
    """Textbook elimination of the free-node system with the Dirichlet values moved right."""
    D = A.dense()
    f = mask.astype(bool)
    rhs = b[f] - D[np.ix_(f, ~f)] @ gext[~f]
    x = gext.copy()
    x[f] = np.linalg.solve(D[np.ix_(f, f)], rhs)
    return x


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_jcg_and_dsolve_match_dense_solve(oracle_mod, seed):
    p = inputs.random_problem(seed, n0=(3, 4, 2), levels=1)
    n, A, b, mask, gext = _level_system(oracle_mod, p)
    x_ref = _dense_solution(A, b, mask, gext)
    x_cg, st = oracle_mod.jcg(A, mask, b, gext, gext, rtol=1e-14)
    assert st["status"] == 0 and st["iters"] > 0
    scale = np.abs(x_ref).max()
    assert np.abs(x_cg - x_ref).max() <= 1e-11 * scale
    x_ds, s = oracle_mod.dsolve(n, A, mask, b, gext)
    assert s == 0
    assert np.abs(x_ds - x_ref).max() <= 1e-12 * scale


def test_jcg_zero_iterations_when_converged(oracle_mod):
    p = inputs.random_problem(5, n0=(2, 2, 2), levels=1)
    n, A, b, mask, gext = _level_system(oracle_mod, p)
    x_ref = _dense_solution(A, b, mask, gext)
    x, st = oracle_mod.jcg(A, mask, b, gext, x_ref, rtol=1e-8)
    assert st["iters"] == 0 and st["rel_res"] < 1e-8
    assert np.array_equal(x, x_ref)


def test_jcg_reports_iteration_cap(oracle_mod):
    p = inputs.random_problem(6, n0=(4, 4, 4), levels=1)
    n, A, b, mask, gext = _level_system(oracle_mod, p)
    _, st = oracle_mod.jcg(A, mask, b, gext, gext, rtol=1e-14, max_iters=2)
    assert st["status"] == 3 and st["iters"] == 2


def test_jcg_residual_test_uses_lifted_rhs_norm(oracle_mod):
    p = inputs.random_problem(8, n0=(3, 3, 3), levels=1, face_bc=[0] * 6)
    n, A, b, mask, gext = _level_system(oracle_mod, p)
    _, st = oracle_mod.jcg(A, mask, b, gext, gext, rtol=1e-6)
    f = mask.astype(bool)
    want = np.linalg.norm((b - A.matvec(gext))[f])
    assert st["rhs_norm"] == pytest.approx(want, rel=1e-13)
    assert st["rel_res"] <= 1.01e-6


def test_fe_solution_is_second_order(oracle_mod):
    """Manufactured u = exp(x+y+z): the max-norm error of the FE solution falls by 4 per
    refinement (order 2.00, the U_h-u columns of the Sec. 5 tables)."""
    errs = []
    for n in (4, 8, 16):
        p = inputs.exp_cube(levels=1, n0=(n, n, n))
        nn, A, b, mask, gext = _level_system(oracle_mod, p)
        x, s = oracle_mod.dsolve(nn, A, mask, b, gext)
        assert s == 0
        errs.append(np.abs(x - p["u_exact"].ravel()).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.05), orders


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("precond", [1, 0])
def test_single_pass_jcg_has_the_iterates_of_textbook_jcg(oracle_mod, seed, precond):
    """The single-pass arrangement reaches, after every step count k, the iterate the textbook
    recurrence reaches after k steps (exact arithmetic makes them equal; FP64 keeps them within
    1e-10 over these short runs): a dropped or mis-signed term in the expanded r.z or ||r||
    changes beta from the second step on and fails this at once."""
    p = inputs.random_problem(seed, n0=(4, 3, 5), levels=1)
    n, A, b, mask, gext = _level_system(oracle_mod, p)
    for k in (1, 2, 3, 5, 8, 13):
        x_ref, st_ref = oracle_mod.pcg(A, mask, b, gext, gext, rtol=1e-30, max_iters=k, precond=precond, fixed=1)
        x_sp, st_sp = oracle_mod.pcg_single_pass(A, mask, b, gext, gext, rtol=1e-30, max_iters=k, precond=precond)
        assert st_ref["iters"] == st_sp["iters"] == k
        assert st_sp["status"] == 3
        assert np.abs(x_sp - x_ref).max() <= 1e-10 * np.abs(x_ref).max(), k


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_single_pass_jcg_converges_like_textbook_jcg(oracle_mod, seed):
    """To a tolerance: the same step count (within one, the test reading the expanded norm
    instead of the recursively updated residual), the true residual below the tolerance, and the
    dense solution."""
    p = inputs.random_problem(seed, n0=(3, 4, 2), levels=1)
    n, A, b, mask, gext = _level_system(oracle_mod, p)
    x_ref = _dense_solution(A, b, mask, gext)
    x_cg, st = oracle_mod.jcg(A, mask, b, gext, gext, rtol=1e-12)
    x_sp, st_sp = oracle_mod.pcg_single_pass(A, mask, b, gext, gext, rtol=1e-12)
    assert st_sp["status"] == 0 and abs(st_sp["iters"] - st["iters"]) <= 1
    assert st_sp["rel_res"] <= 1e-12 * 1.01
    assert np.abs(x_sp - x_ref).max() <= 1e-9 * np.abs(x_ref).max()


def test_openmp_build_gives_the_one_thread_results(oracle_mod):
    """The OpenMP build parallelises only the CSR rows and the element-wise vector updates (dot
    products stay sequential), so every level's solution is bit-identical to the one-thread
    build's; both report the set-up and solve seconds."""
    p = inputs.cos_cube(levels=4, n0=(4, 4, 4), rtol=1e-10)
    a, sa = oracle_mod.ecmg(p, p["rtol"])
    b, sb = oracle_mod.ecmg(p, p["rtol"], threads=4)
    assert sa["threads"] == 1 and sb["threads"] >= 1
    assert sa["iters"] == sb["iters"]
    for x, y in zip(a, b):
        assert np.array_equal(x["U"], y["U"]) and np.array_equal(x["Ut"], y["Ut"])
    for s in (sa, sb):
        assert s["seconds_assembly"] > 0.0 and s["seconds_solve"] > 0.0
