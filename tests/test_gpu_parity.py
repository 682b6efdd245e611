"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances, from the arithmetic of each path:
  - set-up vectors and the FP64 operator: rounding-order differences only, 1e-13 relative;
  - FP32 operator: difference form on FP32-rounded data, 1e-5 of max |A x|;
  - FP64 solves: the method's own bar, 1e-10 relative in max norm and JCG iteration counts
    within +-1 of the oracle's;
  - MIXED solves: true relative residual <= rtol and discretisation error within 1 % of the
    oracle's.
"""
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


def _level_h(p, l):
    return [(p["hi"][a] - p["lo"][a]) / (p["n0"][a] << l) for a in range(3)]


def _oracle_levels(oracle_mod, p):
    """beta per level (coarsening) and the oracle's assembled matrices."""
    L = p["levels"]
    betas = [None] * L
    betas[L - 1] = np.asarray(p["beta"], dtype=np.float64).ravel()
    for l in range(L - 2, -1, -1):
        betas[l] = oracle_mod.coarsen_beta([v << l for v in p["n0"]], betas[l + 1])
    return betas


def _cube_elements_ragged():
    """One beta, every face Dirichlet, cubic elements on a box of 5 x 3 x 7 coarse cells: the
    constant-coefficient kernels with ragged tiles on every axis."""
    return inputs.random_problem(31, n0=(5, 3, 7), levels=4, box=(1.25, 0.75, 1.75), face_bc=[0] * 6,
                                 contrast=1.0, rtol=1e-9)


PROBLEMS = {
    "exp_cube": lambda: inputs.exp_cube(levels=4, rtol=1e-10),
    "cube_elements_ragged": _cube_elements_ragged,
    # variable beta on cubic elements without Robin terms (the fixed-point element sums), one
    # with every face Dirichlet and one with Neumann faces (free boundary nodes)
    "random_cube_dirichlet": lambda: inputs.random_problem(51, n0=(3, 2, 4), levels=4, box=(0.75, 0.5, 1.0),
                                                           face_bc=[0] * 6, rtol=1e-10),
    "random_cube_neumann": lambda: inputs.random_problem(52, n0=(2, 3, 2), levels=4, box=(0.5, 0.75, 0.5),
                                                         face_bc=[0, 1, 1, 0, 1, 0], alpha=[0.0] * 6, rtol=1e-10),
    "random_mixed_bc_0": lambda: inputs.random_problem(0, n0=(2, 3, 2), levels=4, rtol=1e-10),
    "random_mixed_bc_1": lambda: inputs.random_problem(1, n0=(3, 2, 2), levels=3, rtol=1e-10),
    "problem1_load": lambda: inputs.paper_problem1(levels=4, rtol=1e-9),
    "variable_box": lambda: inputs.variable_box(levels=3, n0=(2, 2, 4), rtol=1e-9),
    # one beta everywhere (tensor-product FP64 path) on non-cubic elements with Robin faces
    "aniso_uniform_robin": lambda: inputs.random_problem(7, n0=(2, 3, 2), levels=4, rtol=1e-10, contrast=1.0,
                                                         face_bc=[1, 0, 1, 0, 1, 1],
                                                         alpha=[0.5, 0.0, 2.0, 0.0, 0.0, 1.0]),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_setup_vectors_match_oracle(E, oracle_mod, name):
    import torch
    p = PROBLEMS[name]()
    s = E.solver_from_problem(p)
    s.solve()
    betas = _oracle_levels(oracle_mod, p)
    L = p["levels"]
    loads = [None] * L
    f = np.asarray(p["f"], dtype=np.float64).ravel()
    gR = None if p.get("gR") is None else np.asarray(p["gR"], dtype=np.float64).ravel()
    for l in range(L - 1, -1, -1):
        n = [v << l for v in p["n0"]]
        if p["f_mode"] == 1:
            loads[l] = f if l == L - 1 else oracle_mod.restrict_load(n, loads[l + 1])
        else:
            step = 1 << (L - 1 - l)
            fl = np.asarray(p["f"])[::step, ::step, ::step].ravel()
            gl = None if gR is None else np.asarray(p["gR"])[::step, ::step, ::step].ravel()
            loads[l] = oracle_mod.load_nodal(n, _level_h(p, l), fl, p["face_bc"], gl)
    for l in range(L):
        bg = _np(s.get(E.ECMG_VEC_BETA, l)).ravel()
        assert np.array_equal(bg, betas[l]), l  # same summation order: bit-exact
        b = _np(s.get(E.ECMG_VEC_B, l)).ravel()
        scale = np.abs(loads[l]).max()
        assert np.abs(b - loads[l]).max() <= 1e-13 * scale, l
    s.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("precision", [0, 1])
def test_operator_matches_csr(E, oracle_mod, name, precision):
    import torch
    p = PROBLEMS[name]()
    s = E.solver_from_problem(p, precision=precision)
    s.solve()
    betas = _oracle_levels(oracle_mod, p)
    for l in range(p["levels"]):
        n = [v << l for v in p["n0"]]
        A = oracle_mod.assemble(n, _level_h(p, l), betas[l], p["face_bc"], p["alpha"])
        x = inputs.random_vector(100 + l, (n[2] + 1, n[1] + 1, n[0] + 1))
        want = A.matvec(x.ravel())
        xt = torch.tensor(x, device="cuda")
        got = _np(s.apply(xt, level=l, precision=precision)).ravel()
        scale = np.abs(want).max()
        tol = 1e-13 if precision == 0 else 1e-5
        assert np.abs(got - want).max() <= tol * scale, (l, np.abs(got - want).max() / scale)
    s.close()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("variant", [0, 1])
def test_fp64_solve_matches_oracle(E, oracle_mod, name, variant):
    p = PROBLEMS[name]()
    lv, ost = oracle_mod.ecmg(p, p["rtol"], exp_variant=variant)
    assert ost["status"] == 0
    s = E.solver_from_problem(p, precision=0, exp_variant=variant)
    gst, status = s.solve()
    assert status == 0, gst
    for l in range(p["levels"]):
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= 1e-10, (l, _rel(U, lv[l]["U"]))
        if l >= 2:
            assert abs(gst["iters"][l] - ost["iters"][l]) <= 1, (l, gst["iters"], ost["iters"])
            assert gst["rel_res"][l] <= p["rtol"] * 1.01
            W = _np(s.get(E.ECMG_VEC_W, l))
            assert _rel(W, lv[l]["W"]) <= 1e-10, (l, _rel(W, lv[l]["W"]))
            Ut = _np(s.get(E.ECMG_VEC_UTILDE, l))
            assert _rel(Ut, lv[l]["Ut"]) <= 1e-10, (l, _rel(Ut, lv[l]["Ut"]))
        assert gst["rhs_norm"][l] == pytest.approx(ost["rhs_norm"][l], rel=1e-12)
    s.close()


@pytest.mark.parametrize("name", ["exp_cube", "cube_elements_ragged", "random_cube_dirichlet", "random_cube_neumann",
                                  "problem1_load", "random_mixed_bc_0"])
@pytest.mark.parametrize("cg_form", [0, 2])  # two-pass step, and the default (single pass on these small levels)
def test_mixed_solve_reaches_tolerance_and_fp64_accuracy(E, oracle_mod, name, cg_form):
    p = PROBLEMS[name]()
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    s = E.solver_from_problem(p, precision=1, cg_form=cg_form)
    gst, status = s.solve()
    assert status == 0, gst
    L = p["levels"]
    for l in range(2, L):
        assert gst["rel_res"][l] <= p["rtol"], (l, gst["rel_res"])
        # FP32 inner iterations with FP64 residual replacement keep the Krylov recurrence: on
        # most problems they take exactly the FP64 iteration count. Problem 1 (a single
        # eigenmode, where FP64 JCG converges in a few steps) loses that edge to FP32 rounding,
        # which brings in every mode: then CG needs O(n) iterations, n the elements per axis. A
        # broken recurrence would run into the iteration cap.
        n = max(v << l for v in p["n0"])
        assert gst["iters"][l] <= max(3 * ost["iters"][l] + 2, 4 * n), (l, gst["iters"], ost["iters"])
        U = _np(s.get(E.ECMG_VEC_U, l))
        # the mixed solution satisfies the same residual test, so it differs from the oracle's
        # by at most what two solutions inside the tolerance can differ by
        assert _rel(U, lv[l]["U"]) <= 1e-7, (l, _rel(U, lv[l]["U"]))
    if p.get("u_exact") is not None:
        ue = np.asarray(p["u_exact"])
        e_mixed = np.abs(_np(s.get(E.ECMG_VEC_U, L - 1)) - ue).max()
        e_oracle = np.abs(lv[L - 1]["U"] - ue).max()
        assert e_mixed == pytest.approx(e_oracle, rel=0.01)
    s.close()


@pytest.mark.parametrize("cg_form", [0, 2])
def test_graph_and_eager_paths_agree_bitwise(E, cg_form):
    p = PROBLEMS["random_mixed_bc_0"]()
    outs = []
    for use_graph in (1, 0):
        for precision in (0, 1):
            s = E.solver_from_problem(p, precision=precision, use_graph=use_graph, cg_form=cg_form)
            st, status = s.solve()
            assert status == 0
            outs.append((precision, _np(s.get(E.ECMG_VEC_U)), st["iters"]))
            s.close()
    for prec in (0, 1):
        a = [o for o in outs if o[0] == prec]
        assert np.array_equal(a[0][1], a[1][1]) and a[0][2] == a[1][2]


def test_repeated_solves_are_deterministic(E):
    p = PROBLEMS["exp_cube"]()
    s = E.solver_from_problem(p, precision=1)
    s.solve()
    u1 = _np(s.get(E.ECMG_VEC_U))
    s.solve()
    u2 = _np(s.get(E.ECMG_VEC_U))
    assert np.array_equal(u1, u2)
    s.close()


# Problems whose finest grids span several stencil tiles in x and y with ragged last tiles,
# and many z-blocks at small kz; one all-Dirichlet cube (cubic-element path) and one box with
# Robin faces on x-, y+ and z-.
TILE_PROBLEMS = {
    "cos_cube_40": lambda: inputs.cos_cube(levels=4, n0=(5, 5, 5), rtol=1e-10),
    "random_box_robin": lambda: inputs.random_problem(11, n0=(5, 3, 4), levels=4, rtol=1e-10,
                                                      face_bc=[1, 0, 0, 1, 1, 0],
                                                      alpha=[0.5, 0.0, 0.0, 2.0, 1.0, 0.0]),
}


@pytest.mark.parametrize("name", sorted(TILE_PROBLEMS))
@pytest.mark.parametrize("cg_form", [0, 2])
def test_mixed_tile_shapes_agree(E, oracle_mod, name, cg_form):
    """Every FP32 stencil tile shape gives the same mixed solve (up to the order of the p.q
    partial sums), within the mixed bar of the oracle."""
    p = TILE_PROBLEMS[name]()
    L = p["levels"]
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    s = E.solver_from_problem(p, precision=1, cg_form=cg_form)
    ref, status = s.solve()
    assert status == 0, ref
    U_ref = _np(s.get(E.ECMG_VEC_U))
    for ry, kz in [(1, 4), (1, 16), (2, 4), (2, 8), (2, 64)]:
        for l in range(2, L):
            s.set_tiles(ry, kz, level=l)
        assert s.get_tiles(-1) == (ry, kz)
        st, status = s.solve()
        assert status == 0, (ry, kz, st)
        for l in range(2, L):
            assert st["rel_res"][l] <= p["rtol"], (ry, kz, l, st["rel_res"])
            assert abs(st["iters"][l] - ref["iters"][l]) <= 1, (ry, kz, st["iters"], ref["iters"])
        U = _np(s.get(E.ECMG_VEC_U))
        assert _rel(U, U_ref) <= 1e-7, (ry, kz, _rel(U, U_ref))
        assert _rel(U, lv[L - 1]["U"]) <= 1e-7, (ry, kz, _rel(U, lv[L - 1]["U"]))
    s.close()


def test_tile_shape_validation(E):
    p = PROBLEMS["exp_cube"]()
    s = E.solver_from_problem(p, precision=1)
    for ry, kz in [(3, 16), (4, 16), (0, 16), (1, 3), (2, 2048)]:
        with pytest.raises(E.EcmgError):
            s.set_tiles(ry, kz)
    with pytest.raises(E.EcmgError):
        s.set_tiles(1, 16, level=99)
    s.close()
    s64 = E.solver_from_problem(p, precision=0)
    with pytest.raises(E.EcmgError):
        s64.set_tiles(1, 16)
    with pytest.raises(E.EcmgError):
        s64.get_tiles()
    s64.close()


def test_autotuned_solve_matches_oracle(E, oracle_mod):
    """autotune=1 picks a shape on the 64^3 level (>= 2^18 nodes) and the solve keeps the
    mixed bar."""
    p = inputs.cos_cube(levels=5, n0=(4, 4, 4), rtol=1e-10)
    L = p["levels"]
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    s = E.solver_from_problem(p, precision=1, autotune=1)
    ry, kz = s.get_tiles(-1)
    assert ry in (1, 2) and 4 <= kz <= 1024
    st, status = s.solve()
    assert status == 0, st
    assert st["rel_res"][L - 1] <= p["rtol"]
    U = _np(s.get(E.ECMG_VEC_U))
    assert _rel(U, lv[L - 1]["U"]) <= 1e-7
    ue = np.asarray(p["u_exact"])
    assert np.abs(U - ue).max() == pytest.approx(np.abs(lv[L - 1]["U"] - ue).max(), rel=0.01)
    s.close()


def test_mixed_jump_problem_matches_oracle(E, oracle_mod):
    """Coefficient jump 1 | 100 and a singular solution: MIXED solve against the oracle."""
    p = inputs.jump_singular(levels=5, n0=(4, 2, 2), rtol=1e-10)
    L = p["levels"]
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    s = E.solver_from_problem(p, precision=1)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, L):
        assert st["rel_res"][l] <= p["rtol"], (l, st["rel_res"])
        for which, key in ((E.ECMG_VEC_U, "U"), (E.ECMG_VEC_W, "W"), (E.ECMG_VEC_UTILDE, "Ut")):
            got = _np(s.get(which, l))
            assert _rel(got, lv[l][key]) <= 1e-7, (l, key, _rel(got, lv[l][key]))
    s.close()


@pytest.mark.parametrize("name", ["exp_cube", "random_mixed_bc_0", "problem1_load", "aniso_uniform_robin"])
def test_fp64_ecmg_cg_matches_oracle(E, oracle_mod, name):
    """ECMG_cg (plain CG on line 8 of Alg. 4): the FP64 path against the oracle's CG."""
    p = PROBLEMS[name]()
    lv, ost = oracle_mod.ecmg(p, p["rtol"], precond=0)
    assert ost["status"] == 0
    s = E.solver_from_problem(p, precision=0, preconditioner=E.ECMG_PREC_NONE)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, p["levels"]):
        assert abs(st["iters"][l] - ost["iters"][l]) <= 1, (l, st["iters"], ost["iters"])
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= 1e-10, (l, _rel(U, lv[l]["U"]))
    s.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_fixed_schedule_matches_oracle(E, oracle_mod, precond):
    """Alg. 3's fixed step counts m_j = ceil(m_L beta^(L-j)): exactly m_j steps per level, FP64
    against the oracle; MIXED takes the same step counts and ends with status OK."""
    p = PROBLEMS["random_mixed_bc_0"]()
    L = p["levels"]
    lv, ost = oracle_mod.ecmg(p, p["rtol"], precond=precond, schedule=1, mL=3, sched_beta=2.5)
    want = [oracle_mod.schedule_steps(L, l, 3, 2.5) for l in range(2, L)]
    assert ost["iters"][2:] == want
    opts = dict(preconditioner=E.ECMG_PREC_JACOBI if precond else E.ECMG_PREC_NONE,
                schedule=E.ECMG_SCHED_FIXED, sched_mL=3, sched_beta=2.5)
    s = E.solver_from_problem(p, precision=0, **opts)
    st, status = s.solve()
    assert status == 0, st
    assert st["iters"][2:L] == want, (st["iters"], want)
    for l in range(2, L):
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= 1e-10, (l, _rel(U, lv[l]["U"]))
    s.close()
    m = E.solver_from_problem(p, precision=1, **opts)
    st, status = m.solve()
    assert status == 0, st
    assert st["iters"][2:L] == want, (st["iters"], want)
    m.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_problem2_anisotropic_matches_oracle(E, oracle_mod, precision):
    """Problem 2 of Sec. 5 (elements 0.1 x 0.25 x 0.2 on the coarsest grid, Neumann faces,
    eps 1e-12): FP64 to the method's bar, MIXED to the mixed bar."""
    p = inputs.paper_problem2(levels=4, rtol=1e-12)
    L = p["levels"]
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    s = E.solver_from_problem(p, precision=precision)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, L):
        assert st["rel_res"][l] <= 1e-12 * 1.01, (l, st["rel_res"])
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= (1e-10 if precision == 0 else 1e-9), (l, _rel(U, lv[l]["U"]))
        if precision == 0:
            assert abs(st["iters"][l] - ost["iters"][l]) <= 1, (l, st["iters"], ost["iters"])
    s.close()


# ---- compact inputs: separable f and g_D, one beta (on-device assembly) ------------------------
SEPARABLE = {
    "cos_cube_compact": lambda: inputs.cos_cube_compact(levels=4, n0=(4, 4, 4), rtol=1e-10),
    "random_separable_dirichlet": lambda: inputs.random_separable(21, n0=(3, 2, 2), levels=4),
    "random_separable_robin": lambda: inputs.random_separable(22, n0=(2, 3, 2), levels=4, gD_terms=1,
                                                              face_bc=[0, 1, 1, 0, 1, 0]),
}


def _dense_from_compact(oracle_mod, p):
    """The same problem with dense inputs, assembled by the oracle from the compact data."""
    L = p["levels"]
    n = inputs.finest(p["n0"], L)
    d = dict(p)
    d["f"] = oracle_mod.load_separable(n, _level_h(p, L - 1), p["f_terms"], p["f"])
    d["f_mode"] = 1
    d["gD"] = oracle_mod.nodal_separable(n, p["gD_terms"], p["gD"]) if p["gD_terms"] else None
    d["beta"] = np.full((n[2], n[1], n[0]), p["beta_const"])
    for k in ("f_terms", "gD_terms", "beta_const"):
        d.pop(k)
    return d


@pytest.mark.parametrize("name", sorted(SEPARABLE))
def test_separable_setup_matches_oracle(E, oracle_mod, name):
    """The load assembled on the device from Gauss samples (and its coarse restrictions), beta
    from beta_const and g_D from its factors equal the oracle's definitions on every level."""
    import torch
    p = SEPARABLE[name]()
    d = _dense_from_compact(oracle_mod, p)
    s = E.solver_from_problem(p, precision=0)
    s.solve()
    L = p["levels"]
    betas = _oracle_levels(oracle_mod, d)
    load = np.asarray(d["f"]).ravel()
    for l in range(L - 1, -1, -1):
        n = [v << l for v in p["n0"]]
        if l < L - 1:
            load = oracle_mod.restrict_load(n, load)
        b = _np(s.get(E.ECMG_VEC_B, l)).ravel()
        assert np.abs(b - load).max() <= 1e-13 * np.abs(load).max(), (l, np.abs(b - load).max())
        assert np.array_equal(_np(s.get(E.ECMG_VEC_BETA, l)).ravel(), betas[l]), l
        if d["gD"] is not None:
            step = 1 << (L - 1 - l)
            g = np.asarray(d["gD"])[::step, ::step, ::step].ravel()
            dirichlet = oracle_mod.dirichlet_mask(n, p["face_bc"]) == 0
            U = _np(s.get(E.ECMG_VEC_U, l)).ravel()
            assert np.abs(U[dirichlet] - g[dirichlet]).max() <= 1e-14 * np.abs(g).max(), l
    s.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", sorted(SEPARABLE))
@pytest.mark.parametrize("precision", [0, 1])
def test_separable_solve_matches_oracle(E, oracle_mod, name, precision):
    p = SEPARABLE[name]()
    d = _dense_from_compact(oracle_mod, p)
    lv, ost = oracle_mod.ecmg(d, d["rtol"])
    assert ost["status"] == 0
    s = E.solver_from_problem(p, precision=precision)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, p["levels"]):
        assert st["rel_res"][l] <= p["rtol"] * 1.01, (l, st["rel_res"])
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= (1e-10 if precision == 0 else 1e-7), (l, _rel(U, lv[l]["U"]))
        if precision == 0:
            assert abs(st["iters"][l] - ost["iters"][l]) <= 1, (l, st["iters"], ost["iters"])
    s.close()


def test_compact_and_dense_inputs_give_the_same_solve(E, oracle_mod):
    """The compact path changes only how the inputs reach the device: with the oracle's dense
    assembly of the same data, the FP64 solve agrees to rounding and takes the same steps."""
    p = inputs.cos_cube_compact(levels=4, n0=(4, 4, 4), rtol=1e-10)
    d = _dense_from_compact(oracle_mod, p)
    a = E.solver_from_problem(p, precision=0)
    b = E.solver_from_problem(d, precision=0)
    sa, _ = a.solve()
    sb, _ = b.solve()
    assert all(abs(x - y) <= 1 for x, y in zip(sa["iters"], sb["iters"])), (sa["iters"], sb["iters"])
    L = p["levels"]
    assert _rel(_np(a.get(E.ECMG_VEC_U, L - 1)), _np(b.get(E.ECMG_VEC_U, L - 1))) <= 1e-12
    a.close()
    b.close()


# ---- the FP32 search-direction kernel (K1) itself, on every path and tile shape -----------------
K1_PROBLEMS = {
    # one beta, every face Dirichlet: the constant-coefficient path
    "exp_cube": lambda: inputs.exp_cube(levels=4, rtol=1e-10),
    "cos_cube_ragged": lambda: inputs.cos_cube(levels=3, n0=(9, 5, 7), rtol=1e-8),
    "cube_elements_ragged": _cube_elements_ragged,
    # general path: variable beta, Robin faces, non-cubic elements
    "random_mixed_bc_0": lambda: inputs.random_problem(0, n0=(2, 3, 2), levels=4, rtol=1e-10),
    "variable_box": lambda: inputs.variable_box(levels=3, n0=(2, 2, 4), rtol=1e-9),
}


@pytest.mark.parametrize("name", sorted(K1_PROBLEMS))
@pytest.mark.parametrize("tiles", [None, (1, 4), (2, 4), (2, 7)])
@pytest.mark.parametrize("cg_form", [2, 0])  # default (single-pass levels), two-pass (ring form of K1)
def test_k1_operator_matches_csr(E, oracle_mod, name, tiles, cg_form):
    """q = A p from the kernel the MIXED iteration runs (ECMG_APPLY_K1) against the oracle's
    assembled matrix on the nodes off Dirichlet faces: FP32 bar 1e-5 of max |A x|. Small kz
    spreads a level over several z-blocks with a ragged last one. On two-pass levels the kernel
    reads p_old from the level's ring of search directions (4D tensor map)."""
    import torch
    p = K1_PROBLEMS[name]()
    s = E.solver_from_problem(p, precision=1, cg_form=cg_form)
    s.solve()
    betas = _oracle_levels(oracle_mod, p)
    for l in range(2, p["levels"]):
        if tiles is not None:
            s.set_tiles(tiles[0], tiles[1], level=l)
        n = [v << l for v in p["n0"]]
        A = oracle_mod.assemble(n, _level_h(p, l), betas[l], p["face_bc"], p["alpha"])
        free = oracle_mod.dirichlet_mask(n, p["face_bc"]) == 1
        x = inputs.random_vector(300 + l, (n[2] + 1, n[1] + 1, n[0] + 1))
        want = A.matvec(x.ravel())
        got = _np(s.apply(torch.tensor(x, device="cuda"), level=l, precision=E.ECMG_APPLY_K1)).ravel()
        scale = np.abs(want[free]).max()
        assert np.abs(got[free] - want[free]).max() <= 1e-5 * scale, (l, np.abs(got[free] - want[free]).max() / scale)
        assert np.all(got[~free] == 0.0)
    s.close()


@pytest.mark.parametrize("cg_form", [0, 2])
def test_beta_change_under_a_recorded_graph_switches_the_stencil_path(E, oracle_mod, cg_form):
    """A MIXED graph recorded while beta was uniform runs the constant-coefficient stencil
    kernel; after the caller rewrites beta in place with a variable field, the next solve must
    notice (the kernel checks the level flag), record again with the general kernel and give
    the same result as a fresh handle."""
    import torch
    p = inputs.exp_cube(levels=4, rtol=1e-10)
    q = inputs.random_problem(3, n0=(4, 4, 4), levels=4, rtol=1e-10, face_bc=[0] * 6)
    beta = torch.ones(np.asarray(p["beta"]).shape, dtype=torch.float64, device="cuda")
    f = torch.tensor(np.asarray(p["f"]), device="cuda")
    gD = torch.tensor(np.asarray(p["gD"]), device="cuda")
    s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], beta, f, gD, None,
                 rtol=1e-10, precision=1, cg_form=cg_form)
    st1, status = s.solve()
    assert status == 0, st1
    beta.copy_(torch.tensor(np.asarray(q["beta"]), device="cuda"))
    st2, status = s.solve()
    assert status == 0, st2
    U2 = _np(s.get(E.ECMG_VEC_U, -1))
    d = dict(p, beta=np.asarray(q["beta"]))
    fresh = E.solver_from_problem(d, precision=1, cg_form=cg_form)
    st3, status = fresh.solve()
    assert status == 0
    assert st2["iters"] == st3["iters"], (st2["iters"], st3["iters"])
    assert np.array_equal(U2, _np(fresh.get(E.ECMG_VEC_U, -1)))
    lv, ost = oracle_mod.ecmg(d, d["rtol"])
    assert _rel(U2, lv[-1]["U"]) <= 1e-7
    s.close()
    fresh.close()


@pytest.mark.parametrize("name", ["exp_cube", "cos_cube_cube", "cube_elements_ragged", "random_cube_dirichlet",
                                  "random_cube_neumann", "variable_box", "problem1_load", "random_mixed_bc_0"])
def test_mixed_reported_residual_is_the_true_residual(E, oracle_mod, name):
    """The residual the MIXED solve reports on every level (from its last FP64 residual
    evaluation: the exact constant-coefficient kernel on one-beta all-Dirichlet cubes, the
    general one elsewhere) is ||b - A U|| / ||f_h|| of the returned U, recomputed by the oracle
    with its assembled matrix; the two differ only by the FP32 rounding of r."""
    p = inputs.cos_cube(levels=4, n0=(4, 4, 4), rtol=1e-9) if name == "cos_cube_cube" else PROBLEMS[name]()
    s = E.solver_from_problem(p, precision=1)
    st, status = s.solve()
    assert status == 0, st
    betas = _oracle_levels(oracle_mod, p)
    for l in range(2, p["levels"]):
        n = [v << l for v in p["n0"]]
        A = oracle_mod.assemble(n, _level_h(p, l), betas[l], p["face_bc"], p["alpha"])
        free = oracle_mod.dirichlet_mask(n, p["face_bc"]) == 1
        U = _np(s.get(E.ECMG_VEC_U, l)).ravel()
        b = _np(s.get(E.ECMG_VEC_B, l)).ravel()
        r = (b - A.matvec(U))[free]
        rel = np.sqrt(np.dot(r, r)) / st["rhs_norm"][l]
        assert rel == pytest.approx(st["rel_res"][l], rel=1e-4), (l, rel, st["rel_res"][l])
    s.close()


def _random_case(seed):
    """Seeded random problem of random shape: coarsest 1..3 elements per axis, 3 or 4 levels,
    cubic or stretched elements, one or many betas, random face types and Robin alphas."""
    rng = np.random.default_rng(seed)
    n0 = tuple(int(v) for v in rng.integers(1, 4, 3))
    levels = int(rng.integers(3, 5))
    if rng.random() < 0.5:
        h0 = float(rng.uniform(0.2, 0.5))
        box = tuple(h0 * v for v in n0)  # cubic elements
    else:
        box = tuple(float(v) for v in rng.uniform(0.5, 1.5, 3))
    contrast = 1.0 if rng.random() < 0.4 else 10.0
    return inputs.random_problem(int(seed), n0=n0, levels=levels, box=box, contrast=contrast, rtol=1e-10)


@pytest.mark.parametrize("seed", range(200, 216))
@pytest.mark.parametrize("precision", [0, 1])
def test_random_problems_match_oracle(E, oracle_mod, seed, precision):
    """Randomised parity sweep over shapes, boundary types and coefficient fields: FP64 to the
    method's bar (1e-10, iterations +-1), MIXED to the mixed bar (residual test met, U within
    1e-7 of the oracle's)."""
    p = _random_case(seed)
    lv, ost = oracle_mod.ecmg(p, p["rtol"])
    assert ost["status"] == 0
    # MIXED: the two-pass step here (the single-pass sweep is in test_gpu_single_pass.py)
    s = E.solver_from_problem(p, precision=precision, cg_form=0)
    st, status = s.solve()
    assert status == 0, (p["n0"], p["levels"], p["face_bc"], st)
    for l in range(2, p["levels"]):
        U = _np(s.get(E.ECMG_VEC_U, l))
        assert _rel(U, lv[l]["U"]) <= (1e-10 if precision == 0 else 1e-7), (l, _rel(U, lv[l]["U"]))
        assert st["rel_res"][l] <= p["rtol"] * 1.01, (l, st["rel_res"])
        if precision == 0:
            assert abs(st["iters"][l] - ost["iters"][l]) <= 1, (l, st["iters"], ost["iters"])
    s.close()


@pytest.mark.parametrize("name", ["random_cube_dirichlet", "random_mixed_bc_0"])
def test_dense_beta_read_in_one_pass_or_unaligned_gives_the_same_solve(E, name):
    """A MIXED solve reads a 16-byte aligned dense beta in one pass (packing, FP32 copy, uniform
    test and the coarsening of the level below); a beta array that starts 8 bytes into its
    allocation takes the separate passes. Both give the same beta on every level and the same
    solve, bit for bit."""
    import torch
    p = PROBLEMS[name]()
    t = lambda a: None if a is None else torch.as_tensor(np.asarray(a), dtype=torch.float64).contiguous().cuda()
    beta = t(p["beta"])
    buf = torch.empty(beta.numel() + 1, dtype=torch.float64, device="cuda")
    shifted = buf[1:]
    shifted.copy_(beta.ravel())
    assert beta.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    out = []
    for b in (beta, shifted):
        s = E.Solver(p["n0"], p["levels"], p["lo"], p["hi"], p["face_bc"], p["alpha"], b, t(p["f"]), t(p.get("gD")),
                     t(p.get("gR")), f_mode=p.get("f_mode", 0), rtol=p["rtol"], precision=1)
        st, status = s.solve()
        assert status == 0, st
        out.append(([_np(s.get(E.ECMG_VEC_BETA, l)) for l in range(p["levels"])], _np(s.get(E.ECMG_VEC_U)), st["iters"]))
        s.close()
    for l in range(p["levels"]):
        assert np.array_equal(out[0][0][l], out[1][0][l]), l
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
