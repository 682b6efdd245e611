"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

The oracle cannot solve 512^3, so these tests compare the CUDA path with the oracle on sampled
outputs it computes one node at a time (the operator, EXP_finite, EXP_true; pinned to the
whole-grid oracle in test_oracle_pointwise.py), and check properties that hold at any size:
the residual test on every level, MIXED against FP64 on the same system, the orders of the
discretisation and extrapolation errors between the two finest levels."""
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


def _sample_nodes(n, count, seed):
    """Random nodes plus the 8 corners and a node on every face and edge."""
    rng = np.random.default_rng(seed)
    pts = set()
    for c in range(8):
        pts.add(tuple(n[a] if (c >> a) & 1 else 0 for a in range(3)))
    for a in range(3):
        for side in (0, n[a]):
            q = [n[b] // 2 + 1 for b in range(3)]
            q[a] = side
            pts.add(tuple(q))
            r = [side if b == a else (0 if b == (a + 1) % 3 else n[b] // 3) for b in range(3)]
            pts.add(tuple(r))
    while len(pts) < count:
        pts.add(tuple(int(rng.integers(0, n[a] + 1)) for a in range(3)))
    return sorted(pts)


def _at(v, n, nodes):
    flat = np.asarray(v).ravel()
    return np.array([flat[i + (n[0] + 1) * (j + (n[1] + 1) * k)] for i, j, k in nodes])


def _max_err(v, ue):
    return float(np.abs(np.asarray(v) - ue).max())


def test_cos_cube_512_mixed_full_size(E, oracle_mod):
    """The benchmark workload: MIXED at 512^3 with autotuned tiles."""
    import torch
    p = inputs.cos_cube(levels=7, rtol=1e-10)
    L = p["levels"]
    s = E.solver_from_problem(p, precision=E.ECMG_MIXED, autotune=1)
    st, status = s.solve()
    assert status == 0, st
    for l in range(L):
        bound = 1e-12 if l < 2 else p["rtol"]
        assert st["rel_res"][l] <= bound * 1.0001, (l, st["rel_res"])
    n = [v << (L - 1) for v in p["n0"]]
    h = [1.0 / v for v in n]
    nodes = _sample_nodes(n, 600, 1)
    ue = np.asarray(p["u_exact"])
    U = {l: _np(s.get(E.ECMG_VEC_U, l)) for l in (L - 3, L - 2, L - 1)}
    err = {l: _max_err(U[l], inputs.cos_cube(levels=l + 1, rtol=1e-10)["u_exact"]) if l < L - 1 else
           _max_err(U[l], ue) for l in (L - 2, L - 1)}
    # second order between the two finest levels
    assert 3.8 < err[L - 2] / err[L - 1] < 4.2, err
    # EXP_finite and EXP_true of the finest level at sampled nodes, from the GPU's coarser U
    nc1 = [v // 2 for v in n]
    W = _np(s.get(E.ECMG_VEC_W))
    want_w = oracle_mod.exp_finite_at(n, U[L - 2].ravel(), U[L - 3].ravel(), nodes)
    interior = [k for k, (i, j, kk) in enumerate(nodes) if 0 < i < n[0] and 0 < j < n[1] and 0 < kk < n[2]]
    got_w = _at(W, n, nodes)
    assert np.abs(got_w[interior] - want_w[interior]).max() <= 1e-13 * np.abs(want_w).max()
    Ut = _np(s.get(E.ECMG_VEC_UTILDE))
    want_t = oracle_mod.exp_true_at(n, U[L - 1].ravel(), U[L - 2].ravel(), nodes)
    assert np.abs(_at(Ut, n, nodes) - want_t).max() <= 1e-13 * np.abs(want_t).max()
    # the operator of the finest level at sampled nodes, both precisions
    x = inputs.random_vector(512, (n[2] + 1, n[1] + 1, n[0] + 1))
    xt = torch.tensor(x, device="cuda")
    want = oracle_mod.apply_at(n, h, np.ones(n[0] * n[1] * n[2]), p["face_bc"], p["alpha"], x.ravel(), nodes)
    for prec, tol in ((E.ECMG_FP64, 1e-13), (E.ECMG_MIXED, 1e-5)):
        got = _at(_np(s.apply(xt, precision=prec)), n, nodes)
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), (prec, np.abs(got - want).max())
    # the FP32 stencil kernel of the iteration itself, with the autotuned tile shape: q = A x on
    # the nodes off the Dirichlet faces, 0 on them
    got = _at(_np(s.apply(xt, precision=E.ECMG_APPLY_K1)), n, nodes)
    free = np.array([0 < c[0] < n[0] and 0 < c[1] < n[1] and 0 < c[2] < n[2] for c in nodes])
    assert np.abs(got[free] - want[free]).max() <= 1e-5 * np.abs(want[free]).max()
    assert np.all(got[~free] == 0.0)
    del xt
    # b - A U recomputed by the oracle at sampled free nodes: every component of a residual with
    # ||r||_2 <= rtol ||f_h||_2 is at most that
    b = _np(s.get(E.ECMG_VEC_B)).ravel()
    fnodes = [t for t in _sample_nodes(n, 420, 3) if all(0 < t[a] < n[a] for a in range(3))]
    assert len(fnodes) >= 300
    r = _at(b, n, fnodes) - oracle_mod.apply_at(n, h, np.ones(n[0] * n[1] * n[2]), p["face_bc"], p["alpha"],
                                                U[L - 1].ravel(), fnodes)
    assert np.abs(r).max() <= p["rtol"] * st["rhs_norm"][L - 1] * 1.0001, np.abs(r).max()
    # the error norms of the library (max and RMS over all 513^3 nodes) against numpy
    Ud = s.get(E.ECMG_VEC_U)
    ued = torch.tensor(ue, device="cuda")
    mx, rms = s.norms(Ud, ued)
    d = U[L - 1] - ue
    assert mx == np.abs(d).max()
    assert rms == pytest.approx(float(np.sqrt(np.mean(d * d))), rel=1e-12)
    del Ud, ued, d
    s.close()
    # the same system in FP64: the same discretisation error to 1 %, and the same solution node
    # by node to well below that error
    s64 = E.solver_from_problem(p, precision=E.ECMG_FP64)
    st64, status = s64.solve()
    assert status == 0
    U64 = _np(s64.get(E.ECMG_VEC_U))
    e64 = _max_err(U64, ue)
    assert np.abs(U[L - 1] - U64).max() <= 1e-7 * np.abs(U64).max(), np.abs(U[L - 1] - U64).max()
    del U64
    assert err[L - 1] == pytest.approx(e64, rel=0.01)
    for l in range(2, L):
        assert abs(st64["iters"][l] - st["iters"][l]) <= max(2, 0.1 * st64["iters"][l]), (st64["iters"], st["iters"])
    s64.close()
    # the single-pass MIXED step (ECMG_CG_SINGLE_PASS) on the same workload: the residual test on
    # every level, the same error to 1 %, and the two-pass step counts within 10 %
    sp = E.solver_from_problem(p, precision=E.ECMG_MIXED, autotune=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st_sp, status = sp.solve()
    assert status == 0, st_sp
    for l in range(2, L):
        assert st_sp["rel_res"][l] <= p["rtol"] * 1.0001, (l, st_sp["rel_res"])
        assert abs(st_sp["iters"][l] - st["iters"][l]) <= max(2, 0.1 * st["iters"][l]), (st_sp["iters"], st["iters"])
    assert _max_err(_np(sp.get(E.ECMG_VEC_U)), ue) == pytest.approx(e64, rel=0.01)
    sp.close()


def test_variable_box_full_size_fp64(E, oracle_mod):
    """Configuration 2 at 512 x 512 x 1024 elements in FP64: variable beta, Robin on z = 0."""
    import torch
    p = inputs.variable_box(levels=7, rtol=1e-9)
    L = p["levels"]
    s = E.solver_from_problem(p, precision=E.ECMG_FP64)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, L):
        assert st["rel_res"][l] <= p["rtol"] * 1.0001, (l, st["rel_res"])
    n = [v << (L - 1) for v in p["n0"]]
    h = [(p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    ue = np.asarray(p["u_exact"])
    coarse = inputs.variable_box(levels=L - 1, rtol=1e-9)
    e_f = _max_err(_np(s.get(E.ECMG_VEC_U)), ue)
    e_c = _max_err(_np(s.get(E.ECMG_VEC_U, L - 2)), coarse["u_exact"])
    assert 3.6 < e_c / e_f < 4.4, (e_c, e_f)
    # extrapolation improves on U (its fourth order needs algebraic errors below h^4, far under
    # what rtol = 1e-9 leaves at this size), and equals the oracle's EXP_true at sampled nodes
    Ut = _np(s.get(E.ECMG_VEC_UTILDE))
    assert _max_err(Ut, ue) < e_f, (_max_err(Ut, ue), e_f)
    nodes = _sample_nodes(n, 400, 2)
    want_t = oracle_mod.exp_true_at(n, _np(s.get(E.ECMG_VEC_U)).ravel(), _np(s.get(E.ECMG_VEC_U, L - 2)).ravel(),
                                    nodes)
    assert np.abs(_at(Ut, n, nodes) - want_t).max() <= 1e-13 * np.abs(want_t).max()
    x = inputs.random_vector(1024, (n[2] + 1, n[1] + 1, n[0] + 1))
    want = oracle_mod.apply_at(n, h, np.asarray(p["beta"]).ravel(), p["face_bc"], p["alpha"], x.ravel(), nodes)
    got = _at(_np(s.apply(torch.tensor(x, device="cuda"))), n, nodes)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    s.close()


def test_batched_workload_full_size(E, oracle_mod):
    """The batched workload of bench.py: every problem reaches the tolerance, and the residual
    b - A U recomputed by the oracle at sampled nodes of each finest level is within it."""
    import torch
    probs = inputs.batch_problems()
    dev = []
    for q in probs:
        d = dict(q)
        d["beta"] = torch.as_tensor(q["beta"]).cuda()
        d["f"] = torch.as_tensor(q["f"]).cuda()
        dev.append(d)
    bs = E.BatchSolver(dev, rtol=1e-8)
    stats, status = bs.solve()
    assert status == 0
    for i, q in enumerate(probs[:16]):
        L = q["levels"]
        assert stats[i]["rel_res"][L - 1] <= 1e-8
        n = [v << (L - 1) for v in q["n0"]]
        h = [(q["hi"][a] - q["lo"][a]) / n[a] for a in range(3)]
        U = _np(bs.get(i, E.ECMG_VEC_U)).ravel()
        b = _np(bs.get(i, E.ECMG_VEC_B)).ravel()
        nodes = [t for t in _sample_nodes(n, 200, 10 + i) if all(0 < t[a] < n[a] for a in range(3))]
        r = _at(b, n, nodes) - oracle_mod.apply_at(n, h, q["beta"].ravel(), q["face_bc"], q["alpha"], U, nodes)
        # every component of a residual with ||r|| <= 1e-8 ||f_h|| is at most that
        assert np.abs(r).max() <= 1e-8 * stats[i]["rhs_norm"][L - 1] * 1.0001, (i, np.abs(r).max())
    for i in range(len(probs)):
        assert stats[i]["rel_res"][probs[i]["levels"] - 1] <= 1e-8
    bs.close()


def test_jump_singular_full_size_mixed(E, oracle_mod):
    """Configuration 5 at 1024 x 512 x 512 elements, MIXED, rtol 1e-8 (data evaluated on the
    device)."""
    import torch
    p = inputs.jump_singular(levels=7, rtol=1e-8, device="cuda")
    L = p["levels"]
    s = E.solver_from_problem(p, precision=E.ECMG_MIXED, autotune=1)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, L):
        assert st["rel_res"][l] <= p["rtol"] * 1.0001, (l, st["rel_res"])
    # at rtol 1e-8 with contrast 100 and h = 1/512 the algebraic error (~5e-5) exceeds the
    # discretisation error, so the error is only bounded here; the residual is checked below
    u = p["u_exact"]
    assert (s.get(E.ECMG_VEC_U) - u).abs().max().item() < 1e-3
    n = [v << (L - 1) for v in p["n0"]]
    h = [(p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    nodes = _sample_nodes(n, 300, 5)
    x = inputs.random_vector(77, (n[2] + 1, n[1] + 1, n[0] + 1))
    beta = p["beta"].cpu().numpy().ravel()
    want = oracle_mod.apply_at(n, h, beta, p["face_bc"], p["alpha"], x.ravel(), nodes)
    got = _at(_np(s.apply(torch.tensor(x, device="cuda"))), n, nodes)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # b - A U recomputed by the oracle at sampled free nodes is within the residual test
    U = _np(s.get(E.ECMG_VEC_U)).ravel()
    b = _np(s.get(E.ECMG_VEC_B)).ravel()
    free = [t for t in nodes if t[0] < n[0] and all(0 < t[a] < n[a] for a in (1, 2))]
    r = _at(b, n, free) - oracle_mod.apply_at(n, h, beta, p["face_bc"], p["alpha"], U, free)
    assert np.abs(r).max() <= p["rtol"] * st["rhs_norm"][L - 1] * 1.0001, np.abs(r).max()
    s.close()


def test_jump_singular_full_size_single_pass(E, oracle_mod):
    """Configuration 5 with the single-pass MIXED step on its general path (variable beta, a
    Robin face): the residual test on every level, and b - A U recomputed by the oracle at
    sampled free nodes within the test."""
    p = inputs.jump_singular(levels=7, rtol=1e-8, device="cuda")
    L = p["levels"]
    s = E.solver_from_problem(p, precision=E.ECMG_MIXED, autotune=1, cg_form=E.ECMG_CG_SINGLE_PASS)
    st, status = s.solve()
    assert status == 0, st
    for l in range(2, L):
        assert st["rel_res"][l] <= p["rtol"] * 1.0001, (l, st["rel_res"])
    assert (s.get(E.ECMG_VEC_U) - p["u_exact"]).abs().max().item() < 1e-3
    n = [v << (L - 1) for v in p["n0"]]
    h = [(p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    beta = p["beta"].cpu().numpy().ravel()
    U = _np(s.get(E.ECMG_VEC_U)).ravel()
    b = _np(s.get(E.ECMG_VEC_B)).ravel()
    free = [t for t in _sample_nodes(n, 300, 6) if t[0] < n[0] and all(0 < t[a] < n[a] for a in (1, 2))]
    r = _at(b, n, free) - oracle_mod.apply_at(n, h, beta, p["face_bc"], p["alpha"], U, free)
    assert np.abs(r).max() <= p["rtol"] * st["rhs_norm"][L - 1] * 1.0001, np.abs(r).max()
    s.close()


def test_problem2_full_size_against_paper(E):
    """Problem 2 at the paper's finest grid 640 x 256 x 320 (MIXED, eps 1e-12): the errors the
    paper prints for that row (tables 'table3'/'table4'), ||U-u|| to 2 % and ||W-U|| to 10 %."""
    import json
    import os
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "problem2_tables.json")))
    want = tab["rows"]["640x256x320"]
    p = inputs.paper_problem2(levels=7, rtol=1e-12)
    s = E.solver_from_problem(p, precision=E.ECMG_MIXED)
    st, status = s.solve()
    assert status == 0, st
    assert st["rel_res"][6] <= 1e-12 * 1.01
    U = _np(s.get(E.ECMG_VEC_U))
    W = _np(s.get(E.ECMG_VEC_W))
    ue = np.asarray(p["u_exact"])
    e = U - ue
    assert np.abs(e).max() == pytest.approx(want["U_inf"], rel=0.02)
    assert np.sqrt(np.mean(e * e)) == pytest.approx(want["U_L2"], rel=0.02)
    assert np.abs(W - U).max() == pytest.approx(want["WU_inf"], rel=0.10)
    s.close()
