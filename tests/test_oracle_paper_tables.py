"""The whole oracle (Alg. 4) against the numbers the paper prints for Problem 1 (Sec. 5).

The load is the exact functional int f phi_i (f_mode 1). With the 27-node Lagrange variant
of EXP_finite (the Remark in Sec. 4.3) the oracle reproduces the printed iteration counts,
final relative residuals, ||U-u||, ||W-U|| and r_h; the 20-node Serendipity variant gives the
same ||U-u|| and ||W-U|| within 6 % (L2) and 30 % (max). The extrapolated solution U~ comes out
4-6 % above the printed values under every reading tried, so that column is a soft pin.
"""
import json
import os

import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

TAB = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "problem1_tables.json")))


def _run(oracle_mod, eps, variant):
    p = inputs.paper_problem1(levels=4, rtol=eps)
    lv, st = oracle_mod.ecmg(p, eps, exp_variant=variant)
    assert st["status"] == 0
    rows = {}
    for l, size in ((2, "32"), (3, "64")):
        s = 1 << (3 - l)
        ue = p["u_exact"][::s, ::s, ::s]
        U, W, Ut = lv[l]["U"], lv[l]["W"], lv[l]["Ut"]
        eU, eT, eW = oracle_mod.norms(U, ue), oracle_mod.norms(Ut, ue), oracle_mod.norms(W, U)
        rows[size] = dict(iters=st["iters"][l], RRe=st["rel_res"][l], U_L2=eU[1], U_inf=eU[0],
                          Ut_L2=eT[1], Ut_inf=eT[0], WU_L2=eW[1], WU_inf=eW[0], r_h=eW[1] / eU[1])
    return rows


@pytest.mark.parametrize("eps_key,eps", [("eps_1e-8", 1e-8), ("eps_1e-9", 1e-9), ("eps_1e-10", 1e-10)])
def test_problem1_lagrange27_reproduces_tables(oracle_mod, eps_key, eps):
    rows = _run(oracle_mod, eps, 1)
    for size, want in TAB[eps_key].items():
        if size.startswith("_") or size == "citation":
            continue
        got = rows[size]
        assert got["iters"] == want["iters"], (size, got["iters"])
        for k, tol in (("RRe", 0.02), ("U_L2", 0.01), ("U_inf", 0.01), ("WU_L2", 0.01),
                       ("r_h", 0.01), ("WU_inf", 0.01)):
            if k in want:
                assert got[k] == pytest.approx(want[k], rel=tol), (size, k, got[k])
        for k in ("Ut_L2", "Ut_inf"):
            if k in want:
                assert got[k] == pytest.approx(want[k], rel=0.10), (size, k, got[k])


def test_problem1_serendipity20_close_to_tables(oracle_mod):
    rows = _run(oracle_mod, 1e-9, 0)
    for size, want in TAB["eps_1e-9"].items():
        if size == "citation":
            continue
        got = rows[size]
        assert got["U_L2"] == pytest.approx(want["U_L2"], rel=0.01)
        assert got["U_inf"] == pytest.approx(want["U_inf"], rel=0.01)
        assert got["WU_L2"] == pytest.approx(want["WU_L2"], rel=0.06)
        assert got["WU_inf"] == pytest.approx(want["WU_inf"], rel=0.30)
        assert abs(got["iters"] - want["iters"]) <= 2


@pytest.mark.parametrize("eps_key,eps", [("1e-8", 1e-8), ("1e-9", 1e-9), ("1e-10", 1e-10)])
def test_problem1_ecmg_cg_reproduces_tables(oracle_mod, eps_key, eps):
    """ECMG_cg (Alg. 4 with line 8 plain CG, Sec. 3): the printed CG iteration counts on the 32^3
    and 64^3 grids, to one iteration (same 27-node variant and exact load as above)."""
    p = inputs.paper_problem1(levels=4, rtol=eps)
    lv, st = oracle_mod.ecmg(p, eps, exp_variant=1, precond=0)
    assert st["status"] == 0
    want = TAB["ecmg_cg_iters"][eps_key]
    for l, size in ((2, "32"), (3, "64")):
        assert abs(st["iters"][l] - want[size]) <= 1, (eps_key, size, st["iters"][l], want[size])
        assert st["rel_res"][l] <= eps


def test_fixed_schedule_follows_eq_ee(oracle_mod):
    """Alg. 3's fixed step counts, eq. (ee): m_j = ceil(m_L beta^(L-j)) on the levels above the two
    direct ones (j = 1 .. L, finest j = L gets m_L), e.g. m_j = 4 * 4^(L-j)."""
    assert [oracle_mod.schedule_steps(7, l, 4, 4.0) for l in range(2, 7)] == [1024, 256, 64, 16, 4]
    assert [oracle_mod.schedule_steps(5, l, 3, 2.5) for l in range(2, 5)] == [19, 8, 3]
    p = inputs.exp_cube(levels=5, rtol=1e-10)
    lv, st = oracle_mod.ecmg(p, 1e-10, schedule=1, mL=2, sched_beta=3.0, precond=0)
    assert st["status"] == 0
    assert st["iters"][2:] == [18, 6, 2]
    # more steps shrink the residual (a fixed count, not a tolerance, ends each level)
    lv2, st2 = oracle_mod.ecmg(p, 1e-10, schedule=1, mL=8, sched_beta=3.0, precond=0)
    assert st2["rel_res"][4] < st["rel_res"][4]


TAB2 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "problem2_tables.json")))


def test_problem2_reproduces_tables(oracle_mod):
    """Problem 2 (anisotropic elements, coarsest 10x4x5, eps 1e-12): the oracle's discretisation
    and extrapolation errors against tables 'table3'/'table4' on the three coarsest printed rows.
    ||U-u|| to 1 %, ||U~-u|| to 3 %, ||W-U|| and r_h to 6 %; the printed iteration counts are
    10-25 % below the oracle's (the paper's JCG details are not stated), so only a 30 % band."""
    p = inputs.paper_problem2(levels=5, rtol=1e-12)
    lv, st = oracle_mod.ecmg(p, 1e-12, exp_variant=0)
    assert st["status"] == 0
    L = p["levels"]
    for l, key in ((2, "40x16x20"), (3, "80x32x40"), (4, "160x64x80")):
        want = TAB2["rows"][key]
        s = 1 << (L - 1 - l)
        ue = p["u_exact"][::s, ::s, ::s]
        eU, eT, eW = oracle_mod.norms(lv[l]["U"], ue), oracle_mod.norms(lv[l]["Ut"], ue), oracle_mod.norms(lv[l]["W"], lv[l]["U"])
        got = dict(U_inf=eU[0], U_L2=eU[1], Ut_inf=eT[0], Ut_L2=eT[1], WU_inf=eW[0], WU_L2=eW[1], r_h=eW[1] / eU[1])
        for k, tol in (("U_inf", 0.01), ("U_L2", 0.01), ("Ut_inf", 0.03), ("Ut_L2", 0.03), ("WU_inf", 0.06),
                       ("WU_L2", 0.06), ("r_h", 0.06)):
            assert got[k] == pytest.approx(want[k], rel=tol), (key, k, got[k], want[k])
        assert abs(st["iters"][l] - want["iters"]) <= 0.3 * want["iters"], (key, st["iters"][l])
        assert st["rel_res"][l] <= 1e-12
