"""The compact input forms of the load assembly on the device, against the oracle's definitions
(through the C ABI):

  - f at the points of the 3x3x3 Gauss rule of every finest element (ECMG_F_GAUSS): the load
    int f phi_i of Sec. 2 with that rule, plus the face mass of the nodal g_R on Robin faces, and
    its restrictions P^T b on the coarse levels (oracle.load_gauss, oracle.load_nodal with f = 0,
    oracle.restrict_load);
  - separable f with a variable (dense) beta;
  - every compact form inside a batch (ecmg_create_batched).

Bars as in test_gpu_parity.py: set-up vectors 1e-13 relative, FP64 solves 1e-10 and iteration
counts within 1, MIXED solves 1e-7 relative to the oracle's solution."""
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


def _level_h(p, l):
    return [(p["hi"][a] - p["lo"][a]) / (p["n0"][a] << l) for a in range(3)]


GAUSS = {
    "exp_cube_gauss": lambda: inputs.exp_cube_gauss(levels=4, n0=(4, 4, 4)),
    "random_gauss_robin": lambda: inputs.random_gauss(31, n0=(2, 3, 2), levels=4, face_bc=[1, 0, 1, 0, 1, 0]),
    "random_gauss_dirichlet": lambda: inputs.random_gauss(32, n0=(3, 2, 2), levels=3, face_bc=[0] * 6),
}


def _dense_from_gauss(oracle_mod, p):
    """The same problem with the finest load functional assembled by the oracle."""
    L = p["levels"]
    n = inputs.finest(p["n0"], L)
    h = _level_h(p, L - 1)
    b = oracle_mod.load_gauss(n, h, p["f"]).ravel()
    if p.get("gR") is not None and any(bc == 1 for bc in p["face_bc"]):
        zero = np.zeros((n[2] + 1) * (n[1] + 1) * (n[0] + 1))
        b = b + np.ravel(oracle_mod.load_nodal(n, h, zero, p["face_bc"], np.asarray(p["gR"]).ravel()))
    d = dict(p)
    d["f"] = b.reshape(n[2] + 1, n[1] + 1, n[0] + 1)
    d["f_mode"] = 1
    d["gR"] = None
    return d


@pytest.mark.parametrize("name", sorted(GAUSS))
def test_gauss_point_load_matches_oracle_on_every_level(E, oracle_mod, name):
    p = GAUSS[name]()
    d = _dense_from_gauss(oracle_mod, p)
    s = E.solver_from_problem(p, precision=0)
    s.solve()
    L = p["levels"]
    load = np.asarray(d["f"]).ravel()
    for l in range(L - 1, -1, -1):
        n = [v << l for v in p["n0"]]
        if l < L - 1:
            load = oracle_mod.restrict_load(n, load)
        b = _np(s.get(E.ECMG_VEC_B, l)).ravel()
        assert np.abs(b - load).max() <= 1e-13 * np.abs(load).max(), (l, np.abs(b - load).max())
    s.close()


@pytest.mark.parametrize("name", sorted(GAUSS))
@pytest.mark.parametrize("precision", [0, 1])
def test_gauss_point_solve_matches_oracle(E, oracle_mod, name, precision):
    p = GAUSS[name]()
    d = _dense_from_gauss(oracle_mod, p)
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


def test_gauss_point_load_converges_at_second_order(E):
    """With f given at the Gauss points the FE solution converges to u = e^{x+y+z} at order 2."""
    errs = []
    for levels in (3, 4, 5):
        p = inputs.exp_cube_gauss(levels=levels, n0=(4, 4, 4))
        s = E.solver_from_problem(p, precision=0)
        s.solve()
        errs.append(np.abs(_np(s.get(E.ECMG_VEC_U)) - np.asarray(p["u_exact"])).max())
        s.close()
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4, errs


def test_separable_f_with_variable_beta_matches_oracle(E, oracle_mod):
    """Separable f (the compact load form) with a dense lognormal beta: the load is the oracle's
    per-element definition and the solves match the oracle's."""
    import torch
    p = inputs.random_separable(41, n0=(2, 3, 2), levels=4, face_bc=[0, 1, 1, 0, 1, 0])
    L = p["levels"]
    n = inputs.finest(p["n0"], L)
    rng = np.random.default_rng(41)
    beta = np.exp(np.clip(rng.standard_normal((n[2], n[1], n[0])), -1.5, 1.5))
    p["beta"] = beta
    p["beta_const"] = 0.0
    d = dict(p)
    d["f"] = oracle_mod.load_separable(n, _level_h(p, L - 1), p["f_terms"], p["f"])
    d["f_mode"] = 1
    d["gD"] = oracle_mod.nodal_separable(n, p["gD_terms"], p["gD"]) if p["gD_terms"] else None
    for k in ("f_terms", "gD_terms", "beta_const"):
        d.pop(k)
    lv, ost = oracle_mod.ecmg(d, d["rtol"])
    assert ost["status"] == 0
    for precision in (0, 1):
        s = E.solver_from_problem(p, precision=precision)
        st, status = s.solve()
        assert status == 0, st
        assert np.array_equal(_np(s.get(E.ECMG_VEC_BETA)).ravel(), beta.ravel())
        b = _np(s.get(E.ECMG_VEC_B)).ravel()
        want = np.asarray(d["f"]).ravel()
        assert np.abs(b - want).max() <= 1e-13 * np.abs(want).max()
        for l in range(2, L):
            assert st["rel_res"][l] <= p["rtol"] * 1.01
            U = _np(s.get(E.ECMG_VEC_U, l))
            assert _rel(U, lv[l]["U"]) <= (1e-10 if precision == 0 else 1e-7), (precision, l)
        s.close()
    torch.cuda.synchronize()


def _batch_device(p):
    import torch
    q = dict(p)
    for k in ("beta", "f", "gD", "gR"):
        v = p.get(k)
        q[k] = None if v is None else torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64).cuda()
    return q


def test_compact_inputs_in_a_batch_match_the_oracle(E, oracle_mod):
    """A batch mixing every input form -- dense nodal f, separable f and g_D with one beta, f at
    the Gauss points with nodal g_R -- solved together; each problem against the oracle on its
    dense assembly, and the same FP32 steps (within 2) as the single-problem solve."""
    import torch
    probs = [inputs.exp_cube(levels=4, rtol=1e-10),
             inputs.cos_cube_compact(levels=4, n0=(4, 4, 4), rtol=1e-10),
             inputs.random_separable(22, n0=(2, 3, 2), levels=4, gD_terms=1, face_bc=[0, 1, 1, 0, 1, 0]),
             GAUSS["exp_cube_gauss"](),
             GAUSS["random_gauss_robin"]()]
    dense = []
    for p in probs:
        if p["f_mode"] == 2:
            L = p["levels"]
            n = inputs.finest(p["n0"], L)
            d = dict(p)
            d["f"] = oracle_mod.load_separable(n, _level_h(p, L - 1), p["f_terms"], p["f"])
            d["f_mode"] = 1
            d["gD"] = oracle_mod.nodal_separable(n, p["gD_terms"], p["gD"]) if p["gD_terms"] else None
            d["beta"] = np.full((n[2], n[1], n[0]), p["beta_const"])
            dense.append(d)
        elif p["f_mode"] == 3:
            dense.append(_dense_from_gauss(oracle_mod, p))
        else:
            dense.append(p)
    dev = [_batch_device(p) for p in probs]
    for q, p in zip(dev, probs):
        q["f_terms"] = p.get("f_terms", 0)
        q["gD_terms"] = p.get("gD_terms", 0)
        q["beta_const"] = p.get("beta_const", 0.0)
    bs = E.BatchSolver(dev, rtol=1e-10)
    stats, status = bs.solve()
    assert status == 0, stats
    for i, (p, d) in enumerate(zip(probs, dense)):
        lv, ost = oracle_mod.ecmg(d, 1e-10)
        L = p["levels"]
        b = _np(bs.get(i, E.ECMG_VEC_B)).ravel()
        want = np.asarray(d["f"]).ravel()
        if p["f_mode"] != 0:
            assert np.abs(b - want).max() <= 1e-13 * np.abs(want).max(), i
        for l in range(2, L):
            assert stats[i]["rel_res"][l] <= 1e-10, (i, l, stats[i]["rel_res"])
            U = _np(bs.get(i, E.ECMG_VEC_U, l))
            assert _rel(U, lv[l]["U"]) <= 1e-7, (i, l, _rel(U, lv[l]["U"]))
        single = E.solver_from_problem(p, precision=1, rtol=1e-10, cg_form=E.ECMG_CG_TWO_PASS)
        sst, sstatus = single.solve()
        assert sstatus == 0
        single.close()
        for l in range(2, L):
            assert abs(stats[i]["iters"][l] - sst["iters"][l]) <= 2, (i, l, stats[i]["iters"], sst["iters"])
    bs.close()
    torch.cuda.synchronize()
