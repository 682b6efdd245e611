"""Pins of the oracle's extrapolation operators (Sec. 4.2-4.3) against the paper's printed
formulas and against exactness properties that follow from the asymptotic expansion (asy)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_formulas.json")))


def _frac(p):
    return float(Fraction(p[0], p[1]))


def _paper_node(m):
    """(a, b, c) of the paper's node number m = 1 + a + 5b + 25c."""
    m -= 1
    return (m % 5, (m // 5) % 5, m // 25)


def test_serendipity_node_list_matches_paper_numbering(oracle_mod):
    nodes = [tuple(v) for v in oracle_mod.serendipity_nodes()]
    g = GOLD["node_numbering"]
    want = [_paper_node(m) for m in g["corners"] + g["x_midpoints"] + g["y_midpoints"] + g["z_midpoints"]]
    assert nodes == want


def test_w35_weights(oracle_mod):
    g = GOLD["w35"]
    N = oracle_mod.serendipity(*g["point_natural_coords"])
    nodes = [tuple(v) for v in oracle_mod.serendipity_nodes()]
    # node 35 itself sits at natural coordinates (1, -1/2, -1/2)
    a, b, c = _paper_node(35)
    assert ((a - 2) / 2, (b - 2) / 2, (c - 2) / 2) == tuple(g["point_natural_coords"])
    want = np.zeros(20)
    for m, w in zip(g["paper_node_numbers"], g["weights"]):
        want[nodes.index(_paper_node(m))] = _frac(w)
    assert np.allclose(N, want, atol=1e-15)


def test_serendipity_kronecker_unity_and_quadratic_reproduction(oracle_mod):
    nodes = oracle_mod.serendipity_nodes()
    nat = (nodes - 2) / 2.0
    for m in range(20):
        N = oracle_mod.serendipity(*nat[m])
        assert np.allclose(N, np.eye(20)[m], atol=1e-15)
    rng = np.random.default_rng(0)
    mons = [lambda x, y, z: 1 + 0 * x, lambda x, y, z: x, lambda x, y, z: y, lambda x, y, z: z,
            lambda x, y, z: x * x, lambda x, y, z: y * y, lambda x, y, z: z * z,
            lambda x, y, z: x * y, lambda x, y, z: y * z, lambda x, y, z: x * z,
            lambda x, y, z: x * y * z, lambda x, y, z: x * x * y, lambda x, y, z: z * z * x]
    for pt in rng.uniform(-1, 1, (10, 3)):
        N = oracle_mod.serendipity(*pt)
        for f in mons:
            vals = np.array([f(*q) for q in nat])
            assert N @ vals == pytest.approx(f(*pt), abs=1e-14)


def _level_values(n, box, fn):
    z, y, x = np.meshgrid(*[np.linspace(0, box[a], n[a] + 1) for a in (2, 1, 0)], indexing="ij")
    return fn(x, y, z).ravel()


@pytest.mark.parametrize("variant", ["serendipity20", "lagrange27"])
def test_exp_finite_exact_on_quadratic_plus_h2(oracle_mod, variant):
    """U^k = q + A h_k^2 with q quadratic and A affine on levels l-2, l-1 gives W = q + A h_l^2
    on level l exactly: the corner and midpoint formulas cancel the h^2 term (eq. (asy)) and
    both interpolations reproduce quadratics."""
    rng = np.random.default_rng(11)
    c = rng.uniform(-1, 1, 13)
    q = lambda x, y, z: (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y
                         + c[6] * z * z + c[7] * x * y + c[8] * y * z + c[9] * x * z)
    A = lambda x, y, z: c[10] * x - c[11] * y + c[12] * z + 0.3
    n = [8, 4, 12]
    box = (1.0, 0.6, 1.3)
    hl = box[0] / n[0]
    U = {}
    for s in (1, 2):
        nk = [v // (2 ** s) for v in n]
        hk = hl * 2 ** s
        U[s] = _level_values(nk, box, lambda x, y, z: q(x, y, z) + A(x, y, z) * hk * hk)
    fn = oracle_mod.exp_finite if variant == "serendipity20" else oracle_mod.exp_finite27
    W = fn(n, U[1], U[2])
    want = _level_values(n, box, lambda x, y, z: q(x, y, z) + A(x, y, z) * hl * hl)
    assert np.abs(W - want).max() < 1e-13


def test_exp_finite_1d_formulas(oracle_mod):
    """Data varying along x only: EXP_finite reduces to eqs. (jiedian), (zhongdian), (sifen1)
    and (sifen2) at the five points of each coarse interval."""
    g = GOLD
    rng = np.random.default_rng(4)
    n = [8, 4, 4]
    u1 = rng.uniform(-1, 1, n[0] // 2 + 1)   # level l-1 values along x
    u0 = rng.uniform(-1, 1, n[0] // 4 + 1)   # level l-2 values along x
    U1 = np.broadcast_to(u1, (n[2] // 2 + 1, n[1] // 2 + 1, u1.size)).ravel()
    U0 = np.broadcast_to(u0, (n[2] // 4 + 1, n[1] // 4 + 1, u0.size)).ravel()
    for fn in (oracle_mod.exp_finite, oracle_mod.exp_finite27):
        W = fn(n, U1, U0).reshape(n[2] + 1, n[1] + 1, n[0] + 1)
        assert np.allclose(W, W[0:1, 0:1, :], atol=1e-14)
        w = W[0, 0]
        for j in range(n[0] // 4):
            a, b, m = u1[2 * j], u1[2 * j + 2], u1[2 * j + 1]
            A0, B0 = u0[j], u0[j + 1]
            jd = g["jiedian"]
            assert w[4 * j] == pytest.approx(_frac(jd["U1"]) * a + _frac(jd["U0"]) * A0, abs=1e-14)
            zd = g["zhongdian"]
            assert w[4 * j + 2] == pytest.approx(
                _frac(zd["U1_mid"]) * m + _frac(zd["U1_ends"]) * (a + b) + _frac(zd["U0_ends"]) * (A0 + B0), abs=1e-14)
            for key, off in (("sifen1", 1), ("sifen2", 3)):
                s = g[key]
                want = (_frac(s["U1_j"]) * a + _frac(s["U1_mid"]) * m + _frac(s["U1_j1"]) * b
                        + _frac(s["U0_j"]) * A0 + _frac(s["U0_j1"]) * B0)
                assert w[4 * j + off] == pytest.approx(want, abs=1e-14)


def test_exp_true_formulas_and_exactness(oracle_mod):
    """(i) eq. (t1) at coarse nodes and eq. (chenlin) at edge centres, with the printed
    coefficients; (ii) U^k = u + A h_k^2 with A trilinear gives U~ = u exactly at every fine
    node, for arbitrary u."""
    g = GOLD
    rng = np.random.default_rng(9)
    n = [6, 4, 8]
    U1 = rng.uniform(-1, 1, (n[2] + 1, n[1] + 1, n[0] + 1))
    U0 = rng.uniform(-1, 1, (n[2] // 2 + 1, n[1] // 2 + 1, n[0] // 2 + 1))
    Ut = oracle_mod.exp_true(n, U1.ravel(), U0.ravel()).reshape(U1.shape)
    t1 = g["t1"]
    assert np.allclose(Ut[::2, ::2, ::2], _frac(t1["U1"]) * U1[::2, ::2, ::2] + _frac(t1["U0"]) * U0, atol=1e-14)
    cl = g["chenlin"]
    d = U1[::2, ::2, ::2] - U0
    want = _frac(cl["U1_mid"]) * U1[::2, ::2, 1::2] + _frac(cl["U1_ends"]) * (U1[::2, ::2, :-1:2] + U1[::2, ::2, 2::2]) \
        + _frac(cl["U0_ends"]) * (U0[:, :, :-1] + U0[:, :, 1:])
    assert np.allclose(Ut[::2, ::2, 1::2], want, atol=1e-14)
    # exactness
    box = (0.6, 0.4, 0.8)
    hl = box[0] / n[0]
    c = rng.uniform(-1, 1, 8)
    A = lambda x, y, z: c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z + c[7] * x * y * z
    u = lambda x, y, z: np.sin(3 * x) * np.exp(y) + z ** 3
    V1 = _level_values(n, box, lambda x, y, z: u(x, y, z) + A(x, y, z) * hl ** 2)
    V0 = _level_values([v // 2 for v in n], box, lambda x, y, z: u(x, y, z) + A(x, y, z) * (2 * hl) ** 2)
    Ut2 = oracle_mod.exp_true(n, V1, V0)
    assert np.abs(Ut2 - _level_values(n, box, u)).max() < 1e-13


@pytest.mark.parametrize("variant", [0, 1])
def test_orders_of_w_and_extrapolated_solution(oracle_mod, variant):
    """Manufactured u = exp(x+y+z), 4^3 -> 32^3, tight tolerance: ||W-U|| has order 3
    (Sec. 4.4) and ||U~-u|| order 4 (eq. (t1)/(chenlin)), as in the tables of Sec. 5."""
    p = inputs.exp_cube(levels=4, rtol=1e-12)
    lv, st = oracle_mod.ecmg(p, 1e-12, exp_variant=variant)
    assert st["status"] == 0
    wu, ut = [], []
    for l in (2, 3):
        s = 1 << (3 - l)
        ue = p["u_exact"][::s, ::s, ::s]
        wu.append(oracle_mod.norms(lv[l]["W"], lv[l]["U"])[1])
        ut.append(oracle_mod.norms(lv[l]["Ut"], ue)[1])
    assert abs(np.log2(wu[0] / wu[1]) - 3.0) < 0.15
    assert abs(np.log2(ut[0] / ut[1]) - 4.0) < 0.2
