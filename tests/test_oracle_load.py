"""Pins of the oracle's load functional of Sec. 2 (b_i = int f phi_i + face terms, by tensor Gauss
quadrature element by element) against closed forms, and of the LOAD-mode inputs the problem
generators compute (cos_cube, Problems 1 and 2 of Sec. 5, the coefficient-jump box) against it."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs

PI = np.pi


def _exact_hat_integrals(coef, n, lo, hi):
    """int poly(t) phi_i(t) dt for the hats of a uniform n-interval grid on [lo, hi], from exact
    antiderivatives of the polynomial times each linear piece of the hat."""
    P = np.polynomial.Polynomial
    p = P(coef)
    h = (hi - lo) / n
    x = lo + np.arange(n + 1) * h
    out = np.zeros(n + 1)
    for i in range(n + 1):
        if i > 0:
            F = (p * P([-x[i - 1], 1.0]) / h).integ()
            out[i] += F(x[i]) - F(x[i - 1])
        if i < n:
            F = (p * P([x[i + 1], -1.0]) / h).integ()
            out[i] += F(x[i + 1]) - F(x[i])
    return out


def _outer(iz, iy, ix):
    return iz[:, None, None] * iy[None, :, None] * ix[None, None, :]


def test_constant_f_and_g_give_the_hat_volumes_and_areas(oracle_mod):
    n, lo, hi = (4, 3, 5), (0.0, -1.0, 0.5), (2.0, 0.5, 1.0)
    one = lambda x, y, z: np.ones_like(x * y * z)
    b = oracle_mod.load_functional(n, lo, hi, one, q=2)
    hv = []
    for a in range(3):
        h = (hi[a] - lo[a]) / n[a]
        v = np.full(n[a] + 1, h)
        v[0] = v[-1] = 0.5 * h
        hv.append(v)
    np.testing.assert_allclose(b, _outer(hv[2], hv[1], hv[0]), rtol=1e-14, atol=0)
    assert b.sum() == pytest.approx(np.prod([hi[a] - lo[a] for a in range(3)]), rel=1e-14)
    # a constant g on the face y = y_1 adds the face hat areas on that node plane only
    zero = lambda x, y, z: np.zeros_like(x * y * z)
    c = oracle_mod.load_functional(n, lo, hi, zero, q=2, faces=[(1, 1, lambda x, y, z: 2.0 + 0.0 * (x * y * z))])
    want = np.zeros_like(c)
    want[:, 1, :] = 2.0 * np.outer(hv[2], hv[0])
    np.testing.assert_allclose(c, want, rtol=1e-14, atol=1e-300)


def test_polynomial_f_matches_exact_integrals(oracle_mod):
    """f = x y^2 - z^3 x + 2 (not separable as one term) with degree <= 4 per axis: the 3-point
    rule is exact, so b equals the sum of the terms' exact outer products. A transposed axis, a
    wrong hat corner or a wrong weight fails it."""
    n, lo, hi = (5, 4, 3), (-0.2, 0.3, 1.0), (0.9, 1.1, 1.6)
    f = lambda x, y, z: x * y * y - z ** 3 * x + 2.0
    b = oracle_mod.load_functional(n, lo, hi, f, q=3)
    I = lambda a, c: _exact_hat_integrals(c, n[a], lo[a], hi[a])
    want = (_outer(I(2, [1.0]), I(1, [0, 0, 1.0]), I(0, [0, 1.0]))
            - _outer(I(2, [0, 0, 0, 1.0]), I(1, [1.0]), I(0, [0, 1.0]))
            + 2.0 * _outer(I(2, [1.0]), I(1, [1.0]), I(0, [1.0])))
    np.testing.assert_allclose(b, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_polynomial_face_term_matches_exact_integrals(oracle_mod):
    n, lo, hi = (3, 4, 5), (0.0, 0.0, 0.0), (1.5, 1.0, 2.0)
    zero = lambda x, y, z: np.zeros_like(x * y * z)
    for axis, idx in ((0, 3), (2, 0), (1, 2)):
        g = lambda x, y, z: (x + 1.0) * (y * y + z) + 0.0 * (x * y * z)
        b = oracle_mod.load_functional(n, lo, hi, zero, q=3, faces=[(axis, idx, g)])
        c = lo[axis] + idx * (hi[axis] - lo[axis]) / n[axis]
        I = lambda a, cf: _exact_hat_integrals(cf, n[a], lo[a], hi[a])
        e = [np.zeros(n[a] + 1) for a in range(3)]
        e[axis][idx] = 1.0
        # g = (x + 1) y^2 + (x + 1) z, with the face's own coordinate fixed at c
        fac1 = [[1.0, 1.0], [0, 0, 1.0], [1.0]]   # (x + 1), y^2, 1
        fac2 = [[1.0, 1.0], [1.0], [0, 1.0]]      # (x + 1), 1, z
        want = np.zeros_like(b)
        for fac in (fac1, fac2):
            parts = []
            for a in range(3):
                if a == axis:
                    parts.append(e[a] * np.polynomial.polynomial.polyval(c, fac[a]))
                else:
                    parts.append(I(a, fac[a]))
            want += _outer(parts[2], parts[1], parts[0])
        np.testing.assert_allclose(b, want, rtol=0, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("name", ["cos_cube", "problem1", "problem2"])
def test_generator_load_functionals_equal_the_oracle_definition(oracle_mod, name):
    """The exact LOAD-mode inputs of the separable workloads (1D hat integrals by 6-point Gauss,
    multiplied out) equal the oracle's element-by-element 6-point rule at <= 16^3."""
    if name == "cos_cube":
        p = inputs.cos_cube(levels=2, n0=(8, 8, 8))
        f = lambda x, y, z: 3.0 * PI * PI * np.cos(PI * x) * np.cos(PI * y) * np.cos(PI * z)
    elif name == "problem1":
        p = inputs.paper_problem1(levels=2, n0=(6, 8, 7))
        f = lambda x, y, z: 0.75 * PI * PI * np.sin(0.5 * PI * x) * np.sin(0.5 * PI * y) * np.sin(0.5 * PI * z)
    else:
        p = inputs.paper_problem2(levels=2, n0=(5, 2, 3))
        f = lambda x, y, z: (2.5 * PI * PI - 1.0) * np.exp(z) * np.sin(1.5 * PI * x) * np.sin(0.5 * PI * y)
    assert p["f_mode"] == 1
    n = inputs.finest(p["n0"], p["levels"])
    want = oracle_mod.load_functional(n, p["lo"], p["hi"], f, q=6)
    got = np.asarray(p["f"])
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())


def test_jump_generator_load_equals_the_oracle_definition(oracle_mod):
    """The coefficient-jump box: f = -beta Laplace(r^1.5) = -3.75 beta r^-1/2 with beta 1 | 100
    across x = 1, the interface term (beta- - beta+) du/dx = -99 * 1.5 x r^-1/2 on x = 1, and the
    Robin datum g_R = alpha u + beta du/dn = r^1.5 on x = 0 (du/dx = 0 there), each by the 3-point
    rule the generator states."""
    p = inputs.jump_singular(levels=3, n0=(4, 2, 2))
    n = inputs.finest(p["n0"], p["levels"])
    r = lambda x, y, z: np.sqrt(x * x + y * y + z * z)
    f = lambda x, y, z: -3.75 * np.where(x < 1.0, 1.0, 100.0) * r(x, y, z) ** -0.5
    g_int = lambda x, y, z: (1.0 - 100.0) * 1.5 * x * r(x, y, z) ** -0.5
    g_rob = lambda x, y, z: r(x, y, z) ** 1.5
    want = oracle_mod.load_functional(n, p["lo"], p["hi"], f, q=3, faces=[(0, n[0] // 2, g_int), (0, 0, g_rob)])
    got = np.asarray(p["f"])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_gauss_point_load_equals_the_functional_with_the_same_rule(oracle_mod):
    """oracle.load_gauss (f given at the Gauss points, ECMG_F_GAUSS) is int f phi_i by the 3-point
    rule: equal to load_functional with q = 3 on a smooth and on a discontinuous f, and the hat
    volumes for constant f."""
    n, lo, hi = (5, 3, 4), (0.0, -1.0, 0.5), (2.0, 0.5, 1.0)
    h = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    for f in (lambda x, y, z: np.exp(x - 2 * y) * np.cos(3 * z),
              lambda x, y, z: np.where(x < 1.0, 1.0, 100.0) * (x * x + y * y + z * z) ** -0.25):
        got = oracle_mod.load_gauss(n, h, inputs.gauss_samples(n, lo, hi, f))
        want = oracle_mod.load_functional(n, lo, hi, f, q=3)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())
    one = oracle_mod.load_gauss(n, h, np.ones((n[2], n[1], n[0], 3, 3, 3)))
    assert one.sum() == pytest.approx(np.prod([hi[a] - lo[a] for a in range(3)]), rel=1e-14)
    assert one[0, 0, 0] == pytest.approx(h[0] * h[1] * h[2] / 8.0, rel=1e-14)
