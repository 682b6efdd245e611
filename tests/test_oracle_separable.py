"""Pins of the oracle's separable load assembly (the definition b_i = int f phi_i of Sec. 2 by
tensor Gauss quadrature) against closed forms and the exact coarse restriction."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs


def _h(p, l):
    return [(p["hi"][a] - p["lo"][a]) / (p["n0"][a] << l) for a in range(3)]


def _exact_hat_integrals(coef, n, lo, hi):
    """int poly(t) phi_i(t) dt over [lo, hi] for the hats of a uniform n-interval grid, by exact
    antiderivatives of the polynomial times each linear piece."""
    P = np.polynomial.Polynomial
    p = P(coef)
    h = (hi - lo) / n
    x = lo + np.arange(n + 1) * h
    out = np.zeros(n + 1)
    for i in range(n + 1):
        if i > 0:  # rising piece (t - x_{i-1}) / h on [x_{i-1}, x_i]
            F = (p * P([-x[i - 1], 1.0]) / h).integ()
            out[i] += F(x[i]) - F(x[i - 1])
        if i < n:  # falling piece (x_{i+1} - t) / h on [x_i, x_{i+1}]
            F = (p * P([x[i + 1], -1.0]) / h).integ()
            out[i] += F(x[i + 1]) - F(x[i])
    return out


def test_constant_f_gives_the_hat_volumes(oracle_mod):
    n, lo, hi = (5, 3, 4), (0.0, -1.0, 2.0), (1.0, 0.5, 3.0)
    one = lambda t: np.ones_like(t)
    s = inputs.separable_samples(n, lo, hi, [(one, one, one)])
    h = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    b = oracle_mod.load_separable(n, h, 1, s)
    v = []
    for a in range(3):
        w = np.full(n[a] + 1, h[a])
        w[0] = w[-1] = 0.5 * h[a]
        v.append(w)
    want = v[2][:, None, None] * v[1][None, :, None] * v[0][None, None, :]
    np.testing.assert_allclose(b, want, rtol=1e-14, atol=0)
    assert b.sum() == pytest.approx(np.prod([hi[a] - lo[a] for a in range(3)]), rel=1e-14)


def test_polynomial_terms_match_exact_integrals(oracle_mod):
    """Three terms of random degree-<= 4 factors on a box with unequal intervals per axis: the
    3-point rule is exact, so b equals the sum over terms of outer products of exact 1D hat
    integrals (any transposed axis, wrong corner or weight fails)."""
    rng = np.random.default_rng(5)
    n, lo, hi = (6, 4, 5), (-0.3, 0.1, 1.0), (0.9, 1.7, 1.6)
    terms, coefs = [], []
    for _ in range(3):
        cs = [rng.standard_normal(5) for _ in range(3)]
        coefs.append(cs)
        terms.append(tuple((lambda t, c=c: np.polynomial.polynomial.polyval(t, c)) for c in cs))
    s = inputs.separable_samples(n, lo, hi, terms)
    assert s.shape == (3, 3 * sum(n))
    h = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    b = oracle_mod.load_separable(n, h, 3, s)
    want = np.zeros_like(b)
    for cs in coefs:
        I = [_exact_hat_integrals(cs[a], n[a], lo[a], hi[a]) for a in range(3)]
        want += I[2][:, None, None] * I[1][None, :, None] * I[0][None, None, :]
    np.testing.assert_allclose(b, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_restriction_of_the_fine_load_is_the_coarse_load(oracle_mod):
    """Every coarse hat is a combination of fine hats (prolongation weights 1, 1/2), so the
    restricted fine functional equals the functional on the coarse grid when both are exact."""
    p = inputs.random_separable(11, n0=(2, 3, 2), levels=3)
    L = p["levels"]
    fine = oracle_mod.load_separable(inputs.finest(p["n0"], L), _h(p, L - 1), p["f_terms"], p["f"])
    for l in range(L - 2, -1, -1):
        nc = [v << l for v in p["n0"]]
        fine = oracle_mod.restrict_load(nc, fine.ravel()).reshape(nc[2] + 1, nc[1] + 1, nc[0] + 1)
        direct = oracle_mod.load_separable(nc, _h(p, l), p["f_terms"],
                                           inputs.separable_samples(nc, p["lo"], p["hi"], p["f_factors"]))
        np.testing.assert_allclose(fine, direct, rtol=0, atol=1e-13 * np.abs(direct).max())


def test_nodal_separable_is_the_function_at_the_nodes(oracle_mod):
    p = inputs.random_separable(12, n0=(2, 3, 2), levels=3)
    n = inputs.finest(p["n0"], p["levels"])
    g = oracle_mod.nodal_separable(n, p["gD_terms"], p["gD"])
    x, y, z = (p["lo"][a] + np.arange(n[a] + 1) * (p["hi"][a] - p["lo"][a]) / n[a] for a in range(3))
    want = sum(fz(z)[:, None, None] * fy(y)[None, :, None] * fx(x)[None, None, :] for fx, fy, fz in p["gD_factors"])
    np.testing.assert_allclose(g, want, rtol=0, atol=1e-14 * np.abs(want).max())
