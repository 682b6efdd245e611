"""The oracle's single-node evaluations (used by the full-size GPU parity tests, where the
whole-grid oracle would be too slow) equal the whole-grid functions they restate, at every
node of small ragged grids: or_apply_at against the rows of the assembled CSR matrix (itself
pinned to the closed-form element matrix), or_exp_finite_at against or_exp_finite, and
or_exp_true_at against or_exp_true."""
import itertools

import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs


def _all_nodes(n):
    return list(itertools.product(range(n[0] + 1), range(n[1] + 1), range(n[2] + 1)))


@pytest.mark.parametrize("face_bc,alpha", [([0] * 6, [0.0] * 6),
                                           ([1, 0, 0, 1, 1, 0], [0.5, 0.0, 0.0, 2.0, 1.0, 0.0]),
                                           ([1] * 6, [0.3, 0.7, 1.1, 0.0, 2.0, 0.4])])
def test_apply_at_equals_csr_rows(oracle_mod, face_bc, alpha):
    n, h = (5, 3, 4), (0.2, 0.35, 0.15)
    rng = np.random.default_rng(5)
    beta = np.exp(rng.standard_normal(n[0] * n[1] * n[2]))
    x = rng.uniform(-1, 1, (n[0] + 1) * (n[1] + 1) * (n[2] + 1))
    A = oracle_mod.assemble(n, h, beta, face_bc, alpha)
    y = A.matvec(x)
    nodes = _all_nodes(n)
    ya = oracle_mod.apply_at(n, h, beta, face_bc, alpha, x, nodes)
    idx = [i + (n[0] + 1) * (j + (n[1] + 1) * k) for i, j, k in nodes]
    assert np.allclose(ya, y[idx], rtol=1e-13, atol=1e-14 * np.abs(y).max())


def test_exp_finite_at_equals_whole_grid(oracle_mod):
    n = (8, 12, 4)
    rng = np.random.default_rng(6)
    n1 = [v // 2 for v in n]
    n0 = [v // 4 for v in n]
    U1 = rng.uniform(-1, 1, (n1[0] + 1) * (n1[1] + 1) * (n1[2] + 1))
    U0 = rng.uniform(-1, 1, (n0[0] + 1) * (n0[1] + 1) * (n0[2] + 1))
    W = oracle_mod.exp_finite(n, U1, U0)
    nodes = _all_nodes(n)
    Wa = oracle_mod.exp_finite_at(n, U1, U0, nodes)
    idx = [i + (n[0] + 1) * (j + (n[1] + 1) * k) for i, j, k in nodes]
    assert np.array_equal(Wa, W[idx])


def test_exp_true_at_equals_whole_grid(oracle_mod):
    n = (6, 4, 10)
    rng = np.random.default_rng(7)
    nc = [v // 2 for v in n]
    U1 = rng.uniform(-1, 1, (n[0] + 1) * (n[1] + 1) * (n[2] + 1))
    U0 = rng.uniform(-1, 1, (nc[0] + 1) * (nc[1] + 1) * (nc[2] + 1))
    Ut = oracle_mod.exp_true(n, U1, U0)
    nodes = _all_nodes(n)
    Ua = oracle_mod.exp_true_at(n, U1, U0, nodes)
    idx = [i + (n[0] + 1) * (j + (n[1] + 1) * k) for i, j, k in nodes]
    assert np.array_equal(Ua, Ut[idx])
