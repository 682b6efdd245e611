"""Pins of the oracle's discretisation (Sec. 2) against facts independent of its code:
Gauss quadrature of the trilinear basis, closed-form stencil rows, conservation identities."""
import numpy as np
import pytest

from paper_1506_02983_gb300 import inputs


def _trilinear_grads(hx, hy, hz, q=2):
    """Values and gradients of the 8 trilinear basis functions at q^3 Gauss points of the
    box [0,hx]x[0,hy]x[0,hz], local node r = a + 2b + 4c. Written from the definition of the
    basis, independently of the oracle."""
    g, w = np.polynomial.legendre.leggauss(q)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for i in range(q):
        for j in range(q):
            for k in range(q):
                pts.append((g[i], g[j], g[k]))
                wts.append(w[i] * w[j] * w[k] * hx * hy * hz)
    H = (hx, hy, hz)
    vals = np.zeros((len(pts), 8))
    grads = np.zeros((len(pts), 8, 3))
    for p, (s, t, u) in enumerate(pts):
        loc = (s, t, u)
        for r in range(8):
            bits = (r & 1, (r >> 1) & 1, (r >> 2) & 1)
            f1 = [loc[a] if bits[a] else 1.0 - loc[a] for a in range(3)]
            d1 = [(1.0 if bits[a] else -1.0) / H[a] for a in range(3)]
            vals[p, r] = f1[0] * f1[1] * f1[2]
            grads[p, r] = (d1[0] * f1[1] * f1[2], f1[0] * d1[1] * f1[2], f1[0] * f1[1] * d1[2])
    return np.array(wts), vals, grads


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.3, 0.7, 1.9), (0.125, 0.25, 0.0625)])
def test_element_matrix_matches_quadrature(oracle_mod, h):
    w, _, G = _trilinear_grads(*h)
    Kq = np.einsum("p,pia,pja->ij", w, G, G)
    K = oracle_mod.element_matrix(*h)
    assert np.allclose(K, Kq, rtol=1e-13, atol=1e-15)
    assert np.allclose(K, K.T)
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-13)


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.3, 0.7, 1.9)])
def test_mass_matrices_match_quadrature(oracle_mod, h):
    w, V, _ = _trilinear_grads(*h)
    Mq = np.einsum("p,pi,pj->ij", w, V, V)
    assert np.allclose(oracle_mod.element_mass(*h), Mq, rtol=1e-13)
    # face mass: bilinear basis on an ha x hb rectangle
    ha, hb = h[0], h[1]
    g, gw = np.polynomial.legendre.leggauss(2)
    g = 0.5 * (g + 1)
    gw = 0.5 * gw
    Mf = np.zeros((4, 4))
    for i in range(2):
        for j in range(2):
            s, t = g[i], g[j]
            phi = np.array([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t])
            Mf += gw[i] * gw[j] * ha * hb * np.outer(phi, phi)
    assert np.allclose(oracle_mod.face_mass(ha, hb), Mf, rtol=1e-13)


def test_assembled_interior_row_closed_form(oracle_mod):
    """Cube elements, beta = 1: interior row = 8h/3 at the centre, 0 for the 6 face
    neighbours, -h/6 for the 12 edge neighbours, -h/12 for the 8 corner neighbours."""
    n = [4, 4, 4]
    h = 0.25
    A = oracle_mod.assemble(n, [h] * 3, np.ones(64), [0] * 6, [0.0] * 6)
    D = A.dense()
    row = D[2 + 5 * (2 + 5 * 2)].reshape(5, 5, 5)[1:4, 1:4, 1:4]
    for dk in range(3):
        for dj in range(3):
            for di in range(3):
                nz = (di != 1) + (dj != 1) + (dk != 1)
                want = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[nz]
                assert row[dk, dj, di] == pytest.approx(want, abs=1e-15)


def test_assembled_matrix_symmetric_and_neumann_rows_sum_to_zero(oracle_mod):
    p = inputs.random_problem(3, n0=(3, 2, 2), levels=1)
    n = p["n0"]
    h = [(p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    # pure Neumann (all faces Robin with alpha = 0): every row sums to zero
    A = oracle_mod.assemble(n, h, p["beta"], [1] * 6, [0.0] * 6).dense()
    assert np.allclose(A, A.T, atol=1e-14)
    assert np.allclose(A.sum(axis=1), 0.0, atol=1e-13)
    # Robin alpha on face x=lo adds alpha * (face area) to the total of all entries
    al = [0.7, 0, 0, 0, 0, 0]
    A2 = oracle_mod.assemble(n, h, p["beta"], [1] * 6, al).dense()
    area = (p["hi"][1] - p["lo"][1]) * (p["hi"][2] - p["lo"][2])
    assert A2.sum() == pytest.approx(0.7 * area, rel=1e-12)
    assert np.all(np.linalg.eigvalsh(A2) > -1e-12)


def test_constant_beta_annihilates_linear_functions(oracle_mod):
    """For constant beta, a(l, phi_i) = 0 for every linear l and interior node i."""
    n = [4, 3, 5]
    h = [0.2, 0.3, 0.15]
    A = oracle_mod.assemble(n, h, 2.5 * np.ones(60), [0] * 6, [0.0] * 6)
    z, y, x = np.meshgrid(*[np.arange(n[a] + 1) * h[a] for a in (2, 1, 0)], indexing="ij")
    lin = (1.0 + 2.0 * x - 3.0 * y + 0.5 * z).ravel()
    r = A.matvec(lin).reshape(n[2] + 1, n[1] + 1, n[0] + 1)
    assert np.abs(r[1:-1, 1:-1, 1:-1]).max() < 1e-13


def test_load_vector_integrates_exactly(oracle_mod):
    """b = M f_I: sum b = int f for f = 1, and sum_i b_i x_i = int x dV (Q1 products are
    integrated exactly by the consistent mass matrix)."""
    n = [3, 4, 2]
    h = [0.5, 0.25, 1.5]
    N = (n[0] + 1) * (n[1] + 1) * (n[2] + 1)
    b = oracle_mod.load_nodal(n, h, np.ones(N), [0] * 6)
    vol = n[0] * h[0] * n[1] * h[1] * n[2] * h[2]
    assert b.sum() == pytest.approx(vol, rel=1e-14)
    x = np.tile(np.arange(n[0] + 1) * h[0], (n[1] + 1) * (n[2] + 1))
    assert (b * x).sum() == pytest.approx(vol * n[0] * h[0] / 2, rel=1e-14)
    # Robin data on face z=hi adds int_F g_R phi_i: g_R = 1 gives the face area
    bc = [0, 0, 0, 0, 0, 1]
    gR = np.ones(N)
    b2 = oracle_mod.load_nodal(n, h, np.zeros(N), bc, gR)
    assert b2.sum() == pytest.approx(n[0] * h[0] * n[1] * h[1], rel=1e-14)


def test_restriction_is_exact_coarse_functional(oracle_mod):
    """For f piecewise trilinear on the coarse grid, P^T (M_h f) = M_2h f."""
    nc = [2, 3, 2]
    nf = [4, 6, 4]
    hc = [0.5, 0.4, 0.6]
    hf = [v / 2 for v in hc]
    rng = np.random.default_rng(7)
    fc = rng.uniform(-1, 1, (nc[2] + 1, nc[1] + 1, nc[0] + 1))
    # coarse trilinear function sampled on the fine grid (interpolation by averaging)
    ff = np.zeros((nf[2] + 1, nf[1] + 1, nf[0] + 1))
    ff[::2, ::2, ::2] = fc
    ff[::2, ::2, 1::2] = 0.5 * (ff[::2, ::2, :-1:2] + ff[::2, ::2, 2::2])
    ff[::2, 1::2, :] = 0.5 * (ff[::2, :-1:2, :] + ff[::2, 2::2, :])
    ff[1::2] = 0.5 * (ff[:-1:2] + ff[2::2])
    bf = oracle_mod.load_nodal(nf, hf, ff.ravel(), [0] * 6)
    bc = oracle_mod.load_nodal(nc, hc, fc.ravel(), [0] * 6)
    assert np.allclose(oracle_mod.restrict_load(nc, bf), bc, rtol=1e-13, atol=1e-15)


def test_coarsening_and_injection(oracle_mod):
    rng = np.random.default_rng(1)
    nc = [2, 3, 1]
    bf = rng.uniform(1, 2, (2, 6, 4))
    bc = oracle_mod.coarsen_beta(nc, bf.ravel()).reshape(1, 3, 2)
    want = bf.reshape(1, 2, 3, 2, 2, 2).mean(axis=(1, 3, 5))
    assert np.allclose(bc, want, rtol=1e-15)
    vf = rng.uniform(-1, 1, (3, 7, 5))
    assert np.array_equal(oracle_mod.inject(nc, vf.ravel()).reshape(2, 4, 3), vf[::2, ::2, ::2])


def test_dirichlet_mask(oracle_mod):
    m = oracle_mod.dirichlet_mask([2, 2, 2], [0, 1, 1, 1, 1, 0]).reshape(3, 3, 3)
    assert m[:, :, 0].sum() == 0 and m[2].sum() == 0
    assert m.sum() == 2 * 3 * 2
