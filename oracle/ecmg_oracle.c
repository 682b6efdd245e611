/*
 * ecmg_oracle.c -- plain, slow, FP64 CPU oracle for the ECMG_jcg method of
 * K. Pan, D. He, H. Hu, "A new extrapolation cascadic multigrid method for 3D elliptic
 * boundary value problems on rectangular domains" (arXiv 1506.02983).
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark are the only users. The CUDA library never includes, links or calls this file;
 * the two share no code, header, table or constant.
 *
 * Everything here is written for a reader checking it against the paper:
 *   - the FE system A_h u_h = f_h of Sec. 2 is assembled element by element into CSR;
 *   - DSOLVE on the two coarsest grids is a banded Cholesky factorisation (Alg. 4, lines 1-2);
 *   - JCG is the textbook Jacobi-preconditioned CG with the relative-residual test of
 *     Alg. 4, lines 7-9;
 *   - EXP_finite follows Sec. 4.3 literally: 8 corner values by eq. (jiedian), 12 edge
 *     midpoints by eq. (zhongdian), the other 105 of 125 nodes by the 20-node Serendipity
 *     interpolation eq. (inter) with the shape functions printed in Sec. 4.3;
 *   - or_exp_finite27 is the 27-node tri-quadratic Lagrange variant of the Remark in Sec. 4.3
 *     (face and body centres by averaged diagonal mid-point formulas);
 *   - EXP_true follows Sec. 4.3 (last paragraph): eq. (t1) at coarse nodes, eq. (chenlin) at
 *     edge, face and body centres.
 *
 * Pins (checked in tests/ marked "not gpu"): closed-form and quadrature checks of the element
 * and mass matrices, assembled-row closed form, linear-function annihilation, dense direct
 * solve on tiny grids, FE order 2, the W_35 weights printed in Sec. 4.3, exactness of
 * EXP_finite on quadratic-plus-h^2 data, exactness of EXP_true on u + trilinear*h^2 data,
 * orders 3 and 4 of W-U and U~-u, and the 1D formulas (sifen1)/(sifen2).
 * Parity is pinned for every function in this file.
 *
 * Readings of places where the paper is silent:
 *   - "P_1" in Sec. 2 is the trilinear Q1 space on hexahedra (27-point stencil).
 *   - beta is one value per element; a coarse element takes the mean of its 8 children.
 *   - the load of the nodal mode is M f_I + sum_F M_F gR_I (consistent mass matrices applied
 *     to nodal interpolants); coarse levels inject f, gD and gR.
 *   - ||f_h|| in the stopping test is the norm of the free-node right-hand side after the
 *     Dirichlet values have been moved to it.
 *   - JCG tests the recursively updated residual; the true residual is reported on exit.
 *   - W is reset to g_D on Dirichlet nodes after EXP_finite.
 *   - In EXP_true a face centre averages eq. (chenlin) over the two face diagonals and the
 *     body centre over the four space diagonals (the averaging rule of the Remark in
 *     Sec. 4.3).
 */
#include "ecmg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int32_t or_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static double wall_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* ----------------------------------------------------------------------------------- */
/* indexing                                                                            */
/* ----------------------------------------------------------------------------------- */
static int64_t node_id(const int32_t n[3], int64_t i, int64_t j, int64_t k)
{
    return i + (int64_t)(n[0] + 1) * (j + (int64_t)(n[1] + 1) * k);
}
static int64_t elem_id(const int32_t n[3], int64_t i, int64_t j, int64_t k)
{
    return i + (int64_t)n[0] * (j + (int64_t)n[1] * k);
}
static int64_t num_nodes(const int32_t n[3])
{
    return (int64_t)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
}
static int64_t num_elems(const int32_t n[3])
{
    return (int64_t)n[0] * n[1] * n[2];
}

/* ----------------------------------------------------------------------------------- */
/* Sec. 2: element matrices of the bilinear form a(u,v) = int beta grad u . grad v       */
/*         + int_{Gamma_R} alpha u v, for the trilinear basis on a box element.          */
/* ----------------------------------------------------------------------------------- */

/* 1D stiffness int phi_s' phi_t' and mass int phi_s phi_t of the two linear hat pieces on an
 * interval of length h. */
static double k1d(double h, int s, int t) { return (s == t ? 1.0 : -1.0) / h; }
static double m1d(double h, int s, int t) { return (s == t ? 2.0 : 1.0) * h / 6.0; }

/* K[a+2b+4c][a'+2b'+4c'] = int_e grad phi . grad phi' for beta = 1.  The trilinear basis is a
 * tensor product, so the integral factorises into 1D stiffness and mass factors. */
void or_element_matrix(double hx, double hy, double hz, double K[64])
{
    for (int r = 0; r < 8; ++r) {
        int a = r & 1, b = (r >> 1) & 1, c = (r >> 2) & 1;
        for (int s = 0; s < 8; ++s) {
            int a2 = s & 1, b2 = (s >> 1) & 1, c2 = (s >> 2) & 1;
            K[r * 8 + s] = k1d(hx, a, a2) * m1d(hy, b, b2) * m1d(hz, c, c2)
                         + m1d(hx, a, a2) * k1d(hy, b, b2) * m1d(hz, c, c2)
                         + m1d(hx, a, a2) * m1d(hy, b, b2) * k1d(hz, c, c2);
        }
    }
}

/* M[a+2b][a'+2b'] = int_F phi phi' on a rectangular face with sides ha, hb. */
void or_face_mass(double ha, double hb, double M[16])
{
    for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s)
            M[r * 4 + s] = m1d(ha, r & 1, s & 1) * m1d(hb, r >> 1, s >> 1);
}

/* Consistent element mass matrix int_e phi phi'. */
void or_element_mass(double hx, double hy, double hz, double M[64])
{
    for (int r = 0; r < 8; ++r)
        for (int s = 0; s < 8; ++s)
            M[r * 8 + s] = m1d(hx, r & 1, s & 1) * m1d(hy, (r >> 1) & 1, (s >> 1) & 1)
                         * m1d(hz, (r >> 2) & 1, (s >> 2) & 1);
}

void or_dirichlet_mask(const int32_t n[3], const int32_t face_bc[6], uint8_t* mask)
{
    for (int64_t k = 0; k <= n[2]; ++k)
        for (int64_t j = 0; j <= n[1]; ++j)
            for (int64_t i = 0; i <= n[0]; ++i) {
                int d = (i == 0 && face_bc[0] == OR_DIRICHLET) || (i == n[0] && face_bc[1] == OR_DIRICHLET)
                     || (j == 0 && face_bc[2] == OR_DIRICHLET) || (j == n[1] && face_bc[3] == OR_DIRICHLET)
                     || (k == 0 && face_bc[4] == OR_DIRICHLET) || (k == n[2] && face_bc[5] == OR_DIRICHLET);
                mask[node_id(n, i, j, k)] = (uint8_t)(d ? 0 : 1); /* 1 = free */
            }
}

/* Robin faces: for face f, the two in-face axes and the fixed coordinate. */
static void face_axes(int f, int* ax_a, int* ax_b, int* ax_n)
{
    int normal = f / 2;
    *ax_n = normal;
    *ax_a = (normal == 0) ? 1 : 0;
    *ax_b = (normal == 2) ? 1 : 2;
}

/* Assemble the full matrix A over all nodes (no boundary elimination) into CSR.
 * The 27 possible neighbours of a row are kept in the fixed order
 * s = (di+1) + 3 (dj+1) + 9 (dk+1); neighbours outside the grid are dropped.
 * rowptr has N+1 entries, col/val at least 27 N. Returns nnz. */
int64_t or_assemble_csr(const int32_t n[3], const double h[3], const double* beta,
                        const int32_t face_bc[6], const double alpha[6],
                        int64_t* rowptr, int64_t* col, double* val)
{
    const int64_t N = num_nodes(n);
    double* dense = (double*)calloc((size_t)N * 27, sizeof(double));
    if (!dense) return -1;
    double K[64];
    or_element_matrix(h[0], h[1], h[2], K);

    /* element loop: A += beta_e K_e */
    for (int64_t ez = 0; ez < n[2]; ++ez)
        for (int64_t ey = 0; ey < n[1]; ++ey)
            for (int64_t ex = 0; ex < n[0]; ++ex) {
                double be = beta[elem_id(n, ex, ey, ez)];
                for (int r = 0; r < 8; ++r) {
                    int a = r & 1, b = (r >> 1) & 1, c = (r >> 2) & 1;
                    int64_t row = node_id(n, ex + a, ey + b, ez + c);
                    for (int s = 0; s < 8; ++s) {
                        int a2 = s & 1, b2 = (s >> 1) & 1, c2 = (s >> 2) & 1;
                        int slot = (a2 - a + 1) + 3 * (b2 - b + 1) + 9 * (c2 - c + 1);
                        dense[row * 27 + slot] += be * K[r * 8 + s];
                    }
                }
            }

    /* Robin faces: A += alpha_F M_F on every quad of face F */
    for (int f = 0; f < 6; ++f) {
        if (face_bc[f] != OR_ROBIN || alpha[f] == 0.0) continue;
        int aa, ab, an;
        face_axes(f, &aa, &ab, &an);
        double M[16];
        or_face_mass(h[aa], h[ab], M);
        int64_t fixed = (f % 2 == 0) ? 0 : n[an];
        for (int64_t qb = 0; qb < n[ab]; ++qb)
            for (int64_t qa = 0; qa < n[aa]; ++qa) {
                for (int r = 0; r < 4; ++r) {
                    int64_t c1[3];
                    c1[an] = fixed; c1[aa] = qa + (r & 1); c1[ab] = qb + (r >> 1);
                    int64_t row = node_id(n, c1[0], c1[1], c1[2]);
                    for (int s = 0; s < 4; ++s) {
                        int64_t c2[3];
                        c2[an] = fixed; c2[aa] = qa + (s & 1); c2[ab] = qb + (s >> 1);
                        int slot = (int)(c2[0] - c1[0] + 1) + 3 * (int)(c2[1] - c1[1] + 1)
                                 + 9 * (int)(c2[2] - c1[2] + 1);
                        dense[row * 27 + slot] += alpha[f] * M[r * 4 + s];
                    }
                }
            }
    }

    /* compress to CSR */
    int64_t nnz = 0;
    for (int64_t k = 0; k <= n[2]; ++k)
        for (int64_t j = 0; j <= n[1]; ++j)
            for (int64_t i = 0; i <= n[0]; ++i) {
                int64_t row = node_id(n, i, j, k);
                rowptr[row] = nnz;
                for (int s = 0; s < 27; ++s) {
                    int64_t di = s % 3 - 1, dj = (s / 3) % 3 - 1, dk = s / 9 - 1;
                    int64_t i2 = i + di, j2 = j + dj, k2 = k + dk;
                    if (i2 < 0 || j2 < 0 || k2 < 0 || i2 > n[0] || j2 > n[1] || k2 > n[2]) continue;
                    col[nnz] = node_id(n, i2, j2, k2);
                    val[nnz] = dense[row * 27 + s];
                    ++nnz;
                }
            }
    rowptr[N] = nnz;
    free(dense);
    return nnz;
}

/* f(v) = int f v + int_{Gamma_R} g_R v with f and g_R replaced by their nodal interpolants:
 * b = M f_I + sum over Robin faces of M_F gR_I (Sec. 2, eq. for f(v)). */
void or_load_nodal(const int32_t n[3], const double h[3], const double* f,
                   const int32_t face_bc[6], const double* gR, double* b)
{
    const int64_t N = num_nodes(n);
    memset(b, 0, (size_t)N * sizeof(double));
    double M[64];
    or_element_mass(h[0], h[1], h[2], M);
    for (int64_t ez = 0; ez < n[2]; ++ez)
        for (int64_t ey = 0; ey < n[1]; ++ey)
            for (int64_t ex = 0; ex < n[0]; ++ex)
                for (int r = 0; r < 8; ++r) {
                    int64_t row = node_id(n, ex + (r & 1), ey + ((r >> 1) & 1), ez + (r >> 2));
                    double s = 0.0;
                    for (int c = 0; c < 8; ++c)
                        s += M[r * 8 + c] * f[node_id(n, ex + (c & 1), ey + ((c >> 1) & 1), ez + (c >> 2))];
                    b[row] += s;
                }
    if (!gR) return;
    for (int fc = 0; fc < 6; ++fc) {
        if (face_bc[fc] != OR_ROBIN) continue;
        int aa, ab, an;
        face_axes(fc, &aa, &ab, &an);
        double MF[16];
        or_face_mass(h[aa], h[ab], MF);
        int64_t fixed = (fc % 2 == 0) ? 0 : n[an];
        for (int64_t qb = 0; qb < n[ab]; ++qb)
            for (int64_t qa = 0; qa < n[aa]; ++qa)
                for (int r = 0; r < 4; ++r) {
                    int64_t c1[3];
                    c1[an] = fixed; c1[aa] = qa + (r & 1); c1[ab] = qb + (r >> 1);
                    double s = 0.0;
                    for (int c = 0; c < 4; ++c) {
                        int64_t c2[3];
                        c2[an] = fixed; c2[aa] = qa + (c & 1); c2[ab] = qb + (c >> 1);
                        s += MF[r * 4 + c] * gR[node_id(n, c2[0], c2[1], c2[2])];
                    }
                    b[node_id(n, c1[0], c1[1], c1[2])] += s;
                }
    }
}

/* (A x) at the single node (i, j, k), straight from the element matrices: beta_e K_e for every
 * element containing the node, plus alpha_F M_F for every quad of a Robin face containing it
 * (the full matrix of Sec. 2, no Dirichlet elimination; the row or_assemble_csr builds). */
double or_apply_at(const int32_t n[3], const double h[3], const double* beta, const int32_t face_bc[6],
                   const double alpha[6], const double* x, int64_t i, int64_t j, int64_t k)
{
    double K[64];
    or_element_matrix(h[0], h[1], h[2], K);
    double y = 0.0;
    for (int r = 0; r < 8; ++r) {
        int a = r & 1, b = (r >> 1) & 1, c = (r >> 2) & 1;
        int64_t ex = i - a, ey = j - b, ez = k - c;  /* element with this node at local corner r */
        if (ex < 0 || ey < 0 || ez < 0 || ex >= n[0] || ey >= n[1] || ez >= n[2]) continue;
        double be = beta[elem_id(n, ex, ey, ez)];
        for (int s = 0; s < 8; ++s) {
            int a2 = s & 1, b2 = (s >> 1) & 1, c2 = (s >> 2) & 1;
            y += be * K[r * 8 + s] * x[node_id(n, ex + a2, ey + b2, ez + c2)];
        }
    }
    const int64_t F[3] = {i, j, k};
    for (int f = 0; f < 6; ++f) {
        if (face_bc[f] != OR_ROBIN || alpha[f] == 0.0) continue;
        int aa, ab, an;
        face_axes(f, &aa, &ab, &an);
        if (F[an] != ((f % 2 == 0) ? 0 : n[an])) continue;
        double M[16];
        or_face_mass(h[aa], h[ab], M);
        for (int r = 0; r < 4; ++r) {
            int64_t qa = F[aa] - (r & 1), qb = F[ab] - (r >> 1);  /* quad with this node at corner r */
            if (qa < 0 || qb < 0 || qa >= n[aa] || qb >= n[ab]) continue;
            for (int s = 0; s < 4; ++s) {
                int64_t c2[3];
                c2[an] = F[an]; c2[aa] = qa + (s & 1); c2[ab] = qb + (s >> 1);
                y += alpha[f] * M[r * 4 + s] * x[node_id(n, c2[0], c2[1], c2[2])];
            }
        }
    }
    return y;
}

void or_csr_matvec(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                   const double* x, double* y)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < N; ++r) {
        double s = 0.0;
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) s += val[q] * x[col[q]];
        y[r] = s;
    }
}

/* ----------------------------------------------------------------------------------- */
/* level transfer (nested grids, refinement by 2 per axis)                                */
/* ----------------------------------------------------------------------------------- */

/* Coarse element = mean of its 8 children.  nc = coarse element counts. */
void or_coarsen_beta(const int32_t nc[3], const double* beta_fine, double* beta_coarse)
{
    int32_t nf[3] = {2 * nc[0], 2 * nc[1], 2 * nc[2]};
    for (int64_t k = 0; k < nc[2]; ++k)
        for (int64_t j = 0; j < nc[1]; ++j)
            for (int64_t i = 0; i < nc[0]; ++i) {
                double s = 0.0;
                for (int c = 0; c < 8; ++c)
                    s += beta_fine[elem_id(nf, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + (c >> 2))];
                beta_coarse[elem_id(nc, i, j, k)] = s / 8.0;
            }
}

/* Coarse node (i,j,k) coincides with fine node (2i,2j,2k). */
void or_inject(const int32_t nc[3], const double* v_fine, double* v_coarse)
{
    int32_t nf[3] = {2 * nc[0], 2 * nc[1], 2 * nc[2]};
    for (int64_t k = 0; k <= nc[2]; ++k)
        for (int64_t j = 0; j <= nc[1]; ++j)
            for (int64_t i = 0; i <= nc[0]; ++i)
                v_coarse[node_id(nc, i, j, k)] = v_fine[node_id(nf, 2 * i, 2 * j, 2 * k)];
}

/* b_coarse = P^T b_fine where P is trilinear prolongation: fine node (I,J,K) receives the
 * coarse value with weight prod_a (1 if I_a even and coincident, 1/2 if odd and adjacent).
 * Each coarse basis function is the sum of fine basis functions with these weights, so P^T b
 * is the exact coarse load functional. */
void or_restrict_load(const int32_t nc[3], const double* b_fine, double* b_coarse)
{
    int32_t nf[3] = {2 * nc[0], 2 * nc[1], 2 * nc[2]};
    memset(b_coarse, 0, (size_t)num_nodes(nc) * sizeof(double));
    for (int64_t K = 0; K <= nf[2]; ++K)
        for (int64_t J = 0; J <= nf[1]; ++J)
            for (int64_t I = 0; I <= nf[0]; ++I) {
                double v = b_fine[node_id(nf, I, J, K)];
                /* coarse neighbours along each axis with their 1D weights */
                int64_t ci[3][2], cnt[3];
                double cw[3][2];
                int64_t F[3] = {I, J, K};
                for (int a = 0; a < 3; ++a) {
                    if (F[a] % 2 == 0) { cnt[a] = 1; ci[a][0] = F[a] / 2; cw[a][0] = 1.0; }
                    else { cnt[a] = 2; ci[a][0] = F[a] / 2; ci[a][1] = F[a] / 2 + 1; cw[a][0] = cw[a][1] = 0.5; }
                }
                for (int p = 0; p < cnt[0]; ++p)
                    for (int q = 0; q < cnt[1]; ++q)
                        for (int r = 0; r < cnt[2]; ++r)
                            b_coarse[node_id(nc, ci[0][p], ci[1][q], ci[2][r])] += cw[0][p] * cw[1][q] * cw[2][r] * v;
            }
}

/* ----------------------------------------------------------------------------------- */
/* Solvers                                                                              */
/* ----------------------------------------------------------------------------------- */

static double dot_masked(int64_t N, const uint8_t* m, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) if (m[i]) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned CG on the free-node system (Alg. 4, lines 7-9).
 * x holds all nodes; its Dirichlet entries are the boundary values and are never changed.
 * gext is the vector equal to g_D on Dirichlet nodes and 0 elsewhere; it is used once, to
 * form ||f_h|| = ||(b - A gext)_free||, the right-hand side after moving the boundary values.
 * Stopping test: ||r||_2 <= rtol ||f_h||_2 on the recursively updated residual, evaluated
 * before the first iteration (zero iterations allowed) and after every update.
 * Returns 0, or 3 when max_iters is reached, or 4 on breakdown (p.q <= 0 or not finite). */
int or_jcg(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
           const uint8_t* mask, const double* b, const double* gext, double* x,
           double rtol, int32_t max_iters, int32_t* iters, double* rel_res_true,
           double* rhs_norm)
{
    return or_pcg(N, rowptr, col, val, mask, b, gext, x, rtol, max_iters, 1, 0, iters, rel_res_true, rhs_norm);
}

/* CG (Alg. 4 line 8 for ECMG_cg) or Jacobi-preconditioned CG (ECMG_jcg), textbook form. precond: 1 = Jacobi
 * (z = D^-1 r), 0 = none (z = r). fixed: 1 = run exactly max_iters iterations with no tolerance
 * test (the m_j steps of Alg. 3), which then is not a failure. */
int or_pcg(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
           const uint8_t* mask, const double* b, const double* gext, double* x,
           double rtol, int32_t max_iters, int32_t precond, int32_t fixed, int32_t* iters, double* rel_res_true,
           double* rhs_norm)
{
    double* r = (double*)malloc((size_t)N * sizeof(double));
    double* z = (double*)malloc((size_t)N * sizeof(double));
    double* p = (double*)malloc((size_t)N * sizeof(double));
    double* q = (double*)malloc((size_t)N * sizeof(double));
    double* dinv = (double*)malloc((size_t)N * sizeof(double));
    int status = 0;

    /* Jacobi preconditioner: the diagonal of A on free nodes (identity for plain CG) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double d = 0.0;
        for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) if (col[t] == i) d = val[t];
        dinv[i] = mask[i] ? (precond ? 1.0 / d : 1.0) : 0.0;
    }

    /* ||f_h|| */
    or_csr_matvec(N, rowptr, col, val, gext, q);
    double fh2 = 0.0;
    for (int64_t i = 0; i < N; ++i) if (mask[i]) { double t = b[i] - q[i]; fh2 += t * t; }
    double fh = sqrt(fh2);
    *rhs_norm = fh;

    /* r = b - A x on free nodes */
    or_csr_matvec(N, rowptr, col, val, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) r[i] = mask[i] ? b[i] - q[i] : 0.0;

    int32_t k = 0;
    double rr = dot_masked(N, mask, r, r);
    if (fixed ? max_iters > 0 : sqrt(rr) > rtol * fh) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
        double rho = dot_masked(N, mask, r, z);
        for (;;) {
            if (k >= max_iters) { status = fixed ? 0 : 3; break; }
            or_csr_matvec(N, rowptr, col, val, p, q);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) if (!mask[i]) q[i] = 0.0;
            double pq = dot_masked(N, mask, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { status = 4; break; }
            double alpha = rho / pq;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                x[i] += alpha * p[i];
                r[i] -= alpha * q[i];
            }
            ++k;
            rr = dot_masked(N, mask, r, r);
            if (!fixed && sqrt(rr) <= rtol * fh) break;
            if (fixed && k >= max_iters) break;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) z[i] = dinv[i] * r[i];
            double rho_new = dot_masked(N, mask, r, z);
            double beta = rho_new / rho;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
            rho = rho_new;
        }
    }
    *iters = k;

    /* true residual on exit */
    or_csr_matvec(N, rowptr, col, val, x, q);
    double tr = 0.0;
    for (int64_t i = 0; i < N; ++i) if (mask[i]) { double t = b[i] - q[i]; tr += t * t; }
    *rel_res_true = (fh > 0.0) ? sqrt(tr) / fh : sqrt(tr);

    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}

/* The same Jacobi-preconditioned CG (Alg. 4, line 8) arranged in one pass over the vectors per
 * step, as the library's ECMG_CG_SINGLE_PASS form runs it. Step k first completes the previous
 * step, x_k = x_{k-1} + alpha_{k-1} p_{k-1} and r_k = r_{k-1} - alpha_{k-1} q_{k-1}, then forms
 * z_k = D^-1 r_k, p_k = z_k + beta_k p_{k-1} and q_k = A p_k, and takes every dot it needs from
 * these vectors: alpha_k = (r_k.z_k) / (p_k.q_k), and the quantities of r_{k+1} = r_k - alpha_k q_k
 * by expanding the products,
 *     r_{k+1}.z_{k+1} = r_k.z_k - 2 alpha_k z_k.q_k + alpha_k^2 q_k.D^-1 q_k,
 *     ||r_{k+1}||^2   = r_k.r_k - 2 alpha_k r_k.q_k + alpha_k^2 q_k.q_k,
 * so beta_{k+1} = r_{k+1}.z_{k+1} / r_k.z_k and the stopping test on ||r_{k+1}|| need no second
 * pass. In exact arithmetic every iterate equals that of or_pcg. On exit the pending step is
 * applied to x. Same outputs as or_pcg (tolerance schedule). */
int or_pcg_single_pass(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                       const uint8_t* mask, const double* b, const double* gext, double* x, double rtol,
                       int32_t max_iters, int32_t precond, int32_t* iters, double* rel_res_true,
                       double* rhs_norm)
{
    double* r = (double*)malloc((size_t)N * sizeof(double));
    double* z = (double*)malloc((size_t)N * sizeof(double));
    double* p = (double*)calloc((size_t)N, sizeof(double));
    double* q = (double*)calloc((size_t)N, sizeof(double));
    double* dinv = (double*)malloc((size_t)N * sizeof(double));
    int status = 0;

    for (int64_t i = 0; i < N; ++i) {
        double d = 0.0;
        for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) if (col[t] == i) d = val[t];
        dinv[i] = mask[i] ? (precond ? 1.0 / d : 1.0) : 0.0;
    }

    or_csr_matvec(N, rowptr, col, val, gext, q);
    double fh2 = 0.0;
    for (int64_t i = 0; i < N; ++i) if (mask[i]) { double t = b[i] - q[i]; fh2 += t * t; }
    double fh = sqrt(fh2);
    *rhs_norm = fh;

    or_csr_matvec(N, rowptr, col, val, x, q);
    for (int64_t i = 0; i < N; ++i) { r[i] = mask[i] ? b[i] - q[i] : 0.0; q[i] = 0.0; }

    int32_t k = 0;
    double alpha_prev = 0.0, beta = 0.0;  /* the pending step and the next direction's coefficient */
    double rr = dot_masked(N, mask, r, r);
    if (sqrt(rr) > rtol * fh) {
        for (;;) {
            if (k >= max_iters) { status = 3; break; }
            for (int64_t i = 0; i < N; ++i) {
                x[i] += alpha_prev * p[i];
                r[i] -= alpha_prev * q[i];
                z[i] = dinv[i] * r[i];
                p[i] = z[i] + beta * p[i];
            }
            or_csr_matvec(N, rowptr, col, val, p, q);
            for (int64_t i = 0; i < N; ++i) if (!mask[i]) q[i] = 0.0;
            double pq = 0.0, rz = 0.0, zq = 0.0, qdq = 0.0, rr_k = 0.0, rq = 0.0, qq = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                if (!mask[i]) continue;
                pq += p[i] * q[i];
                rz += r[i] * z[i];
                zq += z[i] * q[i];
                qdq += q[i] * dinv[i] * q[i];
                rr_k += r[i] * r[i];
                rq += r[i] * q[i];
                qq += q[i] * q[i];
            }
            if (!(pq > 0.0) || !isfinite(pq)) { status = 4; alpha_prev = 0.0; break; }
            const double alpha = rz / pq;
            ++k;
            const double rz_next = rz - 2.0 * alpha * zq + alpha * alpha * qdq;
            const double rr_next = rr_k - 2.0 * alpha * rq + alpha * alpha * qq;
            alpha_prev = alpha;
            if (sqrt(fmax(rr_next, 0.0)) <= rtol * fh) break;
            beta = rz_next / rz;
        }
        for (int64_t i = 0; i < N; ++i) x[i] += alpha_prev * p[i];
    }
    *iters = k;

    or_csr_matvec(N, rowptr, col, val, x, q);
    double tr = 0.0;
    for (int64_t i = 0; i < N; ++i) if (mask[i]) { double t = b[i] - q[i]; tr += t * t; }
    *rel_res_true = (fh > 0.0) ? sqrt(tr) / fh : sqrt(tr);

    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}

/* DSOLVE (Alg. 4, lines 1-2): direct solve of the free-node system by banded Cholesky.
 * The Dirichlet rows and columns are replaced by the identity and their values g_D (held in
 * x on entry) are moved to the right-hand side, so the band is the lexicographic one,
 * w = (n0+1)(n1+1) + (n0+1) + 1. Returns 0, or 2 if the matrix is not positive definite. */
int or_dsolve_banded(const int32_t n[3], int64_t N, const int64_t* rowptr,
                     const int64_t* col, const double* val, const uint8_t* mask,
                     const double* b, double* x)
{
    const int64_t w = (int64_t)(n[0] + 1) * (n[1] + 1) + (n[0] + 1) + 1;
    double* L = (double*)calloc((size_t)N * (size_t)(w + 1), sizeof(double));
    double* rhs = (double*)malloc((size_t)N * sizeof(double));
    if (!L || !rhs) { free(L); free(rhs); return 1; }
#define LB(i, j) L[(size_t)(i) * (size_t)(w + 1) + (size_t)((i) - (j))]
    for (int64_t i = 0; i < N; ++i) {
        if (!mask[i]) { LB(i, i) = 1.0; rhs[i] = x[i]; continue; }
        double s = b[i];
        for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            int64_t j = col[t];
            if (!mask[j]) s -= val[t] * x[j];            /* move boundary values right */
            else if (j <= i) LB(i, j) = val[t];           /* lower triangle, free-free */
        }
        rhs[i] = s;
    }
    int status = 0;
    for (int64_t i = 0; i < N && !status; ++i) {
        int64_t j0 = (i - w > 0) ? i - w : 0;
        for (int64_t j = j0; j <= i; ++j) {
            double s = LB(i, j);
            int64_t k0 = (j - w > j0) ? j - w : j0;
            for (int64_t k = k0; k < j; ++k) s -= LB(i, k) * LB(j, k);
            if (j == i) {
                if (!(s > 0.0)) { status = 2; break; }
                LB(i, i) = sqrt(s);
            } else {
                LB(i, j) = s / LB(j, j);
            }
        }
    }
    if (!status) {
        for (int64_t i = 0; i < N; ++i) {            /* L y = rhs */
            double s = rhs[i];
            int64_t j0 = (i - w > 0) ? i - w : 0;
            for (int64_t j = j0; j < i; ++j) s -= LB(i, j) * rhs[j];
            rhs[i] = s / LB(i, i);
        }
        for (int64_t i = N - 1; i >= 0; --i) {       /* L^T x = y */
            double s = rhs[i];
            int64_t j1 = (i + w < N - 1) ? i + w : N - 1;
            for (int64_t j = i + 1; j <= j1; ++j) s -= LB(j, i) * rhs[j];
            rhs[i] = s / LB(i, i);
        }
        for (int64_t i = 0; i < N; ++i) if (mask[i]) x[i] = rhs[i];
    }
#undef LB
    free(L); free(rhs);
    return status;
}

/* ----------------------------------------------------------------------------------- */
/* Sec. 4.3: 20-node tri-quadratic Serendipity interpolation on the 5x5x5 node patch of a */
/* coarse element. Local node (a,b,c), a,b,c in 0..4, is the paper's node 1+a+5b+25c and   */
/* sits at natural coordinates ((a-2)/2, (b-2)/2, (c-2)/2).                                */
/* ----------------------------------------------------------------------------------- */

/* The 20 interpolation nodes in the order: 8 corners (1,5,21,25,101,105,121,125), the
 * x-direction midpoints (3,23,103,123), y-direction (11,15,111,115), z-direction
 * (51,55,71,75).  abc[3m..3m+2] = local (a,b,c) of node m. */
static const int32_t SER_NODES[20][3] = {
    {0,0,0},{4,0,0},{0,4,0},{4,4,0},{0,0,4},{4,0,4},{0,4,4},{4,4,4},
    {2,0,0},{2,4,0},{2,0,4},{2,4,4},
    {0,2,0},{4,2,0},{0,2,4},{4,2,4},
    {0,0,2},{4,0,2},{0,4,2},{4,4,2}};

void or_serendipity_nodes(int32_t abc[60])
{
    for (int m = 0; m < 20; ++m)
        for (int a = 0; a < 3; ++a) abc[3 * m + a] = SER_NODES[m][a];
}

/* Shape functions N_i of Sec. 4.3 (corner, and mid-side in x, y, z). */
void or_serendipity(double xi, double eta, double zeta, double N[20])
{
    for (int m = 0; m < 20; ++m) {
        double xi_i = (SER_NODES[m][0] - 2) / 2.0;
        double eta_i = (SER_NODES[m][1] - 2) / 2.0;
        double zeta_i = (SER_NODES[m][2] - 2) / 2.0;
        if (m < 8) {
            N[m] = 0.125 * (1 + xi_i * xi) * (1 + eta_i * eta) * (1 + zeta_i * zeta)
                 * (xi_i * xi + eta_i * eta + zeta_i * zeta - 2);
        } else if (m < 12) {
            N[m] = 0.25 * (1 - xi * xi) * (1 + eta_i * eta) * (1 + zeta_i * zeta);
        } else if (m < 16) {
            N[m] = 0.25 * (1 - eta * eta) * (1 + xi_i * xi) * (1 + zeta_i * zeta);
        } else {
            N[m] = 0.25 * (1 - zeta * zeta) * (1 + xi_i * xi) * (1 + eta_i * eta);
        }
    }
}

/* EXP_finite (Alg. 4 line 6, Sec. 4.2.2 and 4.3).
 * n: element counts of the target level l (multiples of 4 per axis).
 * U1: FE solution on level l-1 (n/2 elements), U0: on level l-2 (n/4 elements).
 * W: level-l initial guess, all nodes (boundary reset is the caller's job). */
/* The 20 interpolation values of the level-(l-2) element (ex, ey, ez): 8 corners by eq.
 * (jiedian), W = (5 U^1 - U^0)/4, and 12 edge midpoints by eq. (zhongdian) along the edge,
 * W = U^1_mid + (U^1_A - U^0_A + U^1_B - U^0_B)/8. */
static void ser_values(const int32_t n1[3], const int32_t n0[3], const double* U1, const double* U0,
                       int64_t ex, int64_t ey, int64_t ez, double Wi[20])
{
    for (int m = 0; m < 8; ++m) {
        int a = SER_NODES[m][0], b = SER_NODES[m][1], c = SER_NODES[m][2];
        double u1 = U1[node_id(n1, 2 * ex + a / 2, 2 * ey + b / 2, 2 * ez + c / 2)];
        double u0 = U0[node_id(n0, ex + a / 4, ey + b / 4, ez + c / 4)];
        Wi[m] = (5.0 * u1 - u0) / 4.0;
    }
    for (int m = 8; m < 20; ++m) {
        int a = SER_NODES[m][0], b = SER_NODES[m][1], c = SER_NODES[m][2];
        int dir = (m < 12) ? 0 : (m < 16) ? 1 : 2;
        int A[3] = {a, b, c}, B[3] = {a, b, c};
        A[dir] = 0; B[dir] = 4;
        double umid = U1[node_id(n1, 2 * ex + a / 2, 2 * ey + b / 2, 2 * ez + c / 2)];
        double u1A = U1[node_id(n1, 2 * ex + A[0] / 2, 2 * ey + A[1] / 2, 2 * ez + A[2] / 2)];
        double u0A = U0[node_id(n0, ex + A[0] / 4, ey + A[1] / 4, ez + A[2] / 4)];
        double u1B = U1[node_id(n1, 2 * ex + B[0] / 2, 2 * ey + B[1] / 2, 2 * ez + B[2] / 2)];
        double u0B = U0[node_id(n0, ex + B[0] / 4, ey + B[1] / 4, ez + B[2] / 4)];
        Wi[m] = umid + (u1A - u0A + u1B - u0B) / 8.0;
    }
}

/* EXP_finite (Alg. 4 line 6, Sec. 4.2.2 and 4.3).
 * n: element counts of the target level l (multiples of 4 per axis).
 * U1: FE solution on level l-1 (n/2 elements), U0: on level l-2 (n/4 elements).
 * W: level-l initial guess, all nodes (boundary reset is the caller's job). A node on the
 * face between two coarse elements is written by both (the values agree); the element with
 * the larger index writes last. */
void or_exp_finite(const int32_t n[3], const double* U1, const double* U0, double* W)
{
    int32_t n1[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    int32_t n0[3] = {n[0] / 4, n[1] / 4, n[2] / 4};
    for (int64_t ez = 0; ez < n0[2]; ++ez)
        for (int64_t ey = 0; ey < n0[1]; ++ey)
            for (int64_t ex = 0; ex < n0[0]; ++ex) {
                double Wi[20];
                ser_values(n1, n0, U1, U0, ex, ey, ez, Wi);
                /* all 125 nodes of the patch by eq. (inter) */
                for (int c = 0; c <= 4; ++c)
                    for (int b = 0; b <= 4; ++b)
                        for (int a = 0; a <= 4; ++a) {
                            double N[20];
                            or_serendipity((a - 2) / 2.0, (b - 2) / 2.0, (c - 2) / 2.0, N);
                            double s = 0.0;
                            for (int m = 0; m < 20; ++m) s += N[m] * Wi[m];
                            W[node_id(n, 4 * ex + a, 4 * ey + b, 4 * ez + c)] = s;
                        }
            }
}

/* EXP_finite at the single level-l node (I, J, K): the value or_exp_finite leaves there. */
double or_exp_finite_at(const int32_t n[3], const double* U1, const double* U0, int64_t I, int64_t J, int64_t K)
{
    int32_t n1[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    int32_t n0[3] = {n[0] / 4, n[1] / 4, n[2] / 4};
    int64_t e[3], F[3] = {I, J, K};
    int loc[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = F[a] / 4;
        if (e[a] > n0[a] - 1) e[a] = n0[a] - 1;
        loc[a] = (int)(F[a] - 4 * e[a]);
    }
    double Wi[20], N[20];
    ser_values(n1, n0, U1, U0, e[0], e[1], e[2], Wi);
    or_serendipity((loc[0] - 2) / 2.0, (loc[1] - 2) / 2.0, (loc[2] - 2) / 2.0, N);
    double s = 0.0;
    for (int m = 0; m < 20; ++m) s += N[m] * Wi[m];
    return s;
}

/* Variant of EXP_finite from the Remark after the W_35 example (Sec. 4.3): the 6 face
 * centres and the body centre of the coarse element also get extrapolated values, each the
 * arithmetic mean of the mid-point formula (zhongdian) over the diagonals through it (two
 * face diagonals, four space diagonals); the remaining 98 nodes follow from tri-quadratic
 * Lagrange interpolation of the 27 values. */
static double lag3(int node, double t)
{
    /* quadratic Lagrange basis on the nodes -1, 0, 1 */
    if (node == 0) return 0.5 * t * (t - 1.0);
    if (node == 1) return 1.0 - t * t;
    return 0.5 * t * (t + 1.0);
}

void or_exp_finite27(const int32_t n[3], const double* U1, const double* U0, double* W)
{
    int32_t n1[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    int32_t n0[3] = {n[0] / 4, n[1] / 4, n[2] / 4};
    for (int64_t ez = 0; ez < n0[2]; ++ez)
        for (int64_t ey = 0; ey < n0[1]; ++ey)
            for (int64_t ex = 0; ex < n0[0]; ++ex) {
                double V[27]; /* V[a + 3b + 9c], a,b,c in 0..2 = level-(l-1) nodes of the element */
                for (int c = 0; c < 3; ++c)
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a) {
                            int abc[3] = {a, b, c};
                            double u1 = U1[node_id(n1, 2 * ex + a, 2 * ey + b, 2 * ez + c)];
                            int nodd = (a == 1) + (b == 1) + (c == 1);
                            if (nodd == 0) {   /* coarse node: eq. (jiedian) */
                                double u0 = U0[node_id(n0, ex + a / 2, ey + b / 2, ez + c / 2)];
                                V[a + 3 * b + 9 * c] = (5.0 * u1 - u0) / 4.0;
                                continue;
                            }
                            /* eq. (zhongdian) on every diagonal through the node, averaged */
                            double acc = 0.0;
                            int ndiag = 0;
                            int first_odd = (a == 1) ? 0 : ((b == 1) ? 1 : 2);
                            for (int s = 0; s < 8; ++s) {
                                int ok = 1;
                                for (int t = 0; t < 3; ++t) if (abc[t] != 1 && ((s >> t) & 1)) ok = 0;
                                if (!ok || ((s >> first_odd) & 1)) continue;
                                int A[3], B[3];
                                for (int t = 0; t < 3; ++t) {
                                    if (abc[t] != 1) { A[t] = B[t] = abc[t]; }
                                    else { int bit = (s >> t) & 1; A[t] = 2 * bit; B[t] = 2 - 2 * bit; }
                                }
                                double dA = U1[node_id(n1, 2 * ex + A[0], 2 * ey + A[1], 2 * ez + A[2])]
                                          - U0[node_id(n0, ex + A[0] / 2, ey + A[1] / 2, ez + A[2] / 2)];
                                double dB = U1[node_id(n1, 2 * ex + B[0], 2 * ey + B[1], 2 * ez + B[2])]
                                          - U0[node_id(n0, ex + B[0] / 2, ey + B[1] / 2, ez + B[2] / 2)];
                                acc += u1 + (dA + dB) / 8.0;
                                ++ndiag;
                            }
                            V[a + 3 * b + 9 * c] = acc / ndiag;
                        }
                for (int c = 0; c <= 4; ++c)
                    for (int b = 0; b <= 4; ++b)
                        for (int a = 0; a <= 4; ++a) {
                            double xi = (a - 2) / 2.0, eta = (b - 2) / 2.0, zeta = (c - 2) / 2.0;
                            double s = 0.0;
                            for (int k = 0; k < 3; ++k)
                                for (int j = 0; j < 3; ++j)
                                    for (int i = 0; i < 3; ++i)
                                        s += lag3(i, xi) * lag3(j, eta) * lag3(k, zeta) * V[i + 3 * j + 9 * k];
                            W[node_id(n, 4 * ex + a, 4 * ey + b, 4 * ez + c)] = s;
                        }
            }
}

/* EXP_true at the level-l node (I, J, K). */
double or_exp_true_at(const int32_t n[3], const double* U1, const double* U0, int64_t I, int64_t J, int64_t K)
{
    int32_t nc[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    int64_t F[3] = {I, J, K};
    int odd[3], nodd = 0;
    for (int a = 0; a < 3; ++a) { odd[a] = (int)(F[a] & 1); nodd += odd[a]; }
    double u1 = U1[node_id(n, I, J, K)];
    if (nodd == 0) {
        double u0 = U0[node_id(nc, I / 2, J / 2, K / 2)];
        return (4.0 * u1 - u0) / 3.0;
    }
    /* The coarse nodes around (I,J,K) are F_a/2 + {0,1} on odd axes, F_a/2 on even axes. A
     * diagonal through (I,J,K) pairs each such coarse node with its mirror image; eq.
     * (chenlin) on that diagonal is u1 + (d(A) + d(B))/6 with d = U^1 - U^0 at coarse nodes.
     * Average over the 2^(nodd-1) diagonals. */
    double acc = 0.0;
    int ndiag = 0;
    for (int s = 0; s < 8; ++s) {
        /* corner choice s on the odd axes; skip even-axis bits and mirrored pairs */
        int ok = 1;
        for (int a = 0; a < 3; ++a) if (!odd[a] && ((s >> a) & 1)) ok = 0;
        if (!ok) continue;
        int first_odd = odd[0] ? 0 : (odd[1] ? 1 : 2);
        if ((s >> first_odd) & 1) continue; /* each diagonal once */
        int64_t A[3], B[3];
        for (int a = 0; a < 3; ++a) {
            if (!odd[a]) { A[a] = B[a] = F[a] / 2; }
            else { int bit = (s >> a) & 1; A[a] = F[a] / 2 + bit; B[a] = F[a] / 2 + 1 - bit; }
        }
        double dA = U1[node_id(n, 2 * A[0], 2 * A[1], 2 * A[2])] - U0[node_id(nc, A[0], A[1], A[2])];
        double dB = U1[node_id(n, 2 * B[0], 2 * B[1], 2 * B[2])] - U0[node_id(nc, B[0], B[1], B[2])];
        acc += u1 + (dA + dB) / 6.0;
        ++ndiag;
    }
    return acc / ndiag;
}

/* EXP_true (Alg. 4 line 10, Sec. 4.2.1 and the last paragraph of Sec. 4.3).
 * n: element counts of level l (even). U1: level-l solution, U0: level-(l-1) solution.
 * Coarse nodes by eq. (t1); nodes halfway between two coarse nodes by eq. (chenlin); face
 * centres average (chenlin) over the two face diagonals, body centres over the four space
 * diagonals. */
void or_exp_true(const int32_t n[3], const double* U1, const double* U0, double* Ut)
{
    for (int64_t K = 0; K <= n[2]; ++K)
        for (int64_t J = 0; J <= n[1]; ++J)
            for (int64_t I = 0; I <= n[0]; ++I)
                Ut[node_id(n, I, J, K)] = or_exp_true_at(n, U1, U0, I, J, K);
}

/* ----------------------------------------------------------------------------------- */
/* Alg. 4: the whole ECMG_jcg method                                                    */
/* ----------------------------------------------------------------------------------- */

/* The max norm and the "L2" norm of the tables of Sec. 5: max |a - b| and the root mean
 * square sqrt(sum (a - b)^2 / N) over all N nodes. A NaN difference makes the max NaN (an
 * error norm must not report a finite value for a vector that holds a NaN); the sum carries
 * it into the RMS by itself. */
void or_norms(int64_t N, const double* a, const double* b, double* max_abs, double* rms)
{
    double m = 0.0, s = 0.0;
    int nan_seen = 0;
    for (int64_t i = 0; i < N; ++i) {
        double d = a[i] - (b ? b[i] : 0.0);
        if (isnan(d)) nan_seen = 1;
        else if (fabs(d) > m) m = fabs(d);
        s += d * d;
    }
    *max_abs = nan_seen ? NAN : m;
    *rms = sqrt(s / (double)N);
}

/* U_all / W_all / Ut_all: caller arrays holding all levels back to back, coarsest first
 * (level l occupies num_nodes(n0 * 2^l) entries). W and Ut are left zero on levels 0, 1. */
int or_ecmg(const or_problem* p, double rtol, int32_t max_iters, int32_t exp_variant,
            double* U_all, double* W_all, double* Ut_all, or_stats* st)
{
    return or_ecmg_ex(p, rtol, max_iters, exp_variant, 1, 0, 0, 0.0, U_all, W_all, Ut_all, st);
}

/* Number of CG steps on level l (>= 2) of an L-level hierarchy in the fixed schedule of Alg. 3,
 * eq. (ee): the paper counts the levels above the two direct ones, j = l - 1 = 1 .. L - 2, and
 * m_j = ceil(m_L beta^(L_p - j)) with L_p = L - 2. */
int32_t or_schedule_steps(int32_t L, int32_t l, int32_t mL, double beta)
{
    return (int32_t)ceil((double)mL * pow(beta, (double)((L - 2) - (l - 1))));
}

/* Alg. 4 with the choices of Sec. 3: precond 1 = JCG (ECMG_jcg), 0 = CG (ECMG_cg); schedule 0 =
 * the relative residual test of line 7, 1 = the fixed step counts of Alg. 3 (eq. (ee)) with m_L
 * and beta. */
int or_ecmg_ex(const or_problem* p, double rtol, int32_t max_iters, int32_t exp_variant, int32_t precond,
               int32_t schedule, int32_t mL, double sched_beta, double* U_all, double* W_all, double* Ut_all,
               or_stats* st)
{
    const int L = p->levels;
    memset(st, 0, sizeof(*st));
    if (L < 3 || L > 16) { st->status = 1; return 1; }
    int has_dirichlet = 0, has_alpha = 0;
    for (int f = 0; f < 6; ++f) {
        if (p->face_bc[f] == OR_DIRICHLET) has_dirichlet = 1;
        else if (p->alpha[f] != 0.0) has_alpha = 1;
    }
    if (!has_dirichlet && !has_alpha) { st->status = 2; return 2; }

    int32_t nl[16][3];
    int64_t off[17];
    off[0] = 0;
    for (int l = 0; l < L; ++l) {
        for (int a = 0; a < 3; ++a) nl[l][a] = p->n0[a] << l;
        off[l + 1] = off[l] + num_nodes(nl[l]);
    }
    memset(W_all, 0, (size_t)off[L] * sizeof(double));
    memset(Ut_all, 0, (size_t)off[L] * sizeof(double));
    double t0 = wall_seconds();

    /* per-level data, finest first: beta by averaging, f / gD / gR by injection (or the load
     * functional by restriction in the load mode) */
    double* beta[16];
    double* fl[16];
    double* gDl[16];
    double* gRl[16];
    for (int l = L - 1; l >= 0; --l) {
        int64_t Nn = num_nodes(nl[l]), Ne = num_elems(nl[l]);
        beta[l] = (double*)malloc((size_t)Ne * sizeof(double));
        fl[l] = (double*)malloc((size_t)Nn * sizeof(double));
        gDl[l] = (double*)calloc((size_t)Nn, sizeof(double));
        gRl[l] = (double*)calloc((size_t)Nn, sizeof(double));
        if (l == L - 1) {
            memcpy(beta[l], p->beta, (size_t)Ne * sizeof(double));
            memcpy(fl[l], p->f, (size_t)Nn * sizeof(double));
            if (p->gD) memcpy(gDl[l], p->gD, (size_t)Nn * sizeof(double));
            if (p->gR) memcpy(gRl[l], p->gR, (size_t)Nn * sizeof(double));
        } else {
            or_coarsen_beta(nl[l], beta[l + 1], beta[l]);
            if (p->f_mode == OR_F_LOAD) or_restrict_load(nl[l], fl[l + 1], fl[l]);
            else or_inject(nl[l], fl[l + 1], fl[l]);
            or_inject(nl[l], gDl[l + 1], gDl[l]);
            or_inject(nl[l], gRl[l + 1], gRl[l]);
        }
    }

    st->seconds_assembly = wall_seconds() - t0;  /* per-level data (coarse beta, loads, g_D) */
    int status = 0;
    for (int l = 0; l < L && !status; ++l) {
        const double ta = wall_seconds();
        const int32_t* n = nl[l];
        int64_t N = num_nodes(n);
        double h[3];
        for (int a = 0; a < 3; ++a) h[a] = (p->hi[a] - p->lo[a]) / n[a];
        int64_t* rowptr = (int64_t*)malloc((size_t)(N + 1) * sizeof(int64_t));
        int64_t* col = (int64_t*)malloc((size_t)N * 27 * sizeof(int64_t));
        double* val = (double*)malloc((size_t)N * 27 * sizeof(double));
        double* b = (double*)malloc((size_t)N * sizeof(double));
        double* gext = (double*)calloc((size_t)N, sizeof(double));
        uint8_t* mask = (uint8_t*)malloc((size_t)N);
        or_assemble_csr(n, h, beta[l], p->face_bc, p->alpha, rowptr, col, val);
        if (p->f_mode == OR_F_LOAD) memcpy(b, fl[l], (size_t)N * sizeof(double));
        else or_load_nodal(n, h, fl[l], p->face_bc, gRl[l], b);
        or_dirichlet_mask(n, p->face_bc, mask);
        for (int64_t i = 0; i < N; ++i) if (!mask[i]) gext[i] = gDl[l][i];
        const double tb = wall_seconds();
        st->seconds_assembly += tb - ta;

        double* U = U_all + off[l];
        if (l < 2) {
            /* lines 1-2: DSOLVE on the two coarsest grids */
            memcpy(U, gext, (size_t)N * sizeof(double));
            if (or_dsolve_banded(n, N, rowptr, col, val, mask, b, U)) status = 2;
            /* report the true relative residual of the direct solve */
            double* q = (double*)malloc((size_t)N * sizeof(double));
            double fh2 = 0.0, rr = 0.0;
            or_csr_matvec(N, rowptr, col, val, gext, q);
            for (int64_t i = 0; i < N; ++i) if (mask[i]) { double t = b[i] - q[i]; fh2 += t * t; }
            or_csr_matvec(N, rowptr, col, val, U, q);
            for (int64_t i = 0; i < N; ++i) if (mask[i]) { double t = b[i] - q[i]; rr += t * t; }
            st->rhs_norm[l] = sqrt(fh2);
            st->rel_res[l] = fh2 > 0 ? sqrt(rr / fh2) : sqrt(rr);
            st->iters[l] = 0;
            free(q);
        } else {
            /* line 6: W = EXP_finite(u_2h, u_4h), boundary values restored */
            double* W = W_all + off[l];
            if (exp_variant == OR_EXP_LAGRANGE27)
                or_exp_finite27(n, U_all + off[l - 1], U_all + off[l - 2], W);
            else
                or_exp_finite(n, U_all + off[l - 1], U_all + off[l - 2], W);
            for (int64_t i = 0; i < N; ++i) if (!mask[i]) W[i] = gext[i];
            /* lines 7-9: JCG from W until the relative residual test passes */
            memcpy(U, W, (size_t)N * sizeof(double));
            const int32_t steps = schedule ? or_schedule_steps(L, l, mL, sched_beta) : max_iters;
            int s = or_pcg(N, rowptr, col, val, mask, b, gext, U, rtol, steps, precond, schedule,
                           &st->iters[l], &st->rel_res[l], &st->rhs_norm[l]);
            if (s) status = s;
            /* line 10: U~ = EXP_true(u_h, u_2h) */
            or_exp_true(n, U, U_all + off[l - 1], Ut_all + off[l]);
        }
        st->seconds_solve += wall_seconds() - tb;
        free(rowptr); free(col); free(val); free(b); free(gext); free(mask);
    }
    for (int l = 0; l < L; ++l) { free(beta[l]); free(fl[l]); free(gDl[l]); free(gRl[l]); }
    st->status = status;
    return status;
}
