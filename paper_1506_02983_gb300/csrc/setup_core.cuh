// setup_core.cuh -- per-point bodies of the level set-up of Alg. 4 (Sec. 2), shared by the
// single-problem kernels (setup.cu) and the batched ones (batch.cu).
#pragma once

#include "ecmg_internal.cuh"
#include "stencil_core.cuh"

namespace ecmg {

// Coarse element (i, j, k) of grid gc: mean of its 8 children on the finer grid gf, summed x
// fastest then y then z.
__device__ __forceinline__ double coarse_beta_at(const double* __restrict__ bf, const Grid& gf, int i, int j, int k)
{
    double s = 0.0;
    for (int c = 0; c < 8; ++c)
        s += bf[gf.off(2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + (c >> 2))];
    return s / 8.0;
}

// b_c = P^T b_f at coarse node (i, j, k), P the trilinear prolongation: fine node 2I + d
// contributes with weight prod_a w(d_a), w(0) = 1, w(+-1) = 1/2. Fine ghost nodes hold 0, so
// no bounds checks.
__device__ __forceinline__ double restrict_at(const double* __restrict__ bf, const Grid& gf, int i, int j, int k)
{
    double s = 0.0;
    for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                double w = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0);
                s += w * bf[gf.off(2 * i + di, 2 * j + dj, 2 * k + dk)];
            }
    return s;
}

// Element count along one axis between node index a and a + d (d in -1..1).
__device__ __forceinline__ int cnt1(int a, int n, int d)
{
    if (d < 0) return a >= 1;
    if (d > 0) return a < n;
    return (a >= 1) + (a < n);
}

// sum over the Robin faces through node (i, j, k) of (M_F gR_I)_i, the consistent face mass of
// the nodal interpolant of g_R (the face term of the load of Sec. 2): a tensor product of the 1D
// masses m(0) = h/3, m(+-1) = h/6 per element over the face's two axes.
__device__ __forceinline__ double robin_load_at(const Grid& g, const Op& op, const double* __restrict__ gR, int i,
                                                int j, int k)
{
    const int idx[3] = {i, j, k};
    const int nn[3] = {g.nx, g.ny, g.nz};
    double s = 0.0;
    for (int fc = 0; fc < 6; ++fc) {
        if (op.bc[fc] != 1) continue;
        const int an = fc / 2;
        if (idx[an] != ((fc & 1) ? nn[an] : 0)) continue;
        const int aa = (an == 0) ? 1 : 0, ab = (an == 2) ? 1 : 2;
        for (int db = -1; db <= 1; ++db)
            for (int da = -1; da <= 1; ++da) {
                const double w = cnt1(idx[aa], nn[aa], da) * (g.h[aa] * (da ? (1.0 / 6.0) : (1.0 / 3.0))) *
                                 (cnt1(idx[ab], nn[ab], db) * (g.h[ab] * (db ? (1.0 / 6.0) : (1.0 / 3.0))));
                if (w == 0.0) continue;
                int o[3] = {0, 0, 0};
                o[aa] = da;
                o[ab] = db;
                s += w * gR[g.off(i + o[0], j + o[1], k + o[2])];
            }
    }
    return s;
}

// b_i = (M f_I + sum over Robin faces of M_F gR_I)_i with the consistent mass matrices of
// Sec. 2. The element mass is a tensor product, so the assembled row is
// prod_a cnt_a(d_a) m_a(d_a), m(0) = h/3 and m(+-1) = h/6 per element, and the sum over the
// 3x3x3 neighbours factorises: x first, then y, then z (no FP64 division per node).
__device__ __forceinline__ double nodal_load_at(const Grid& g, const Op& op, const double* __restrict__ f,
                                                const double* __restrict__ gR, int i, int j, int k)
{
    const int idx[3] = {i, j, k};
    const int nn[3] = {g.nx, g.ny, g.nz};
    double wa[3][3];
    for (int a = 0; a < 3; ++a)
        for (int d = -1; d <= 1; ++d)
            wa[a][d + 1] = cnt1(idx[a], nn[a], d) * (g.h[a] * (d ? (1.0 / 6.0) : (1.0 / 3.0)));
    double s = 0.0;
    for (int dk = -1; dk <= 1; ++dk) {
        if (wa[2][dk + 1] == 0.0) continue;
        double sz = 0.0;
        for (int dj = -1; dj <= 1; ++dj) {
            if (wa[1][dj + 1] == 0.0) continue;
            const double* row = f + g.off(i - 1, j + dj, k + dk);
            sz = fma(wa[1][dj + 1], fma(wa[0][0], row[0], fma(wa[0][1], row[1], wa[0][2] * row[2])), sz);
        }
        s = fma(wa[2][dk + 1], sz, s);
    }
    if (gR) s += robin_load_at(g, op, gR, i, j, k);
    return s;
}

// The 3-point Gauss-Legendre rule on [0, 1]: nodes (1 -+ sqrt(3/5)) / 2 and 1/2, weights 5/18,
// 8/18, 5/18; the layout of f at the rule's points (ECMG_F_GAUSS) takes the nodes in this order.
constexpr double GAUSS3_OFF = 0.38729833462074168852;  // sqrt(3/5) / 2
__device__ __forceinline__ double gauss3_node(int q) { return q == 0 ? 0.5 - GAUSS3_OFF : (q == 1 ? 0.5 : 0.5 + GAUSS3_OFF); }
__device__ __forceinline__ double gauss3_weight(int q) { return q == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }

// b_i = int f phi_i of the weak form of Sec. 2 by the 3x3x3 Gauss rule on every element around
// node i, with f given at the rule's points of every element of the level (f27: 27 values per
// element, elements x fastest, then the points qx fastest, qy, qz), plus the Robin face terms of
// nodal_load_at. On an element where the node is corner (cx, cy, cz), its hat at point q is
// prod_a (c_a ? t_qa : 1 - t_qa); the sum runs over the points axis by axis.
__device__ __forceinline__ double gauss_load_at(const Grid& g, const Op& op, const double* __restrict__ f27,
                                                const double* __restrict__ gR, int i, int j, int k)
{
    const double vol = g.h[0] * g.h[1] * g.h[2];
    double s = 0.0;
    for (int dz = 0; dz < 2; ++dz) {
        const int ez = k - 1 + dz;
        if (ez < 0 || ez >= g.nz) continue;
        for (int dy = 0; dy < 2; ++dy) {
            const int ey = j - 1 + dy;
            if (ey < 0 || ey >= g.ny) continue;
            for (int dx = 0; dx < 2; ++dx) {
                const int ex = i - 1 + dx;
                if (ex < 0 || ex >= g.nx) continue;
                // the node is corner (1 - dx, 1 - dy, 1 - dz) of this element
                const double* fe = f27 + 27 * (ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez));
                double sz = 0.0;
                for (int qz = 0; qz < 3; ++qz) {
                    double sy = 0.0;
                    for (int qy = 0; qy < 3; ++qy) {
                        double sx = 0.0;
                        for (int qx = 0; qx < 3; ++qx) {
                            const double t = gauss3_node(qx);
                            sx = fma(gauss3_weight(qx) * (dx ? 1.0 - t : t), fe[qx + 3 * qy + 9 * qz], sx);
                        }
                        const double t = gauss3_node(qy);
                        sy = fma(gauss3_weight(qy) * (dy ? 1.0 - t : t), sx, sy);
                    }
                    const double t = gauss3_node(qz);
                    sz = fma(gauss3_weight(qz) * (dz ? 1.0 - t : t), sy, sz);
                }
                s = fma(vol, sz, s);
            }
        }
    }
    if (gR) s += robin_load_at(g, op, gR, i, j, k);
    return s;
}

// The same diagonal in FP32 arithmetic from the FP32 betas, for the FP32 iteration of MIXED
// mode: no FP64 division or conversion per node (FP64 runs at 1/64 of the FP32 rate on GB300).
// Robin terms (boundary nodes only) are formed in FP64 and rounded.
// precond 0: the identity on free nodes (plain CG, ECMG_cg).
__device__ __forceinline__ float jacobi32_at(const Grid& g, const Op& op, const float* __restrict__ beta32, int i, int j,
                                            int k, int precond = 1)
{
    if (!precond) return on_dirichlet(g, op, i, j, k) ? 0.f : 1.f;
    float B = 0.f;
    for (int c = 0; c < 8; ++c)
        B += beta32[g.off(i - 1 + (c & 1), j - 1 + ((c >> 1) & 1), k - 1 + (c >> 2))];
    float d = __fmul_rn(op.w032, B);
    if (op.robin && (i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz)) {
        const int idx[3] = {i, j, k};
        const int nn[3] = {g.nx, g.ny, g.nz};
        for (int fc = 0; fc < 6; ++fc) {
            if (!((op.robin_mask >> fc) & 1)) continue;
            int an = fc / 2;
            if (idx[an] != ((fc & 1) ? nn[an] : 0)) continue;
            int aa = (an == 0) ? 1 : 0, ab = (an == 2) ? 1 : 2;
            // alpha h_a h_b / 9 per shared face quad pair, in FP32 (host-rounded weight)
            d += op.rw32[fc] * (float)(4 * cnt1(idx[aa], nn[aa], 0) * cnt1(idx[ab], nn[ab], 0));
        }
    }
    return on_dirichlet(g, op, i, j, k) ? 0.f : __frcp_rn(d);
}

}  // namespace ecmg
