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
    if (gR) {
        for (int fc = 0; fc < 6; ++fc) {
            if (op.bc[fc] != 1) continue;
            int an = fc / 2;
            if (idx[an] != ((fc & 1) ? nn[an] : 0)) continue;
            int aa = (an == 0) ? 1 : 0, ab = (an == 2) ? 1 : 2;
            for (int db = -1; db <= 1; ++db)
                for (int da = -1; da <= 1; ++da) {
                    double w = wa[aa][da + 1] * wa[ab][db + 1];
                    if (w == 0.0) continue;
                    int o[3] = {0, 0, 0};
                    o[aa] = da;
                    o[ab] = db;
                    s += w * gR[g.off(i + o[0], j + o[1], k + o[2])];
                }
        }
    }
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
