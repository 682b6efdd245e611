// exp_core.cuh -- the per-element bodies of EXP_finite and EXP_true (Alg. 4 lines 6 and 10;
// Sec. 4.2 and 4.3), shared by the single-problem kernels (exp.cu) and the batched ones
// (batch.cu). Formulas and notation: exp.cu.
#pragma once

#include <type_traits>

#include "ecmg_internal.cuh"

namespace ecmg {

// Quadratic Lagrange interpolation on the nodes -1, 0, 1 (values v0, v1, v2) at the five
// points -1, -1/2, 0, 1/2, 1 (m = 0..4).
template <int M>
__device__ __forceinline__ double quad5(double v0, double v1, double v2)
{
    if (M == 0) return v0;
    if (M == 2) return v1;
    if (M == 4) return v2;
    if (M == 1) return fma(0.375, v0, fma(0.75, v1, -0.125 * v2));
    return fma(-0.125, v0, fma(0.75, v1, 0.375 * v2));
}

// EXP_finite, for the level-(l-2) element (ex, ey, ez). The element's interpolant is tri-quadratic
// for both variants (every Serendipity monomial has degree <= 2 in each variable), so it is
// fixed by its values at the 3x3x3 level-(l-1) nodes of the element: the 20 extrapolated
// values and, for Serendipity, the interpolant's own face and body centre values
// (N_i at a face centre: -1/4 at the face's corners, 1/2 at its edge midpoints; at the body
// centre: -1/4 at the corners, 1/4 at the edge midpoints). The fine nodes then follow by sum
// factorisation, z first, then y, then x. A thread writes the fine nodes (4 ex + a, ...),
// a = 0..3, plus a = 4 on the last element of an axis.
template <int VARIANT>
__device__ __forceinline__ void exp_finite_element(const Grid& g, const Op& op, const Grid& g1,
                                                   const double* __restrict__ U1, const Grid& g0,
                                                   const double* __restrict__ U0, double* __restrict__ x,
                                                   double* __restrict__ W, int ex, int ey, int ez)
{
    double u1[3][3][3], d[2][2][2], V[3][3][3];  // [c][b][a]
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) u1[c][b][a] = U1[g1.off(2 * ex + a, 2 * ey + b, 2 * ez + c)];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) d[c][b][a] = u1[2 * c][2 * b][2 * a] - U0[g0.off(ex + a, ey + b, ez + c)];
    // corners: eq. (jiedian); edge midpoints: eq. (zhongdian) along the edge
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int nodd = (a == 1) + (b == 1) + (c == 1);
                if (nodd == 0) {
                    V[c][b][a] = fma(0.25, d[c / 2][b / 2][a / 2], u1[c][b][a]);
                } else if (nodd == 1) {
                    const double sd = (a == 1) ? d[c / 2][b / 2][0] + d[c / 2][b / 2][1]
                                    : (b == 1) ? d[c / 2][0][a / 2] + d[c / 2][1][a / 2]
                                               : d[0][b / 2][a / 2] + d[1][b / 2][a / 2];
                    V[c][b][a] = fma(0.125, sd, u1[c][b][a]);
                }
            }
    if (VARIANT == 0) {
        // face and body centres of the Serendipity interpolant
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int nodd = (a == 1) + (b == 1) + (c == 1);
                    if (nodd == 2) {
                        double corners, edges;
                        if (c != 1) {  // face normal z
                            corners = V[c][0][0] + V[c][0][2] + V[c][2][0] + V[c][2][2];
                            edges = V[c][1][0] + V[c][1][2] + V[c][0][1] + V[c][2][1];
                        } else if (b != 1) {  // face normal y
                            corners = V[0][b][0] + V[0][b][2] + V[2][b][0] + V[2][b][2];
                            edges = V[1][b][0] + V[1][b][2] + V[0][b][1] + V[2][b][1];
                        } else {  // face normal x
                            corners = V[0][0][a] + V[0][2][a] + V[2][0][a] + V[2][2][a];
                            edges = V[1][0][a] + V[1][2][a] + V[0][1][a] + V[2][1][a];
                        }
                        V[c][b][a] = fma(0.5, edges, -0.25 * corners);
                    }
                }
        double corners = 0.0, edges = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int nodd = (a == 1) + (b == 1) + (c == 1);
                    if (nodd == 0) corners += V[c][b][a];
                    if (nodd == 1) edges += V[c][b][a];
                }
        V[1][1][1] = 0.25 * (edges - corners);
    } else {
        // Remark of Sec. 4.3: (zhongdian) averaged over the diagonals through the centre
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int nodd = (a == 1) + (b == 1) + (c == 1);
                    if (nodd < 2) continue;
                    double sd = 0.0;
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                            for (int aa = 0; aa < 2; ++aa) {
                                if ((a != 1 && aa != a / 2) || (b != 1 && bb != b / 2) || (c != 1 && cc != c / 2)) continue;
                                sd += d[cc][bb][aa];
                            }
                    V[c][b][a] = fma(nodd == 2 ? 1.0 / 16.0 : 1.0 / 32.0, sd, u1[c][b][a]);
                }
    }
    // sum factorisation over the owned fine nodes
    const int na = (ex == g0.nx - 1) ? 5 : 4, nb = (ey == g0.ny - 1) ? 5 : 4, nc = (ez == g0.nz - 1) ? 5 : 4;
    const bool dx0 = op.bc[0] == 0, dx1 = op.bc[1] == 0, dy0 = op.bc[2] == 0, dy1 = op.bc[3] == 0;
    const bool dz0 = op.bc[4] == 0, dz1 = op.bc[5] == 0;
    auto zstage = [&](auto mc, int c) {
        constexpr int MC = decltype(mc)::value;
        double Z[3][3];
#pragma unroll
        for (int qb = 0; qb < 3; ++qb)
#pragma unroll
            for (int qa = 0; qa < 3; ++qa) Z[qb][qa] = quad5<MC>(V[0][qb][qa], V[1][qb][qa], V[2][qb][qa]);
        const int K = 4 * ez + c;
        const bool dk = (dz0 && K == 0) || (dz1 && K == g.nz);
        auto ystage = [&](auto mb, int b) {
            constexpr int MB = decltype(mb)::value;
            double Y[3];
#pragma unroll
            for (int qa = 0; qa < 3; ++qa) Y[qa] = quad5<MB>(Z[0][qa], Z[1][qa], Z[2][qa]);
            const int J = 4 * ey + b;
            const bool djk = dk || (dy0 && J == 0) || (dy1 && J == g.ny);
            const int64_t orow = g.off(4 * ex, J, K);
            auto put = [&](int a, double w) {
                const int I = 4 * ex + a;
                const int64_t o = orow + a;
                if (djk || (dx0 && I == 0) || (dx1 && I == g.nx)) {
                    W[o] = x[o];
                } else {
                    x[o] = w;
                    W[o] = w;
                }
            };
            put(0, quad5<0>(Y[0], Y[1], Y[2]));
            put(1, quad5<1>(Y[0], Y[1], Y[2]));
            put(2, quad5<2>(Y[0], Y[1], Y[2]));
            put(3, quad5<3>(Y[0], Y[1], Y[2]));
            if (na == 5) put(4, quad5<4>(Y[0], Y[1], Y[2]));
        };
        ystage(std::integral_constant<int, 0>(), 0);
        ystage(std::integral_constant<int, 1>(), 1);
        ystage(std::integral_constant<int, 2>(), 2);
        ystage(std::integral_constant<int, 3>(), 3);
        if (nb == 5) ystage(std::integral_constant<int, 4>(), 4);
    };
    zstage(std::integral_constant<int, 0>(), 0);
    zstage(std::integral_constant<int, 1>(), 1);
    zstage(std::integral_constant<int, 2>(), 2);
    zstage(std::integral_constant<int, 3>(), 3);
    if (nc == 5) zstage(std::integral_constant<int, 4>(), 4);
}

// EXP_true, for the level-(l-1) element (ex, ey, ez): d = U^l - U^{l-1} at its 8 corners,
// interpolated trilinearly to the element's 3x3x3 level-l nodes, divided by 3 and added to U^l.
// The trilinear interpolant at a node with m midpoint coordinates is the sum of the 2^m
// nearest corner values divided by 2^m, so the corner differences are summed by sum
// factorisation (x, then y, then z) and each node takes one FMA with the weight 1/(3 2^m):
// 28 FP64 operations for the 8 owned nodes instead of 62 with averaged values. A thread
// writes the nodes (2 ex + a, ...), a = 0, 1, plus a = 2 on the last element of an axis.
__device__ __forceinline__ void exp_true_from_d(const Grid& g, const double* __restrict__ U1, const Grid& gc,
                                                const double (&d)[2][2][2], double* __restrict__ Ut, int ex, int ey,
                                                int ez)
{
    const double w[4] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 12.0, 1.0 / 24.0};  // 1 / (3 2^m)
    const int na = (ex == gc.nx - 1) ? 3 : 2, nb = (ey == gc.ny - 1) ? 3 : 2, nc = (ez == gc.nz - 1) ? 3 : 2;
    // level-l node offset a (0, 1 = midpoint, 2) from the corner pair (v0, v1) along one axis
    auto pick = [](int a, double v0, double v1) { return a == 0 ? v0 : (a == 2 ? v1 : v0 + v1); };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= na) break;
        double X[2][2];  // [c][b]
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) X[c][b] = pick(a, d[c][b][0], d[c][b][1]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b >= nb) break;
            const double Y0 = pick(b, X[0][0], X[0][1]), Y1 = pick(b, X[1][0], X[1][1]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c >= nc) break;
                const double S = pick(c, Y0, Y1);
                const int64_t o = g.off(2 * ex + a, 2 * ey + b, 2 * ez + c);
                Ut[o] = fma(S, w[(a == 1) + (b == 1) + (c == 1)], U1[o]);
            }
        }
    }
}

__device__ __forceinline__ void exp_true_element(const Grid& g, const double* __restrict__ U1, const Grid& gc,
                                                 const double* __restrict__ U0, double* __restrict__ Ut, int ex,
                                                 int ey, int ez)
{
    double d[2][2][2];  // [c][b][a]
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                d[c][b][a] = U1[g.off(2 * (ex + a), 2 * (ey + b), 2 * (ez + c))] - U0[gc.off(ex + a, ey + b, ez + c)];
    exp_true_from_d(g, U1, gc, d, Ut, ex, ey, ez);
}

// The same with d already formed at the level-(l-1) nodes (D, on grid gc): a corner difference is
// then one load instead of a subtraction that the eight elements sharing the node each repeat
// (7 of the element's 28 FP64 operations); same values, so the same Ut bit for bit.
__device__ __forceinline__ void exp_true_element_d(const Grid& g, const double* __restrict__ U1, const Grid& gc,
                                                   const double* __restrict__ D, double* __restrict__ Ut, int ex,
                                                   int ey, int ez)
{
    double d[2][2][2];  // [c][b][a]
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) d[c][b][a] = D[gc.off(ex + a, ey + b, ez + c)];
    exp_true_from_d(g, U1, gc, d, Ut, ex, ey, ez);
}

}  // namespace ecmg
