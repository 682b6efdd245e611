// exp.cu -- the extrapolation operators of Alg. 4 and the error norms of Sec. 5.
//
// EXP_finite (line 6; Sec. 4.2.2 and 4.3): initial guess of level l from the solutions of
// levels l-1 and l-2. Every coarse (level l-2) element covers a 5x5x5 patch of level-l nodes
// with natural coordinates xi = (a-2)/2, a = 0..4. Its interpolation values are
//   corners:            W = (5 U^1 - U^0) / 4                                  eq. (jiedian)
//   edge midpoints:     W = U^1_mid + (U^1_A - U^0_A + U^1_B - U^0_B) / 8      eq. (zhongdian)
//   (Lagrange variant)  face and body centres: mean of (zhongdian) over the diagonals
//                       through them (Remark in Sec. 4.3)
// and every patch node is sum_m N_m(xi, eta, zeta) W_m with the 20-node Serendipity functions
// of Sec. 4.3 (or the 27-node tri-quadratic Lagrange basis), evaluated below by sum
// factorisation.
//
// EXP_true (line 10; Sec. 4.2.1 and 4.3): with d = U^l - U^{l-1} at the level-(l-1) nodes,
//   U~ = U^l + (1/3) I(d),  I = trilinear interpolation from the coarse nodes,
// which is eq. (t1) at coarse nodes, eq. (chenlin) at edge centres, and the mean of (chenlin)
// over the face / space diagonals at face and body centres.
#include "exp.cuh"

#include <cstring>
#include <type_traits>

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TPB = 256;
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

// EXP_finite, one thread per level-(l-2) element. The element's interpolant is tri-quadratic
// for both variants (every Serendipity monomial has degree <= 2 in each variable), so it is
// fixed by its values at the 3x3x3 level-(l-1) nodes of the element: the 20 extrapolated
// values and, for Serendipity, the interpolant's own face and body centre values
// (N_i at a face centre: -1/4 at the face's corners, 1/2 at its edge midpoints; at the body
// centre: -1/4 at the corners, 1/4 at the edge midpoints). The fine nodes then follow by sum
// factorisation, z first, then y, then x. A thread writes the fine nodes (4 ex + a, ...),
// a = 0..3, plus a = 4 on the last element of an axis.
template <int VARIANT>
__global__ void __launch_bounds__(128) k_exp_finite(Grid g, Op op, Grid g1, const double* __restrict__ U1, Grid g0,
                                                    const double* __restrict__ U0, double* __restrict__ x,
                                                    double* __restrict__ W)
{
    COUNT_LAUNCH();
    const int64_t ne = (int64_t)g0.nx * g0.ny * g0.nz;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ne) return;
    const int ex = (int)(t % g0.nx);
    const int64_t r_ = t / g0.nx;
    const int ey = (int)(r_ % g0.ny);
    const int ez = (int)(r_ / g0.ny);
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

// EXP_true, one thread per level-(l-1) element: d = U^l - U^{l-1} at its 8 corners, divided
// by 3, interpolated trilinearly to the element's 3x3x3 level-l nodes (halves and quarters of
// corner values) and added to U^l. A thread writes the nodes (2 ex + a, ...), a = 0, 1, plus
// a = 2 on the last element of an axis.
__global__ void __launch_bounds__(128) k_exp_true(Grid g, const double* __restrict__ U1, Grid gc,
                                                  const double* __restrict__ U0, double* __restrict__ Ut)
{
    COUNT_LAUNCH();
    const int64_t ne = (int64_t)gc.nx * gc.ny * gc.nz;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ne) return;
    const int ex = (int)(t % gc.nx);
    const int64_t r_ = t / gc.nx;
    const int ey = (int)(r_ % gc.ny);
    const int ez = (int)(r_ / gc.ny);
    double D[3][3][3];  // trilinear interpolant of (U^l - U^{l-1}) / 3 at the 3x3x3 nodes
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                D[2 * c][2 * b][2 * a] = (U1[g.off(2 * (ex + a), 2 * (ey + b), 2 * (ez + c))] -
                                          U0[gc.off(ex + a, ey + b, ez + c)]) * (1.0 / 3.0);  // no FP64 divide
#pragma unroll
    for (int c = 0; c < 3; c += 2)
#pragma unroll
        for (int b = 0; b < 3; b += 2) D[c][b][1] = 0.5 * (D[c][b][0] + D[c][b][2]);
#pragma unroll
    for (int c = 0; c < 3; c += 2)
#pragma unroll
        for (int a = 0; a < 3; ++a) D[c][1][a] = 0.5 * (D[c][0][a] + D[c][2][a]);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) D[1][b][a] = 0.5 * (D[0][b][a] + D[2][b][a]);
    const int na = (ex == gc.nx - 1) ? 3 : 2, nb = (ey == gc.ny - 1) ? 3 : 2, nc = (ez == gc.nz - 1) ? 3 : 2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (c >= nc) break;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b >= nb) break;
            const int64_t orow = g.off(2 * ex, 2 * ey + b, 2 * ez + c);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a >= na) break;
                Ut[orow + a] = U1[orow + a] + D[c][b][a];
            }
        }
    }
}

// Per-block max |a-b| and sum (a-b)^2 over the owned nodes of a level.
__global__ void k_norms(Grid g, const double* __restrict__ a, const double* __restrict__ b,
                        double* __restrict__ part)
{
    COUNT_LAUNCH();
    const int64_t n = (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    double mx = 0.0, ss = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(t % (g.nx + 1));
        const int64_t rr = t / (g.nx + 1);
        const int J = (int)(rr % (g.ny + 1));
        const int K = (int)(rr / (g.ny + 1));
        const int64_t o = g.off(I, J, K);
        const double d = a[o] - (b ? b[o] : 0.0);
        mx = fmax(mx, fabs(d));
        ss = fma(d, d, ss);
    }
    __shared__ double smx[TPB / 32], sss[TPB / 32];
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        smx[warp] = mx;
        sss[warp] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w2 = 1; w2 < TPB / 32; ++w2) {
            mx = fmax(mx, smx[w2]);
            ss += sss[w2];
        }
        part[2 * blockIdx.x] = mx;
        part[2 * blockIdx.x + 1] = ss;
    }
}

inline int blocks_for(int64_t n) { return (int)((n + TPB - 1) / TPB); }
inline int64_t nodes(const Grid& g) { return (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1); }

}  // namespace

void launch_exp_finite(int variant, const Grid& g, const Op& op, const Grid& g1, const double* U1,
                       const Grid& g0, const double* U0, double* x, double* W, cudaStream_t s)
{
    const int64_t ne = (int64_t)g0.nx * g0.ny * g0.nz;
    const int nb = (int)((ne + 127) / 128);
    if (variant == 1)
        k_exp_finite<1><<<nb, 128, 0, s>>>(g, op, g1, U1, g0, U0, x, W);
    else
        k_exp_finite<0><<<nb, 128, 0, s>>>(g, op, g1, U1, g0, U0, x, W);
}

void launch_exp_true(const Grid& g, const double* U1, const Grid& gc, const double* U0, double* Ut,
                     cudaStream_t s)
{
    const int64_t ne = (int64_t)gc.nx * gc.ny * gc.nz;
    k_exp_true<<<(int)((ne + 127) / 128), 128, 0, s>>>(g, U1, gc, U0, Ut);
}

int norms_blocks(const Grid& g)
{
    int b = blocks_for(nodes(g));
    return b < 1024 ? b : 1024;
}

void launch_norms(const Grid& g, const double* a, const double* b, double* part, cudaStream_t s)
{
    k_norms<<<norms_blocks(g), TPB, 0, s>>>(g, a, b, part);
}

unsigned long long launches_exp()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
