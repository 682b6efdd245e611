// exp.cu -- the extrapolation operators of Alg. 4 and the error norms of Sec. 5.
//
// EXP_finite (line 6; Sec. 4.2.2 and 4.3): initial guess of level l from the solutions of
// levels l-1 and l-2. Every coarse (level l-2) element covers a 5x5x5 patch of level-l nodes
// with natural coordinates xi = (a-2)/2, a = 0..4. Its interpolation values are
//   corners:            W = (5 U^1 - U^0) / 4                                  eq. (jiedian)
//   edge midpoints:     W = U^1_mid + (U^1_A - U^0_A + U^1_B - U^0_B) / 8      eq. (zhongdian)
//   (Lagrange variant)  face and body centres: mean of (zhongdian) over the diagonals
//                       through them (Remark in Sec. 4.3)
// and every patch node is the fixed linear combination sum_m N_m(xi, eta, zeta) W_m with the
// 20-node Serendipity functions of Sec. 4.3 (or the 27-node tri-quadratic Lagrange basis).
// The 125 x 20 (125 x 27) weight tables are evaluated once on the host from those formulas.
//
// EXP_true (line 10; Sec. 4.2.1 and 4.3): with d = U^l - U^{l-1} at the level-(l-1) nodes,
//   U~ = U^l + (1/3) I(d),  I = trilinear interpolation from the coarse nodes,
// which is eq. (t1) at coarse nodes, eq. (chenlin) at edge centres, and the mean of (chenlin)
// over the face / space diagonals at face and body centres.
#include "exp.cuh"

#include <cstring>

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TPB = 256;
__constant__ double c_ser[125 * 20];
__constant__ double c_lag[125 * 27];

// The 20 Serendipity nodes of the patch: corners, then x-, y-, z-direction edge midpoints
// (the paper's nodes 1,5,21,25,101,105,121,125 / 3,23,103,123 / 11,15,111,115 / 51,55,71,75).
__host__ __device__ constexpr int ser_node(int m, int axis)
{
    constexpr int T[20][3] = {{0, 0, 0}, {4, 0, 0}, {0, 4, 0}, {4, 4, 0}, {0, 0, 4}, {4, 0, 4}, {0, 4, 4},
                              {4, 4, 4}, {2, 0, 0}, {2, 4, 0}, {2, 0, 4}, {2, 4, 4}, {0, 2, 0}, {4, 2, 0},
                              {0, 2, 4}, {4, 2, 4}, {0, 0, 2}, {4, 0, 2}, {0, 4, 2}, {4, 4, 2}};
    return T[m][axis];
}

__device__ __forceinline__ bool on_dirichlet(const Grid& g, const Op& op, int i, int j, int k)
{
    return (i == 0 && op.bc[0] == 0) || (i == g.nx && op.bc[1] == 0) ||
           (j == 0 && op.bc[2] == 0) || (j == g.ny && op.bc[3] == 0) ||
           (k == 0 && op.bc[4] == 0) || (k == g.nz && op.bc[5] == 0);
}

// Value of the coarse-grid interpolation node (local patch position a, b, c in {0,2,4})
// from U^1 (level l-1, grid g1) and U^0 (level l-2, grid g0) for the element (ex, ey, ez).
struct Src {
    Grid g1, g0;
    const double* U1;
    const double* U0;
    int ex, ey, ez;
    __device__ __forceinline__ double u1(int a, int b, int c) const
    {
        return U1[g1.off(2 * ex + a / 2, 2 * ey + b / 2, 2 * ez + c / 2)];
    }
    __device__ __forceinline__ double d(int a, int b, int c) const  // U^1 - U^0 at a corner
    {
        return u1(a, b, c) - U0[g0.off(ex + a / 4, ey + b / 4, ez + c / 4)];
    }
};

template <int VARIANT>
__global__ void k_exp_finite(Grid g, Op op, Grid g1, const double* __restrict__ U1, Grid g0,
                             const double* __restrict__ U0, double* __restrict__ x,
                             double* __restrict__ W)
{
    COUNT_LAUNCH();
    const int64_t n = (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int I = (int)(t % (g.nx + 1));
    const int64_t rr = t / (g.nx + 1);
    const int J = (int)(rr % (g.ny + 1));
    const int K = (int)(rr / (g.ny + 1));
    const int64_t o = g.off(I, J, K);
    if (on_dirichlet(g, op, I, J, K)) {
        W[o] = x[o];
        return;
    }
    Src s{g1, g0, U1, U0, min(I >> 2, g0.nx - 1), min(J >> 2, g0.ny - 1), min(K >> 2, g0.nz - 1)};
    const int a = I - 4 * s.ex, b = J - 4 * s.ey, c = K - 4 * s.ez;
    const int pt = a + 5 * b + 25 * c;
    double w = 0.0;
    if (VARIANT == 0) {
#pragma unroll
        for (int m = 0; m < 20; ++m) {
            const int na = ser_node(m, 0), nb = ser_node(m, 1), nc = ser_node(m, 2);
            double v;
            if (m < 8) {
                v = s.u1(na, nb, nc) + s.d(na, nb, nc) / 4.0;  // (5 U^1 - U^0)/4
            } else {
                const int dir = (m < 12) ? 0 : (m < 16) ? 1 : 2;
                int A[3] = {na, nb, nc}, B[3] = {na, nb, nc};
                A[dir] = 0;
                B[dir] = 4;
                v = s.u1(na, nb, nc) + (s.d(A[0], A[1], A[2]) + s.d(B[0], B[1], B[2])) / 8.0;
            }
            w += c_ser[pt * 20 + m] * v;
        }
    } else {
        // 27 values at the level-(l-1) nodes of the element, (zhongdian) averaged over every
        // diagonal through the non-corner ones
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int qa = 2 * (q % 3), qb = 2 * ((q / 3) % 3), qc = 2 * (q / 9);
            const int nodd = (qa == 2) + (qb == 2) + (qc == 2);
            double v;
            if (nodd == 0) {
                v = s.u1(qa, qb, qc) + s.d(qa, qb, qc) / 4.0;  // (5 U^1 - U^0)/4
            } else {
                // (zhongdian) on one diagonal adds (d_A + d_B)/8; the mean over the 2^(nodd-1)
                // diagonals adds (sum of d over the 2^nodd corners) / 2^(nodd+2)
                double sum = 0.0;
                for (int cc = 0; cc < 8; ++cc) {
                    const int ca = (qa == 2) ? 4 * (cc & 1) : qa;
                    const int cb = (qb == 2) ? 4 * ((cc >> 1) & 1) : qb;
                    const int cz = (qc == 2) ? 4 * (cc >> 2) : qc;
                    if ((qa != 2 && (cc & 1)) || (qb != 2 && ((cc >> 1) & 1)) || (qc != 2 && (cc >> 2)))
                        continue;
                    sum += s.d(ca, cb, cz);
                }
                v = s.u1(qa, qb, qc) + sum / (double)(4 << nodd);
            }
            w += c_lag[pt * 27 + q] * v;
        }
    }
    x[o] = w;
    W[o] = w;
}

__global__ void k_exp_true(Grid g, const double* __restrict__ U1, Grid gc, const double* __restrict__ U0,
                           double* __restrict__ Ut)
{
    COUNT_LAUNCH();
    const int64_t n = (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int I = (int)(t % (g.nx + 1));
    const int64_t rr = t / (g.nx + 1);
    const int J = (int)(rr % (g.ny + 1));
    const int K = (int)(rr / (g.ny + 1));
    const int oi = I & 1, oj = J & 1, ok = K & 1;
    double s = 0.0;
    for (int c = 0; c <= ok; ++c)
        for (int b = 0; b <= oj; ++b)
            for (int a = 0; a <= oi; ++a) {
                const int ci = (I >> 1) + a, cj = (J >> 1) + b, ck = (K >> 1) + c;
                s += U1[g.off(2 * ci, 2 * cj, 2 * ck)] - U0[gc.off(ci, cj, ck)];
            }
    const double scale = 1.0 / (3.0 * (double)(1 << (oi + oj + ok)));
    const int64_t o = g.off(I, J, K);
    Ut[o] = U1[o] + scale * s;
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

// Host evaluation of the interpolation weights of every patch point.
void ser_weights(double* out)
{
    for (int c = 0; c < 5; ++c)
        for (int b = 0; b < 5; ++b)
            for (int a = 0; a < 5; ++a) {
                const double xi = (a - 2) / 2.0, eta = (b - 2) / 2.0, zeta = (c - 2) / 2.0;
                for (int m = 0; m < 20; ++m) {
                    const double xi_i = (ser_node(m, 0) - 2) / 2.0, eta_i = (ser_node(m, 1) - 2) / 2.0,
                                 zeta_i = (ser_node(m, 2) - 2) / 2.0;
                    double N;
                    if (m < 8)
                        N = 0.125 * (1 + xi_i * xi) * (1 + eta_i * eta) * (1 + zeta_i * zeta) *
                            (xi_i * xi + eta_i * eta + zeta_i * zeta - 2);
                    else if (m < 12)
                        N = 0.25 * (1 - xi * xi) * (1 + eta_i * eta) * (1 + zeta_i * zeta);
                    else if (m < 16)
                        N = 0.25 * (1 - eta * eta) * (1 + xi_i * xi) * (1 + zeta_i * zeta);
                    else
                        N = 0.25 * (1 - zeta * zeta) * (1 + xi_i * xi) * (1 + eta_i * eta);
                    out[(a + 5 * b + 25 * c) * 20 + m] = N;
                }
            }
}

void lag_weights(double* out)
{
    auto L = [](int node, double t) {
        return node == 0 ? 0.5 * t * (t - 1) : node == 1 ? 1 - t * t : 0.5 * t * (t + 1);
    };
    for (int c = 0; c < 5; ++c)
        for (int b = 0; b < 5; ++b)
            for (int a = 0; a < 5; ++a)
                for (int q = 0; q < 27; ++q)
                    out[(a + 5 * b + 25 * c) * 27 + q] =
                        L(q % 3, (a - 2) / 2.0) * L((q / 3) % 3, (b - 2) / 2.0) * L(q / 9, (c - 2) / 2.0);
}

inline int blocks_for(int64_t n) { return (int)((n + TPB - 1) / TPB); }
inline int64_t nodes(const Grid& g) { return (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1); }

}  // namespace

cudaError_t exp_init_tables()
{
    static double ser[125 * 20], lag[125 * 27];
    ser_weights(ser);
    lag_weights(lag);
    cudaError_t e = cudaMemcpyToSymbol(c_ser, ser, sizeof(ser));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_lag, lag, sizeof(lag));
}

void launch_exp_finite(int variant, const Grid& g, const Op& op, const Grid& g1, const double* U1,
                       const Grid& g0, const double* U0, double* x, double* W, cudaStream_t s)
{
    if (variant == 1)
        k_exp_finite<1><<<blocks_for(nodes(g)), TPB, 0, s>>>(g, op, g1, U1, g0, U0, x, W);
    else
        k_exp_finite<0><<<blocks_for(nodes(g)), TPB, 0, s>>>(g, op, g1, U1, g0, U0, x, W);
}

void launch_exp_true(const Grid& g, const double* U1, const Grid& gc, const double* U0, double* Ut,
                     cudaStream_t s)
{
    k_exp_true<<<blocks_for(nodes(g)), TPB, 0, s>>>(g, U1, gc, U0, Ut);
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
