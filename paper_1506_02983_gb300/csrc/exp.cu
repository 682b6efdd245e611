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

#include "exp_core.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TPB = 256;
// EXP_finite: one thread per level-(l-2) element.
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
    exp_finite_element<VARIANT>(g, op, g1, U1, g0, U0, x, W, ex, ey, ez);
}

// EXP_true: one thread per level-(l-1) element.
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
    exp_true_element(g, U1, gc, U0, Ut, ex, ey, ez);
}

// Per-block max |a-b| and sum (a-b)^2 over the owned nodes of a level. The max is taken over
// the bit patterns of |a-b| as unsigned integers: for non-negative doubles that order is the
// numeric one, and every NaN (sign cleared) sorts above +inf, so a NaN anywhere in a - b makes
// the max NaN instead of dropping out as it would with fmax (an error norm must not hide one).
__global__ void k_norms(Grid g, const double* __restrict__ a, const double* __restrict__ b,
                        double* __restrict__ part)
{
    COUNT_LAUNCH();
    const int64_t n = (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    unsigned long long mx = 0ull;
    double ss = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(t % (g.nx + 1));
        const int64_t rr = t / (g.nx + 1);
        const int J = (int)(rr % (g.ny + 1));
        const int K = (int)(rr / (g.ny + 1));
        const int64_t o = g.off(I, J, K);
        const double d = a[o] - (b ? b[o] : 0.0);
        mx = max(mx, (unsigned long long)__double_as_longlong(fabs(d)));
        ss = fma(d, d, ss);
    }
    __shared__ unsigned long long smx[TPB / 32];
    __shared__ double sss[TPB / 32];
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
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
            mx = max(mx, smx[w2]);
            ss += sss[w2];
        }
        part[2 * blockIdx.x] = __longlong_as_double((long long)mx);
        part[2 * blockIdx.x + 1] = ss;
    }
}

inline int blocks_for(int64_t n) { return (int)((n + TPB - 1) / TPB); }
__host__ __device__ inline int64_t nodes(const Grid& g) { return (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1); }

// EXP_true in two passes: d = U^l - U^{l-1} at every level-(l-1) node into D (grid gc), one
// subtraction per node; then one thread per level-(l-1) element from D.
__global__ void __launch_bounds__(TPB) k_exp_true_d(Grid g, const double* __restrict__ U1, Grid gc,
                                                    const double* __restrict__ U0, double* __restrict__ D)
{
    COUNT_LAUNCH();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nodes(gc)) return;
    const int i = (int)(t % (gc.nx + 1));
    const int64_t r_ = t / (gc.nx + 1);
    const int j = (int)(r_ % (gc.ny + 1));
    const int k = (int)(r_ / (gc.ny + 1));
    const int64_t o = gc.off(i, j, k);
    D[o] = U1[g.off(2 * i, 2 * j, 2 * k)] - U0[o];
}
__global__ void __launch_bounds__(128) k_exp_true_from_d(Grid g, const double* __restrict__ U1, Grid gc,
                                                         const double* __restrict__ D, double* __restrict__ Ut)
{
    COUNT_LAUNCH();
    const int64_t ne = (int64_t)gc.nx * gc.ny * gc.nz;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ne) return;
    const int ex = (int)(t % gc.nx);
    const int64_t r_ = t / gc.nx;
    const int ey = (int)(r_ % gc.ny);
    const int ez = (int)(r_ / gc.ny);
    exp_true_element_d(g, U1, gc, D, Ut, ex, ey, ez);
}

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
                     cudaStream_t s, double* D)
{
    const int64_t ne = (int64_t)gc.nx * gc.ny * gc.nz;
    if (D) {
        k_exp_true_d<<<blocks_for(nodes(gc)), TPB, 0, s>>>(g, U1, gc, U0, D);
        k_exp_true_from_d<<<(int)((ne + 127) / 128), 128, 0, s>>>(g, U1, gc, D, Ut);
        return;
    }
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
