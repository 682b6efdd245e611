// separable.cu -- on-device load assembly from separable data (ECMG_F_SEPARABLE) and separable
// Dirichlet data.
//
// For f = sum_t fx_t(x) fy_t(y) fz_t(z) the load functional of Sec. 2, b_i = int f phi_i with
// the trilinear hat phi_i = phi_i(x) phi_j(y) phi_k(z), factorises into 1D hat integrals:
//     b_(i,j,k) = sum_t Hx_t[i] Hy_t[j] Hz_t[k],   Ha_t[i] = int fa_t(s) phi_i(s) ds,
// and the 1D integrals come from 3-point Gauss-Legendre quadrature on every element interval
// (exact for the hat times any polynomial of degree <= 4). Coarser levels take the exact coarse
// functional P^T b, which factorises the same way: each 1D factor is restricted with the 1D
// prolongation weights (1 at the coincident node, 1/2 at the two neighbours). Nodal Dirichlet
// data sum_t gx_t(x) gy_t(y) gz_t(z) injects factor by factor (every second node). The caller
// therefore passes O(T n) numbers instead of N nodal values.
#include "ecmg_internal.cuh"
#include "separable.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TPB = 256;
constexpr int TX = 32, TY = 8;

__host__ __device__ inline int sum_nodes(const Grid& g) { return (g.nx + 1) + (g.ny + 1) + (g.nz + 1); }

// 1D hat integrals of the finest level from Gauss samples: one thread per (term, axis node).
// samples: term-major, then x (3 per interval, interval-major), y, z.
__global__ void k_sep_hat(Grid g, int terms, const double* __restrict__ samples, double* __restrict__ H)
{
    COUNT_LAUNCH();
    const int per = sum_nodes(g);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= terms * per) return;
    const int term = t / per;
    int idx = t % per, a = 0, n = g.nx, soff = 0;
    if (idx > g.nx) {
        idx -= g.nx + 1;
        a = 1;
        n = g.ny;
        soff = 3 * g.nx;
        if (idx > g.ny) {
            idx -= g.ny + 1;
            a = 2;
            n = g.nz;
            soff = 3 * (g.nx + g.ny);
        }
    }
    // 3-point Gauss-Legendre on [0, 1]: nodes (1 -+ sqrt(3/5)) / 2 and 1/2, weights 5/18, 8/18
    const double r = sqrt(0.6);
    const double gq[3] = {0.5 * (1.0 - r), 0.5, 0.5 * (1.0 + r)};
    const double wq[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    const double* s = samples + (size_t)term * 3 * (g.nx + g.ny + g.nz) + soff;
    double acc = 0.0;
    if (idx >= 1)  // interval idx-1: the hat rises, phi = local coordinate
        for (int q = 0; q < 3; ++q) acc = fma(wq[q] * gq[q], s[3 * (idx - 1) + q], acc);
    if (idx < n)   // interval idx: the hat falls, phi = 1 - local coordinate
        for (int q = 0; q < 3; ++q) acc = fma(wq[q] * (1.0 - gq[q]), s[3 * idx + q], acc);
    H[t] = acc * g.h[a];
}

// Coarse 1D factors from the fine ones: restriction (load, P^T) or injection (nodal data).
__global__ void k_sep_coarsen(Grid gc, Grid gf, int terms, const double* __restrict__ Ff, double* __restrict__ Fc,
                              int restrict_)
{
    COUNT_LAUNCH();
    const int pc = sum_nodes(gc), pf = sum_nodes(gf);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= terms * pc) return;
    const int term = t / pc;
    int idx = t % pc, base = 0, nf = gf.nx;
    if (idx > gc.nx) {
        idx -= gc.nx + 1;
        base = gf.nx + 1;
        nf = gf.ny;
        if (idx > gc.ny) {
            idx -= gc.ny + 1;
            base += gf.ny + 1;
            nf = gf.nz;
        }
    }
    const double* f = Ff + (size_t)term * pf + base;
    double v = f[2 * idx];
    if (restrict_) {
        if (2 * idx - 1 >= 0) v += 0.5 * f[2 * idx - 1];
        if (2 * idx + 1 <= nf) v += 0.5 * f[2 * idx + 1];
    }
    Fc[t] = v;
}

// out(i, j, k) = sum_t Fx_t[i] Fy_t[j] Fz_t[k] on every node of the level.
__global__ void k_sep_outer(Grid g, int terms, const double* __restrict__ F, double* __restrict__ out)
{
    COUNT_LAUNCH();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y, k = blockIdx.z;
    if (i > g.nx || j > g.ny) return;
    const int per = sum_nodes(g);
    double v = 0.0;
    for (int t = 0; t < terms; ++t) {
        const double* f = F + (size_t)t * per;
        v = fma(f[i] * f[g.nx + 1 + j], f[g.nx + g.ny + 2 + k], v);
    }
    out[g.off(i, j, k)] = v;
}

// beta = value on every element of the level.
__global__ void k_fill_beta(Grid g, double value, double* __restrict__ beta)
{
    COUNT_LAUNCH();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    beta[g.off(i, j, k)] = value;
}

inline int blocks(int64_t n) { return (int)((n + TPB - 1) / TPB); }

}  // namespace

int64_t sep_factor_len(const Grid& g, int terms) { return (int64_t)terms * sum_nodes(g); }

void sep_load_finest(const Grid& g, int terms, const double* samples, double* H, double* b, cudaStream_t s)
{
    k_sep_hat<<<blocks(sep_factor_len(g, terms)), TPB, 0, s>>>(g, terms, samples, H);
    k_sep_outer<<<dim3((g.nx + TX) / TX, (g.ny + TY) / TY, g.nz + 1), dim3(TX, TY), 0, s>>>(g, terms, H, b);
}

void sep_coarsen(const Grid& gc, const Grid& gf, int terms, const double* Ff, double* Fc, bool restrict_,
                 double* out, cudaStream_t s)
{
    k_sep_coarsen<<<blocks(sep_factor_len(gc, terms)), TPB, 0, s>>>(gc, gf, terms, Ff, Fc, restrict_ ? 1 : 0);
    k_sep_outer<<<dim3((gc.nx + TX) / TX, (gc.ny + TY) / TY, gc.nz + 1), dim3(TX, TY), 0, s>>>(gc, terms, Fc, out);
}

void sep_nodal(const Grid& g, int terms, const double* F, double* out, cudaStream_t s)
{
    k_sep_outer<<<dim3((g.nx + TX) / TX, (g.ny + TY) / TY, g.nz + 1), dim3(TX, TY), 0, s>>>(g, terms, F, out);
}

void fill_beta(const Grid& g, double value, double* beta, cudaStream_t s)
{
    k_fill_beta<<<dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.nz), dim3(TX, TY), 0, s>>>(g, value, beta);
}

unsigned long long launches_separable()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
