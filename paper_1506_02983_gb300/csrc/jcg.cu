// jcg.cu -- Jacobi-preconditioned CG of Alg. 4 (lines 7-9) on the matrix-free Q1 operator.
//
// One JCG iteration is two kernels:
//   K1 (k_pq):     p = D^-1 r + beta p_old, computed on the fly for a tile plus halo in shared
//                  memory; q = A p (27-point stencil, difference form); the iterate update
//                  x += alpha_prev p_old deferred from the previous iteration; p.q.
//   K2 (k_update): r -= alpha q; z = D^-1 r; r.z and r.r.
// The last block to finish each reducing kernel sums the per-block partials in a fixed order
// (deterministic) and advances the scalar recurrence in SolveState: alpha after K1, the
// stopping test of Alg. 4 line 7 and beta after K2. Inside a CUDA graph it also sets the
// condition of the level's WHILE node, so a level runs with no host round trip.
//
// The operator at a node is q1_apply (stencil_core.cuh).
#include "fixed.cuh"
#include "jcg.cuh"
#include "jcg_core.cuh"
#include "march.cuh"
#include "march_fx.cuh"
#include "stencil_core.cuh"

#include <cmath>
#include <type_traits>

namespace ecmg {
namespace {

using namespace fx;

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int NT = mt::NT;
constexpr int KZ_TARGET = 64;
constexpr int UPD_TPB = 256;
constexpr int UPD_MAX_BLOCKS = 152 * 8;

// ---- block / grid reductions --------------------------------------------------------------
template <int NP>
__device__ __forceinline__ void block_sum(double (&v)[NP], double* sh)
{
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
    for (int c = 0; c < NP; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    if (lane == 0)
        for (int c = 0; c < NP; ++c) sh[c * 32 + warp] = v[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NP; ++c) {
            v[c] = (lane < nw) ? sh[c * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        }
    }
    __syncthreads();
}

// Sum v over the whole grid. Returns true in the last block to arrive, whose thread 0 then
// holds the totals in v; every other block returns false.
template <int NP>
__device__ __forceinline__ bool grid_sum(double (&v)[NP], double* partials, unsigned int* arrive)
{
    __shared__ double sh[NP * 32];
    __shared__ unsigned int ticket;
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_sum<NP>(v, sh);
    if (tid == 0) {
        for (int c = 0; c < NP; ++c) partials[bid * NP + c] = v[c];
        __threadfence();
        ticket = atomicAdd(arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return false;
    __threadfence();
    for (int c = 0; c < NP; ++c) v[c] = 0.0;
    for (int b = tid; b < nb; b += nthr)
        for (int c = 0; c < NP; ++c) v[c] += __ldcg(&partials[b * NP + c]);
    block_sum<NP>(v, sh);
    if (tid == 0) *arrive = 0u;
    return tid == 0;
}

// Sum compensated FP32 pairs over a grid of 256-thread blocks in FP32 arithmetic: each block
// merges its threads' pairs (block_merge) into partials (a float2 per double slot), the last
// block to arrive merges the blocks' pairs the same way, and each total is widened to FP64 once.
// Returns true in thread 0 of the last block, which then holds the totals in out. bid and nb: the
// block's index in the grid and the grid's size (the caller's layout, 1D or 3D).
template <int NP>
__device__ __forceinline__ bool grid_merge(CSum (&v)[NP], double* partials, unsigned int* arrive,
                                           double (&out)[NP], int bid, int nb)
{
    __shared__ float2 sh[NP * 8], tot[NP];
    __shared__ unsigned int ticket;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    float2* pp = reinterpret_cast<float2*>(partials);
    block_merge<NP>(v, sh, tot);
    if (tid == 0) {
        for (int c = 0; c < NP; ++c) pp[bid * NP + c] = tot[c];
        __threadfence();
        ticket = atomicAdd(arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return false;
    __threadfence();
    for (int c = 0; c < NP; ++c) v[c] = CSum{0.f, 0.f};
    for (int b = tid; b < nb; b += 256)
#pragma unroll
        for (int c = 0; c < NP; ++c) {
            const float2 p = __ldcg(&pp[b * NP + c]);
            twosum_merge(v[c].s, v[c].c, p.x, p.y);
        }
    block_merge<NP>(v, sh, tot);
    if (tid != 0) return false;
    *arrive = 0u;
    for (int c = 0; c < NP; ++c) out[c] = (double)tot[c].x + (double)tot[c].y;
    return true;
}

// ---- the tiled z-march (march.cuh), one tile per block ---------------------------------------
template <bool ROBIN, bool CUBE, typename VT, typename BT, typename SRC, typename BODY>
__device__ __forceinline__ void march(const Grid& g, const Op& op, const BT* __restrict__ beta,
                                      int kz, SRC src, BODY body)
{
    march_tile<ROBIN, CUBE, VT, BT>(g, op, beta, blockIdx.x, blockIdx.y, blockIdx.z, kz, src, body);
}

// ---- the z-march for a level with one beta everywhere (FP64) ------------------------------
// With constant beta the assembled matrix is the tensor product
//     A = beta (Kx(x)My(x)Mz + Mx(x)Ky(x)Mz + Mx(x)My(x)Kz),
// with the assembled 1D matrices K = -(1/h) d2 and M = (h/6) S, d2 = [1 -2 1] and
// S = [1 4 1]. At an interior node therefore
//     (A v)_i = -(beta/36) (hy hz/hx Sy Sz Lx + hx hz/hy Sx Sz Ly + hx hy/hz Sx Sy Lz),
// L_a = d2_a v. The second differences are formed first (neighbouring values nearly cancel
// exactly) and only then smoothed, so the evaluation is as accurate as the difference form
// while costing about 24 FP64 operations per node instead of about 60. Nodes on the box
// boundary (one-sided 1D rows, Robin terms) take the general difference form.
// full_rows: also evaluate Dirichlet rows (callers that mask them pass false).
template <bool ROBIN, bool CUBE, typename SRC, typename BODY>
__device__ __forceinline__ void march_uniform(const Grid& g, const Op& op, double bu, int kz, bool full_rows,
                                              SRC src, BODY body)
{
    __shared__ double X[3][BY + 2][BX + 2];
    __shared__ double LX[BY + 2][BX];
    __shared__ double LY[BY][BX + 2];
    __shared__ double LZ[BY + 2][BX + 2];
    __shared__ double UZ[BY + 2][BX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int kb = blockIdx.z * kz;
    const int ke = min(kb + kz, g.nz + 1);
    const Weights<double> wts(op);
    const double cx = -bu / 36.0 * g.h[1] * g.h[2] / g.h[0];
    const double cy = -bu / 36.0 * g.h[0] * g.h[2] / g.h[1];
    const double cz = -bu / 36.0 * g.h[0] * g.h[1] / g.h[2];

    auto load_plane = [&](int k) {
        double(*dst)[BX + 2] = X[(k + 3) % 3];
        const int64_t base = g.plane_base(k);
        for (int c = tid; c < (BX + 2) * (BY + 2); c += NT) {
            const int ci = c % (BX + 2), cj = c / (BX + 2);
            const int i = i0 - 1 + ci, j = j0 - 1 + cj;
            double v = 0.0;
            if (i <= g.nx + 1 && j <= g.ny + 1) v = src(base + g.in_plane(i, j));
            dst[cj][ci] = v;
        }
    };
    // second differences along x and y of plane k (for the smoothing in y and x)
    auto form_lxy = [&](int k) {
        const double(*P)[BX + 2] = X[(k + 3) % 3];
        for (int c = tid; c < BX * (BY + 2); c += NT) {
            const int ci = c % BX, cj = c / BX;
            LX[cj][ci] = (P[cj][ci] + P[cj][ci + 2]) - 2.0 * P[cj][ci + 1];
        }
        for (int c = tid; c < (BX + 2) * BY; c += NT) {
            const int ci = c % (BX + 2), cj = c / (BX + 2);
            LY[cj][ci] = (P[cj][ci] + P[cj + 2][ci]) - 2.0 * P[cj + 1][ci];
        }
    };
    const int i = i0 + tx, j = j0 + ty;
    double txm = 0, tx0 = 0, tym = 0, ty0 = 0;
    load_plane(kb - 1);
    __syncthreads();
    form_lxy(kb - 1);
    __syncthreads();
    txm = LX[ty][tx] + 4.0 * LX[ty + 1][tx] + LX[ty + 2][tx];
    tym = LY[ty][tx] + 4.0 * LY[ty][tx + 1] + LY[ty][tx + 2];
    load_plane(kb);
    __syncthreads();
    form_lxy(kb);
    __syncthreads();
    tx0 = LX[ty][tx] + 4.0 * LX[ty + 1][tx] + LX[ty + 2][tx];
    ty0 = LY[ty][tx] + 4.0 * LY[ty][tx + 1] + LY[ty][tx + 2];
    for (int k = kb; k < ke; ++k) {
        load_plane(k + 1);
        __syncthreads();
        form_lxy(k + 1);
        {
            const double(*Pm)[BX + 2] = X[(k + 2) % 3];
            const double(*P0)[BX + 2] = X[k % 3];
            const double(*Pp)[BX + 2] = X[(k + 1) % 3];
            for (int c = tid; c < (BX + 2) * (BY + 2); c += NT) {
                const int ci = c % (BX + 2), cj = c / (BX + 2);
                LZ[cj][ci] = (Pm[cj][ci] + Pp[cj][ci]) - 2.0 * P0[cj][ci];
            }
        }
        __syncthreads();
        const double txp = LX[ty][tx] + 4.0 * LX[ty + 1][tx] + LX[ty + 2][tx];
        const double typ = LY[ty][tx] + 4.0 * LY[ty][tx + 1] + LY[ty][tx + 2];
        for (int c = tid; c < BX * (BY + 2); c += NT) {
            const int ci = c % BX, cj = c / BX;
            UZ[cj][ci] = LZ[cj][ci] + 4.0 * LZ[cj][ci + 1] + LZ[cj][ci + 2];
        }
        __syncthreads();
        if (i <= g.nx && j <= g.ny) {
            const int pm = (k + 2) % 3, p0 = k % 3, pp = (k + 1) % 3;
            auto V = [&](int dx, int dy, int dz) -> double {
                return X[dz < 0 ? pm : (dz > 0 ? pp : p0)][ty + 1 + dy][tx + 1 + dx];
            };
            double Av;
            if (i > 0 && i < g.nx && j > 0 && j < g.ny && k > 0 && k < g.nz) {
                const double A = txm + 4.0 * tx0 + txp;
                const double B = tym + 4.0 * ty0 + typ;
                const double C = UZ[ty][tx] + 4.0 * UZ[ty + 1][tx] + UZ[ty + 2][tx];
                Av = cx * A + cy * B + cz * C;
            } else if (!full_rows && on_dirichlet(g, op, i, j, k)) {
                Av = 0.0;  // row discarded by the caller
            } else {
                // one-sided rows: general form with the elements that exist
                auto be = [&](int ex, int ey, int ez) {
                    const int a = i - 1 + ex, b = j - 1 + ey, c = k - 1 + ez;
                    return (a >= 0 && a < g.nx && b >= 0 && b < g.ny && c >= 0 && c < g.nz) ? bu : 0.0;
                };
                Av = q1_apply<true, ROBIN, CUBE, double>(V, be(0, 0, 0), be(1, 0, 0), be(0, 1, 0), be(1, 1, 0),
                                                         be(0, 0, 1), be(1, 0, 1), be(0, 1, 1), be(1, 1, 1), i, j, k,
                                                         g, op, wts);
            }
            body(i, j, k, g.plane_base(k) + g.in_plane(i, j), Av, V(0, 0, 0));
        }
        __syncthreads();  // the boundary rows above read plane k-1, which the next load replaces
        txm = tx0;
        tx0 = txp;
        tym = ty0;
        ty0 = typ;
    }
}


// ---- exact operator for a level with one beta everywhere ------------------------------------
// With one beta the assembled matrix of the whole box, boundary rows included, is the tensor
// product beta (Kx(x)My(x)Mz + Mx(x)Ky(x)Mz + Mx(x)My(x)Kz) of the assembled 1D matrices
// K = -(1/h) D and M = (h/6) S: at interior nodes D = [1 -2 1] and S = [1 4 1], and at the two
// end nodes each row loses its outer entry, D = [-1 1] and S = [2 1]. A Robin face F adds
// alpha_F (h_a h_b / 36) S_a(x)S_b on its nodes (a, b the in-face axes). All these factors have
// integer entries, so with the iterate in fixed point, x = X 2^-s with 64-bit integers X, the
// parts
//     I_x = Sy Sz Dx X,   I_y = Sx Sz Dy X,   I_z = Sx Sy Dz X,   I_F = S_a S_b X
// are exact integer sums (second differences first, then the [1 4 1] smoothing), and
//     A x = 2^-s ( -(beta/36) (hy hz/hx I_x + hx hz/hy I_y + hx hy/hz I_z)
//                  + sum_F alpha_F (h_a h_b/36) I_F )
// takes a few FP64 operations per node instead of about 30 -- FP64 runs at 1/64 of the FP32
// rate on GB300, integer adds at full rate. The scale puts max |x| just below 2^53, so every
// |I| <= 3 * 144 * 2^53 < 2^63, and writing x in fixed point moves each value by less than
// 2^-53 max |x|, below the rounding error of evaluating the difference form in FP64.

// c v with c = 4 (interior node) or 2 (end node): the centre entry of S
__device__ __forceinline__ long long s_mid(long long v, bool end)
{
    return (long long)((unsigned long long)v << (end ? 1 : 2));
}
// c v with c = 2 (interior) or 1 (end): the centre entry of -D
__device__ __forceinline__ long long d_mid(long long v, bool end) { return end ? v : v + v; }

// INT_OUT (cubic elements, no Robin face): body receives the exact integer sum I = I_x + I_y +
// I_z instead of A x, so that A x = -(beta h / 36) 2^-s I.
// Shared memory of march_fixed, declared once per kernel (a kernel may call the march with two
// bodies).
struct FixedSmem {
    long long X[3][BY + 2][BX + 2];
    long long LX[BY + 2][BX];
    long long LY[BY][BX + 2];
    long long LZ[BY + 2][BX + 2];
    long long UZ[BY + 2][BX];
};

template <bool ROBIN, typename SRC, typename BODY, bool INT_OUT = false>
__device__ __forceinline__ void march_fixed(FixedSmem& sm, const Grid& g, const Op& op, double bu, const FixedFrame& fr,
                                            int kz, SRC src, BODY body)
{
    auto& X = sm.X;
    auto& LX = sm.LX;
    auto& LY = sm.LY;
    auto& LZ = sm.LZ;
    auto& UZ = sm.UZ;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int kb = blockIdx.z * kz;
    const int ke = min(kb + kz, g.nz + 1);
    const double cx = -bu / 36.0 * g.h[1] * g.h[2] / g.h[0] * fr.inv;
    const double cy = -bu / 36.0 * g.h[0] * g.h[2] / g.h[1] * fr.inv;
    const double cz = -bu / 36.0 * g.h[0] * g.h[1] / g.h[2] * fr.inv;
    double af[6];  // Robin face coefficients, times 2^-s
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int an = f / 2, a = an == 0 ? 1 : 0, b = an == 2 ? 1 : 2;
        af[f] = ROBIN ? op.alpha[f] * g.h[a] * g.h[b] / 36.0 * fr.inv : 0.0;
    }

    auto load_plane = [&](int k) {
        long long(*dst)[BX + 2] = X[(k + 3) % 3];
        const int64_t base = g.plane_base(k);
        const bool kin = k >= 0 && k <= g.nz;
        for (int c = tid; c < (BX + 2) * (BY + 2); c += NT) {
            const int ci = c % (BX + 2), cj = c / (BX + 2);
            const int i = i0 - 1 + ci, j = j0 - 1 + cj;
            long long v = 0;
            if (kin && i >= 0 && i <= g.nx && j >= 0 && j <= g.ny) v = to_fixed(src(base + g.in_plane(i, j)), fr.s);
            dst[cj][ci] = v;
        }
    };
    // Dx and Dy of plane k: LX at nodes (i0+ci, j0-1+cj), LY at nodes (i0-1+ci, j0+cj)
    auto form_lxy = [&](int k) {
        const long long(*P)[BX + 2] = X[(k + 3) % 3];
        for (int c = tid; c < BX * (BY + 2); c += NT) {
            const int ci = c % BX, cj = c / BX;
            const int i = i0 + ci;
            LX[cj][ci] = (P[cj][ci] + P[cj][ci + 2]) - d_mid(P[cj][ci + 1], i == 0 || i == g.nx);
        }
        for (int c = tid; c < (BX + 2) * BY; c += NT) {
            const int ci = c % (BX + 2), cj = c / (BX + 2);
            const int j = j0 + cj;
            LY[cj][ci] = (P[cj][ci] + P[cj + 2][ci]) - d_mid(P[cj + 1][ci], j == 0 || j == g.ny);
        }
    };
    const int i = i0 + tx, j = j0 + ty;
    const bool iend = i == 0 || i == g.nx, jend = j == 0 || j == g.ny;
    auto sy_lx = [&]() { return LX[ty][tx] + s_mid(LX[ty + 1][tx], jend) + LX[ty + 2][tx]; };
    auto sx_ly = [&]() { return LY[ty][tx] + s_mid(LY[ty][tx + 1], iend) + LY[ty][tx + 2]; };
    long long txm, tx0, tym, ty0;
    load_plane(kb - 1);
    __syncthreads();
    form_lxy(kb - 1);
    __syncthreads();
    txm = sy_lx();
    tym = sx_ly();
    load_plane(kb);
    __syncthreads();
    form_lxy(kb);
    __syncthreads();
    tx0 = sy_lx();
    ty0 = sx_ly();
    for (int k = kb; k < ke; ++k) {
        const bool kend = k == 0 || k == g.nz;
        load_plane(k + 1);
        __syncthreads();
        form_lxy(k + 1);
        {
            const long long(*Pm)[BX + 2] = X[(k + 2) % 3];
            const long long(*P0)[BX + 2] = X[k % 3];
            const long long(*Pp)[BX + 2] = X[(k + 1) % 3];
            for (int c = tid; c < (BX + 2) * (BY + 2); c += NT) {
                const int ci = c % (BX + 2), cj = c / (BX + 2);
                LZ[cj][ci] = (Pm[cj][ci] + Pp[cj][ci]) - d_mid(P0[cj][ci], kend);
            }
        }
        __syncthreads();
        const long long txp = sy_lx();
        const long long typ = sx_ly();
        for (int c = tid; c < BX * (BY + 2); c += NT) {
            const int ci = c % BX, cj = c / BX;
            const int ii = i0 + ci;
            UZ[cj][ci] = LZ[cj][ci] + s_mid(LZ[cj][ci + 1], ii == 0 || ii == g.nx) + LZ[cj][ci + 2];
        }
        __syncthreads();
        if (i <= g.nx && j <= g.ny) {
            const long long Ix = txm + s_mid(tx0, kend) + txp;
            const long long Iy = tym + s_mid(ty0, kend) + typ;
            const long long Iz = UZ[ty][tx] + s_mid(UZ[ty + 1][tx], jend) + UZ[ty + 2][tx];
            if constexpr (INT_OUT) {
                body(i, j, k, g.plane_base(k) + g.in_plane(i, j), Ix + Iy + Iz);
            } else {
                double Av = cx * (double)Ix + cy * (double)Iy + cz * (double)Iz;
                if (ROBIN && (iend || jend || kend)) {
                    const int pm = (k + 2) % 3, p0 = k % 3, pp = (k + 1) % 3;
                    // S_y S_z X on the node's column (x faces)
                    auto fx = [&](int p) { return X[p][ty][tx + 1] + s_mid(X[p][ty + 1][tx + 1], jend) + X[p][ty + 2][tx + 1]; };
                    // S_x S_z X on the node's row (y faces)
                    auto fy = [&](int p) { return X[p][ty + 1][tx] + s_mid(X[p][ty + 1][tx + 1], iend) + X[p][ty + 1][tx + 2]; };
                    // S_x on row r of the node's plane (z faces)
                    auto fz = [&](int r) { return X[p0][ty + r][tx] + s_mid(X[p0][ty + r][tx + 1], iend) + X[p0][ty + r][tx + 2]; };
                    if (iend) {
                        const long long I = fx(pm) + s_mid(fx(p0), kend) + fx(pp);
                        if (i == 0) Av += af[0] * (double)I;
                        if (i == g.nx) Av += af[1] * (double)I;
                    }
                    if (jend) {
                        const long long I = fy(pm) + s_mid(fy(p0), kend) + fy(pp);
                        if (j == 0) Av += af[2] * (double)I;
                        if (j == g.ny) Av += af[3] * (double)I;
                    }
                    if (kend) {
                        const long long I = fz(0) + s_mid(fz(1), jend) + fz(2);
                        if (k == 0) Av += af[4] * (double)I;
                        if (k == g.nz) Av += af[5] * (double)I;
                    }
                }
                body(i, j, k, g.plane_base(k) + g.in_plane(i, j), Av, 0.0);
            }
        }
        __syncthreads();  // the Robin rows above read plane k-1, which the next load replaces
        txm = tx0;
        tx0 = txp;
        tym = ty0;
        ty0 = typ;
    }
}

// max |x| over a level vector into fs->bits (bit patterns of nonnegative doubles order like the
// values; any Inf or NaN gives exponent 0x7ff). Skipped when no fixed-point operator follows
// (more than one beta, and not `always`), or when a residual replacement is not going to run.
__global__ void __launch_bounds__(UPD_TPB) k_absmax(int64_t n, const double* __restrict__ x, const int* uniform,
                                                   int always, const SolveState* st, int mode, FixedScale* fs,
                                                   unsigned long long* partials)
{
    COUNT_LAUNCH();
    if (!always && !*uniform) return;
    if (st && mode == RES_REPLACE && st->done) return;
    __shared__ unsigned long long sh[UPD_TPB / 32];
    __shared__ unsigned int ticket;
    unsigned long long m = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n / 2; t += stride) {
        const double2 v = x2[t];
        m = max(m, fx::abs_bits(v.x));
        m = max(m, fx::abs_bits(v.y));
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
        m = max(m, fx::abs_bits(x[n - 1]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < UPD_TPB / 32; ++w) m = max(m, sh[w]);
        partials[blockIdx.x] = m;
        __threadfence();
        ticket = atomicAdd(&fs->arrive, 1u);
    }
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    m = 0ull;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = max(m, __ldcg(&partials[b]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) sh[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < UPD_TPB / 32; ++w) m = max(m, sh[w]);
        fs->bits = m;
        fs->arrive = 0u;
    }
}

// Constant coefficient (one beta, every face Dirichlet, cubic elements; the first set by the
// set-up's device flag): A x = c 2^-s I with c = -beta h / 36 and I the exact integer sum of
// march_fixed, so with B = b / c on the same fixed-point scale the residual is c 2^-s (B - I),
// exact in 64-bit integers. ||f_h|| (k_fh2), which reads b anyway, stores bc = b / c with this
// reciprocal on the free nodes and takes max |bc| for the scale.
__device__ __forceinline__ double inv_c_of(const double* __restrict__ beta, const Grid& g)
{
    return -36.0 / (beta[g.off(0, 0, 0)] * g.h[0]);
}

// Uniform-beta dispatch of the FP64 kernels: *uniform is set per level by the set-up.
#define ECMG_FP64_MARCH(T, ROBIN, CUBE, FULL, SRC, BODY)                                    \
    do {                                                                                  \
        if (sizeof(T) == 8 && uniform && *uniform)                                        \
            march_uniform<ROBIN, CUBE>(g, op, (double)beta[g.off(0, 0, 0)], kz, FULL, SRC, BODY); \
        else                                                                              \
            march<ROBIN, CUBE, T, T>(g, op, beta, kz, SRC, BODY);                          \
    } while (0)

// ---- K1: search direction and operator ------------------------------------------------------
template <typename T, bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(NT) k_pq(const Grid g, const Op op, const T* __restrict__ beta,
                                           const int* uniform, const T* __restrict__ r,
                                           const T* __restrict__ dinv, const T* __restrict__ pold,
                                           T* __restrict__ pnew, T* __restrict__ q, T* __restrict__ x,
                                           SolveState* st, double* partials, int pidx, CondHandles ch, int kz)
{
    COUNT_LAUNCH();
    if (st->done) return;
    const T bcg = (T)st->beta;
    const T ap = (T)st->alpha_prev;
    Acc<T> acc;
    const PSource<T> src{dinv, r, pold, bcg};
    auto body = [&](int i, int j, int k, int64_t o, T Av, T pn) {
        const T qv = on_dirichlet(g, op, i, j, k) ? T(0) : Av;
        pnew[o] = pn;
        q[o] = qv;
        if (ap != T(0)) x[o] += ap * pold[o];
        acc.add_prod(pn, qv);
    };
    if constexpr (sizeof(T) == 8) ECMG_FP64_MARCH(T, ROBIN, CUBE, false, src, body);
    else march<ROBIN, CUBE, T, T>(g, op, beta, kz, src, body);
    double v[1] = {acc.value()};
    if (grid_sum<1>(v, partials, &st->arrive)) pq_epilogue(st, v[0], pidx, ch);
}

// ---- residual r = b - A x --------------------------------------------------------------------
// bc: b / c of the constant-coefficient case (from k_fh2), or null when the level can not be
// one (a Robin face, non-cubic elements, FP64 output): then A x in FP64 or fixed point as below.
template <typename OT, bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(NT) k_res(const Grid g, const Op op, const double* __restrict__ beta,
                                            const int* uniform, const double* __restrict__ x,
                                            const double* __restrict__ b, const OT* __restrict__ dinv,
                                            OT* __restrict__ r, SolveState* st, double* partials, int mode,
                                            CondHandles ch, int kz, const FixedScale* fs,
                                            const double* __restrict__ bc)
{
    COUNT_LAUNCH();
    __shared__ FixedSmem fsm;
    if (mode == RES_REPLACE && st->done) return;
    if constexpr (std::is_same<OT, float>::value && CUBE && !ROBIN) {
        if (bc && *uniform) {
            // constant coefficient: r = c 2^-s (B - I) exactly, then rounded to FP32 once;
            // ||r||^2 by compensated FP32 products, r.z = D^-1 r.r (one diagonal)
            const FixedFrame fr = fixed_frame(max(fs->bits, st->bcbits));
            const float fscale = (float)(-beta[g.off(0, 0, 0)] * g.h[0] / 36.0 * fr.inv);
            Acc<float> rr32;
            auto src = [&](int64_t o) -> double { return x[o]; };
            auto body = [&](int i, int j, int k, int64_t o, long long I) {
                float ro = 0.f;
                if (!on_dirichlet(g, op, i, j, k)) ro = __ll2float_rn(to_fixed(bc[o], fr.s) - I) * fscale;
                r[o] = ro;
                rr32.add_prod(ro, ro);
            };
            CSum pr[1] = {CSum{0.f, 0.f}};
            if (fr.finite) {
                march_fixed<false, decltype(src), decltype(body), true>(fsm, g, op, beta[g.off(0, 0, 0)], fr, kz,
                                                                        src, body);
                pr[0] = rr32.v;
            } else if (threadIdx.x == 0 && threadIdx.y == 0) {
                pr[0].s = __int_as_float(0x7fc00000);  // NaN: breakdown, the iterate is not finite
            }
            double v[1];
            const int nb = gridDim.x * gridDim.y * gridDim.z;
            const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            if (grid_merge<1>(pr, partials, &st->arrive, v, bid, nb))
                res_epilogue(st, v[0], (double)dinv[g.off(1, 1, 1)] * v[0], mode, ch);
            return;
        }
    }
    double rr = 0.0;
    Acc<OT> rz;  // r.z in the precision of the iteration that uses it (z = D^-1 r rounded)
    auto src = [&](int64_t o) -> double { return x[o]; };
    auto body = [&](int i, int j, int k, int64_t o, double Av, double) {
        const double rv = on_dirichlet(g, op, i, j, k) ? 0.0 : b[o] - Av;
        const OT ro = (OT)rv;
        r[o] = ro;
        rr = fma(rv, rv, rr);
        rz.add_prod(ro, dinv[o] * ro);
    };
    if (*uniform || CUBE) {
        const FixedFrame fr = fixed_frame(fs->bits);
        if (!fr.finite) {
            if (threadIdx.x == 0 && threadIdx.y == 0) rr = nan("");  // breakdown: the iterate is not finite
        } else if (*uniform) {
            march_fixed<ROBIN>(fsm, g, op, beta[g.off(0, 0, 0)], fr, kz, src, body);
        } else if constexpr (CUBE) {
            // variable beta on cubic elements: integer element sums (march_fx.cuh)
            auto body5 = [&](int i, int j, int k, int64_t o, double Av) { body(i, j, k, o, Av, 0.0); };
            march_range_fxv<ROBIN>(g, beta, x, all_nodes(g), blockIdx.x, blockIdx.y, blockIdx.z, kz, fr, op, body5);
        }
    } else {
        march<ROBIN, CUBE, double, double>(g, op, beta, kz, src, body);
    }
    double v[2] = {rr, rz.value()};
    if (grid_sum<2>(v, partials, &st->arrive)) res_epilogue(st, v[0], v[1], mode, ch);
}

// ---- ||f_h||: the free-node right-hand side with the Dirichlet values moved over (fh_at) -------
// The free nodes form a box F; the nodes of F one step from a Dirichlet face (the shell) carry
// the lift b - A g_ext, all others just b. The shell is summed by its own flat loops, one node
// per thread, so its FP64 stencil never runs in a warp whose other lanes idle (a warp that
// diverges on the FP64 pipe pays for all 32 lanes); the inner box N streams b alone.
struct FhBox {
    int lo[3], hi[3];    // F: free nodes per axis
    int nlo[3], nhi[3];  // N: no Dirichlet face within one step (nlo > nhi: empty)
};
// values of axis a in F but not in N: count, and the idx-th of them
__device__ __forceinline__ int outer_count(const FhBox& B, int a)
{
    return B.nlo[a] > B.nhi[a] ? B.hi[a] - B.lo[a] + 1 : (B.nlo[a] - B.lo[a]) + (B.hi[a] - B.nhi[a]);
}
__device__ __forceinline__ int outer_value(const FhBox& B, int a, int idx)
{
    if (B.nlo[a] > B.nhi[a]) return B.lo[a] + idx;
    const int nl = B.nlo[a] - B.lo[a];
    return idx < nl ? B.lo[a] + idx : B.nhi[a] + 1 + (idx - nl);
}
__device__ __forceinline__ int inner_count(const FhBox& B, int a) { return max(B.nhi[a] - B.nlo[a] + 1, 0); }

// bc: on a MIXED level that may be a constant-coefficient one, the vector that receives b / c;
// with the level's uniform flag set the kernel stores it on the free nodes (the only ones the
// residual reads) and takes max |b / c| into st->bcbits (the exact residual's scale).
template <bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(UPD_TPB) k_fh2(const Grid g, const Op op, const FhBox B,
                                                 const double* __restrict__ beta, const double* __restrict__ x,
                                                 const double* __restrict__ b, SolveState* st, double* partials,
                                                 const int* __restrict__ uniform, double* __restrict__ bc)
{
    COUNT_LAUNCH();
    const Weights<double> wts(op);
    double ss = 0.0;
    // max |b / c| as integer bits (the order of non-negative doubles, NaN above +inf)
    const bool bmax = bc && *uniform;
    const double inv_c = bmax ? inv_c_of(beta, g) : 0.0;
    unsigned long long mb = 0ull;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nFi = B.hi[0] - B.lo[0] + 1, nFj = B.hi[1] - B.lo[1] + 1;
    const int oi = outer_count(B, 0), oj = outer_count(B, 1), ok = outer_count(B, 2);
    const int ii = inner_count(B, 0), ij = inner_count(B, 1), ik = inner_count(B, 2);
    auto shell = [&](int i, int j, int k) {
        const int64_t o = g.off(i, j, k);
        const double f = fh_at<ROBIN, CUBE>(g, op, wts, beta, x, b, o, i, j, k);
        ss = fma(f, f, ss);
        if (bmax) {
            const double v = b[o] * inv_c;
            bc[o] = v;
            mb = max(mb, fx::abs_bits(v));
        }
    };
    // shell 1: planes k of F outside N, every (i, j) of F
    const int64_t n1 = (int64_t)ok * nFj * nFi;
    for (int64_t t = tid; t < n1; t += nthreads) {
        const int i = B.lo[0] + (int)(t % nFi), j = B.lo[1] + (int)((t / nFi) % nFj);
        shell(i, j, outer_value(B, 2, (int)(t / ((int64_t)nFi * nFj))));
    }
    // shell 2: planes of N, rows j of F outside N, every i of F
    const int64_t n2 = (int64_t)ik * oj * nFi;
    for (int64_t t = tid; t < n2; t += nthreads) {
        const int i = B.lo[0] + (int)(t % nFi), j = outer_value(B, 1, (int)((t / nFi) % oj));
        shell(i, j, B.nlo[2] + (int)(t / ((int64_t)nFi * oj)));
    }
    // shell 3: rows of N, nodes i of F outside N
    const int64_t n3 = (int64_t)ik * ij * oi;
    for (int64_t t = tid; t < n3; t += nthreads) {
        const int i = outer_value(B, 0, (int)(t % oi)), j = B.nlo[1] + (int)((t / oi) % ij);
        shell(i, j, B.nlo[2] + (int)(t / ((int64_t)oi * ij)));
    }
    // inner box: rows (j, k) over the warps of the grid, nodes i over the lanes
    const int64_t nrows = (int64_t)ij * ik;
    const int64_t warps = nthreads / 32, wid = tid / 32;
    for (int64_t row = wid; row < nrows; row += warps) {
        const int j = B.nlo[1] + (int)(row % ij), k = B.nlo[2] + (int)(row / ij);
        const int64_t orow = g.off(B.nlo[0], j, k);
        const double* brow = b + orow;
        for (int i = threadIdx.x & 31; i < ii; i += 32) {
            const double bv = brow[i];
            ss = fma(bv, bv, ss);
            if (bmax) {
                const double v = bv * inv_c;
                bc[orow + i] = v;
                mb = max(mb, fx::abs_bits(v));
            }
        }
    }
    if (bmax) {
        __shared__ unsigned long long shm[UPD_TPB / 32];
        for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_down_sync(0xffffffffu, mb, o));
        if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mb;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < UPD_TPB / 32; ++w) mb = max(mb, shm[w]);
            atomicMax(&st->bcbits, mb);  // before this block's arrival in grid_sum
        }
    }
    double v[1] = {ss};
    if (grid_sum<1>(v, partials, &st->arrive)) {
        st->fh2 = v[0];
        st->thresh2 = st->rtol2 * v[0];
    }
}

// ---- y = A x (full matrix, for operator checks) ---------------------------------------------
template <typename T, bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(NT) k_apply(const Grid g, const Op op, const T* __restrict__ beta,
                                              const int* uniform, const T* __restrict__ x,
                                              double* __restrict__ y, int kz, const FixedScale* fs)
{
    COUNT_LAUNCH();
    __shared__ FixedSmem fsm;
    auto src = [&](int64_t o) -> T { return x[o]; };
    auto body = [&](int, int, int, int64_t o, T Av, T) { y[o] = (double)Av; };
    if constexpr (sizeof(T) == 8) {
        if (*uniform) {
            const FixedFrame fr = fixed_frame(fs->bits);
            auto body64 = [&](int, int, int, int64_t o, double Av, double) { y[o] = fr.finite ? Av : nan(""); };
            march_fixed<ROBIN>(fsm, g, op, beta[g.off(0, 0, 0)], fr, kz, src, body64);
        } else {
            march<ROBIN, CUBE, T, T>(g, op, beta, kz, src, body);
        }
    } else {
        march<ROBIN, CUBE, T, T>(g, op, beta, kz, src, body);
    }
}

// ---- ring of search directions (MIXED two-pass levels) -----------------------------------------
constexpr int RING_MAX = 64;

// The pending directions of a level's ring in shared memory, oldest first: their slots and their
// steps alpha rounded to FP32 (the rounding the correction vector's e += alpha p applies). Every
// thread of the block calls it; a barrier follows inside.
__device__ __forceinline__ void ring_pending(const SolveState* st, const double* __restrict__ alpha, int R,
                                             int* sslot, float* sa)
{
    const int pend = st->pend, pbase = st->pbase;
    for (int t = threadIdx.x; t < pend; t += blockDim.x) {
        const int slot = (pbase + t) % R;
        sslot[t] = slot;
        sa[t] = (float)alpha[slot];
    }
    __syncthreads();
}

// acc, then acc = fmaf(alpha_u, p_u, acc) over the pending directions u = 0 .. pend-1 at float4
// index t of the ring's slots (stride elements apart): the fused multiply-adds the correction
// vector performs, in its order. Four directions' loads are issued before their sums.
__device__ __forceinline__ float4 ring_chain(float4 acc, const float* __restrict__ ring, int64_t stride,
                                             const int* sslot, const float* sa, int pend, int64_t t)
{
    auto dir = [&](int u) { return __ldcs(reinterpret_cast<const float4*>(ring + (int64_t)sslot[u] * stride) + t); };
    auto step = [&](float a, const float4 pv) {
        acc.x = fmaf(a, pv.x, acc.x);
        acc.y = fmaf(a, pv.y, acc.y);
        acc.z = fmaf(a, pv.z, acc.z);
        acc.w = fmaf(a, pv.w, acc.w);
    };
    int u = 0;
    for (; u + 4 <= pend; u += 4) {
        const float4 p0 = dir(u), p1 = dir(u + 1), p2 = dir(u + 2), p3 = dir(u + 3);
        step(sa[u], p0);
        step(sa[u + 1], p1);
        step(sa[u + 2], p2);
        step(sa[u + 3], p3);
    }
    for (; u < pend; ++u) step(sa[u], dir(u));
    return acc;
}

// ---- K2: residual update and stopping test ----------------------------------------------------
template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };
__device__ __forceinline__ float& vget(float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
__device__ __forceinline__ double& vget(double2& v, int c) { return c == 0 ? v.x : v.y; }

// Flat over the padded vector, 16-byte vectors (the layout keeps total a multiple of 8).
// cdiag: when not null and *uniform is set (one beta, every face Dirichlet), D^-1 is the constant
// *cdiag on every free node (r = 0 on the others), so r.z = cdiag * r.r and D^-1 is not streamed.
// MIXED with a ring of search directions (ring.base not null): when the ring is full (ring_cap
// directions pending after this step's K1), the blocks also add the pending alpha p to the
// correction vector e, oldest first, and the last block empties the ring.
template <typename T, bool MIXED>
__global__ void __launch_bounds__(UPD_TPB) k_update(int64_t n, T* __restrict__ r, const T* __restrict__ q,
                                                    const T* __restrict__ dinv, SolveState* st,
                                                    double* partials, CondHandles ch, const int* uniform,
                                                    const T* cdiag, const RingArgs ring, float* __restrict__ e)
{
    COUNT_LAUNCH();
    if (st->done) {
        if (ch.use && blockIdx.x == 0 && threadIdx.x == 0) {
            cudaGraphSetConditional(ch.loop, 0);
            if (MIXED) cudaGraphSetConditional(ch.update, 0);
        }
        return;
    }
    // a step behind one that asked for a replacement (levels with a ring, whose loop body checks
    // once per several steps): nothing to do, and the conditions stay as that step set them
    if (MIXED && ring.base && st->need_update) return;
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::n;
    const T a = (T)st->alpha;
    Acc<T> rz, rr;
    const int64_t nv = n / W;
    V* __restrict__ rv4 = reinterpret_cast<V*>(r);
    const V* __restrict__ qv4 = reinterpret_cast<const V*>(q);
    const V* __restrict__ dv4 = reinterpret_cast<const V*>(dinv);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool cc = cdiag && *uniform;
    const bool spill = MIXED && ring.base && st->pend >= ring_cap(st->pring);
    if (spill) {
        __shared__ int sslot[RING_MAX];
        __shared__ float sa[RING_MAX];
        ring_pending(st, ring.alpha, ring.R, sslot, sa);
        const int pend = st->pend;
        const bool es = st->espill != 0;
        float4* e4 = reinterpret_cast<float4*>(e);
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n / 4; t += stride)
            e4[t] = ring_chain(es ? e4[t] : make_float4(0.f, 0.f, 0.f, 0.f), ring.base, ring_stride(n), sslot, sa,
                               pend, t);
    }
    if (cc) {
        // one diagonal: r.z = D^-1 r.r, formed from ||r||^2 after the reduction
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += stride) {
            V rr4 = rv4[t];
            const V q4 = qv4[t];
#pragma unroll
            for (int c = 0; c < W; ++c) {
                const T rv = vget(rr4, c) - a * vget(const_cast<V&>(q4), c);
                vget(rr4, c) = rv;
                rr.add_prod(rv, rv);
            }
            rv4[t] = rr4;
        }
    } else {
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += stride) {
            V rr4 = rv4[t];
            const V q4 = qv4[t], d4 = dv4[t];
#pragma unroll
            for (int c = 0; c < W; ++c) {
                const T rv = vget(rr4, c) - a * vget(const_cast<V&>(q4), c);
                vget(rr4, c) = rv;
                const T zv = vget(const_cast<V&>(d4), c) * rv;
                rz.add_prod(rv, zv);
                rr.add_prod(rv, rv);
            }
            rv4[t] = rr4;
        }
    }
    double v[2];
    bool last;
    if constexpr (sizeof(T) == 4) {
        CSum pr[2] = {rz.v, rr.v};  // FP32 data: the pairs merged in FP32 (grid_merge)
        last = grid_merge<2>(pr, partials, &st->arrive, v, (int)blockIdx.x, (int)gridDim.x);
    } else {
        v[0] = rz.value();
        v[1] = rr.value();
        last = grid_sum<2>(v, partials, &st->arrive);
    }
    if (last) {
        if (cc) v[0] = (double)*cdiag * v[1];
        if (spill) {  // every block has read the pending set above
            st->pbase = (st->pj + 1) % st->pring;
            st->pend = 0;
            st->espill = 1;
        }
        update_epilogue<MIXED>(st, v[0], v[1]);
        if (ch.use) {
            cudaGraphSetConditional(ch.loop, st->done ? 0u : 1u);
            if (MIXED) cudaGraphSetConditional(ch.update, st->need_update ? 1u : 0u);
        }
    }
}

__global__ void k_final64(int64_t n, double* __restrict__ x, const double* __restrict__ pA,
                          const double* __restrict__ pB, const SolveState* st)
{
    COUNT_LAUNCH();
    const double a = st->alpha_prev;
    if (a == 0.0) return;
    const double* p = st->p_latest ? pB : pA;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride)
        x[t] = fma(a, p[t], x[t]);
}

// MIXED fold at a residual replacement: x += e + alpha_prev p, e = 0. The FP32 correction is
// combined in FP32 (one more rounding of an FP32 quantity) and added to x with a single FP64
// operation. On a level with one beta the block also takes max |x| of the new iterate into
// fs->bits, the scale of the exact residual that follows (no separate pass over x).
__global__ void __launch_bounds__(UPD_TPB) k_fold32(int64_t n, double* __restrict__ x, float* __restrict__ e,
                                                   const float* __restrict__ pa, const float* __restrict__ pb,
                                                   const int* __restrict__ uniform, const SolveState* st,
                                                   FixedScale* fs, unsigned long long* partials)
{
    COUNT_LAUNCH();
    if (st->done) return;
    const float* __restrict__ p = (pb && st->p_latest) ? pb : pa;  // pb: the newest p of the pair
    const float a = (float)st->alpha_prev;
    const bool want_max = *uniform != 0;
    __shared__ unsigned long long sh[UPD_TPB / 32];
    __shared__ unsigned int ticket;
    unsigned long long m = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double2* x2 = reinterpret_cast<double2*>(x);
    float4* e4 = reinterpret_cast<float4*>(e);
    const float4* p4 = reinterpret_cast<const float4*>(p);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n / 4; t += stride) {
        const float4 ev = e4[t], pv = p4[t];
        double2 xa = x2[2 * t], xb = x2[2 * t + 1];
        xa.x += widen(fmaf(a, pv.x, ev.x));
        xa.y += widen(fmaf(a, pv.y, ev.y));
        xb.x += widen(fmaf(a, pv.z, ev.z));
        xb.y += widen(fmaf(a, pv.w, ev.w));
        x2[2 * t] = xa;
        x2[2 * t + 1] = xb;
        e4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        m = max(m, max(max(fx::abs_bits(xa.x),
                           fx::abs_bits(xa.y)),
                       max(fx::abs_bits(xb.x),
                           fx::abs_bits(xb.y))));
    }
    for (int64_t t = (n / 4) * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride) {
        x[t] += widen(fmaf(a, p[t], e[t]));
        e[t] = 0.f;
        m = max(m, fx::abs_bits(x[t]));
    }
    if (!want_max) return;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < UPD_TPB / 32; ++w) m = max(m, sh[w]);
        partials[blockIdx.x] = m;
        __threadfence();
        ticket = atomicAdd(&fs->arrive, 1u);
    }
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    m = 0ull;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = max(m, __ldcg(&partials[b]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) sh[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < UPD_TPB / 32; ++w) m = max(m, sh[w]);
        fs->bits = m;
        fs->arrive = 0u;
    }
}

__global__ void k_state_init(SolveState* st, double rtol, double inner, int max_iters, int fixed, int pring)
{
    COUNT_LAUNCH();
    SolveState s = {};
    s.rtol2 = rtol * rtol;
    s.inner2 = inner * inner;
    s.max_iters = max_iters;
    s.fixed = fixed;
    s.pring = pring;  // pj = 0: slot 0 holds the zero direction p_{-1}
    *st = s;
}

// MIXED with a ring of search directions: x64 += e + the pending alpha p, formed in FP32 oldest
// first (e only when a full ring was added to it since the last replacement; e is then zeroed):
// the same fused multiply-adds, in the same order, as the correction vector of the form without
// a ring, added with one FP64 operation. With the level's uniform flag set, also max |x| of the
// new iterate into fs (as k_fold32).
__global__ void __launch_bounds__(UPD_TPB) k_fold_ring(int64_t n, double* __restrict__ x, const float* __restrict__ ring,
                                                      const double* __restrict__ alpha, int R, float* __restrict__ e,
                                                      const int* __restrict__ uniform, const SolveState* st,
                                                      FixedScale* fs, unsigned long long* partials)
{
    COUNT_LAUNCH();
    if (st->done) return;
    __shared__ float sa[RING_MAX];
    __shared__ int sslot[RING_MAX];
    __shared__ unsigned long long sh[UPD_TPB / 32];
    __shared__ unsigned int ticket;
    ring_pending(st, alpha, R, sslot, sa);
    const int pend = st->pend;
    const bool es = st->espill != 0;
    const bool want_max = *uniform != 0;
    unsigned long long m = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double2* x2 = reinterpret_cast<double2*>(x);
    float4* e4 = reinterpret_cast<float4*>(e);
    // n, a level's stored length, is a multiple of 8 (rows are padded to 8 elements): no tail
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n / 4; t += stride) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (es) {
            acc = e4[t];
            e4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        acc = ring_chain(acc, ring, ring_stride(n), sslot, sa, pend, t);
        double2 xa = x2[2 * t], xb = x2[2 * t + 1];
        xa.x += widen(acc.x);
        xa.y += widen(acc.y);
        xb.x += widen(acc.z);
        xb.y += widen(acc.w);
        x2[2 * t] = xa;
        x2[2 * t + 1] = xb;
        m = max(m, max(max(fx::abs_bits(xa.x), fx::abs_bits(xa.y)), max(fx::abs_bits(xb.x), fx::abs_bits(xb.y))));
    }
    if (!want_max) return;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < UPD_TPB / 32; ++w) m = max(m, sh[w]);
        partials[blockIdx.x] = m;
        __threadfence();
        ticket = atomicAdd(&fs->arrive, 1u);
    }
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    m = 0ull;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = max(m, __ldcg(&partials[b]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) sh[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < UPD_TPB / 32; ++w) m = max(m, sh[w]);
        fs->bits = m;
        fs->arrive = 0u;
    }
}

inline bool has_robin(const Op& op)
{
    for (int f = 0; f < 6; ++f)
        if (op.alpha[f] != 0.0) return true;
    return false;
}

inline int stencil_kz(const Grid& g)
{
    const int gx = (g.nx + 1 + BX - 1) / BX, gy = (g.ny + 1 + BY - 1) / BY;
    const int want_blocks = 152 * 4;
    int gz = (want_blocks + gx * gy - 1) / (gx * gy);
    int kz = (g.nz + 1 + gz - 1) / gz;
    // small levels (the direct solves, the first MIXED levels) are FP64-pipe and latency bound:
    // spread them over more SMs with short columns, down to one plane per block
    if (kz < 1) kz = 1;
    if (kz > KZ_TARGET) kz = KZ_TARGET;
    return kz;
}

inline dim3 stencil_grid(const Grid& g, int kz)
{
    return dim3((g.nx + 1 + BX - 1) / BX, (g.ny + 1 + BY - 1) / BY, (g.nz + 1 + kz - 1) / kz);
}

inline int update_blocks(int64_t n)
{
    int64_t b = (n + UPD_TPB * 4 - 1) / (UPD_TPB * 4);
    return (int)(b < UPD_MAX_BLOCKS ? (b > 0 ? b : 1) : UPD_MAX_BLOCKS);
}

}  // namespace

int max_stencil_blocks(const Grid& g)
{
    dim3 d = stencil_grid(g, stencil_kz(g));
    return (int)(d.x * d.y * d.z);
}
int max_stream_blocks() { return UPD_MAX_BLOCKS; }

// Kernel variant for the level: Robin terms present, cubic elements.
#define ECMG_VARIANT(KERNEL, ...)                                                              \
    (has_robin(op) ? (op.cube ? KERNEL<__VA_ARGS__, true, true> : KERNEL<__VA_ARGS__, true, false>) \
                   : (op.cube ? KERNEL<__VA_ARGS__, false, true> : KERNEL<__VA_ARGS__, false, false>))

void launch_pq64(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* r,
                 const double* dinv, const double* pold, double* pnew, double* q, double* x,
                 SolveState* st, Partials pr, int pidx, CondHandles ch, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    ECMG_VARIANT(k_pq, double)<<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, uniform, r, dinv, pold,
                                                                           pnew, q, x, st, pr.buf, pidx, ch, kz);
}
// max |x| for the fixed-point evaluation (a no-op on levels with more than one beta)
void launch_absmax(const Grid& g, const double* x, const int* uniform, const SolveState* st, int mode,
                   Partials pr, cudaStream_t s, bool always)
{
    k_absmax<<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, x, uniform, always ? 1 : 0, st, mode, pr.fs,
                                                        reinterpret_cast<unsigned long long*>(pr.buf));
}
void launch_res64(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* x,
                  const double* b, const double* dinv, double* r, SolveState* st, Partials pr, ResMode mode,
                  CondHandles ch, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    launch_absmax(g, x, uniform, st, (int)mode, pr, s, op.cube != 0);
    ECMG_VARIANT(k_res, double)<<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, uniform, x, b, dinv, r,
                                                                            st, pr.buf, (int)mode, ch, kz, pr.fs,
                                                                            nullptr);
}
bool constant_coefficient_shape(const Grid& g, const Op& op)
{
    bool diri = true;
    for (int f = 0; f < 6; ++f) diri &= op.bc[f] == 0;
    return diri && op.cube && g.nx >= 2 && g.ny >= 2 && g.nz >= 2;
}
void launch_res32(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* x,
                  const double* b, const float* dinv, float* r, SolveState* st, Partials pr, ResMode mode,
                  CondHandles ch, cudaStream_t s, const double* bc)
{
    const int kz = stencil_kz(g);
    launch_absmax(g, x, uniform, st, (int)mode, pr, s, op.cube != 0);
    if (!constant_coefficient_shape(g, op)) bc = nullptr;
    ECMG_VARIANT(k_res, float)<<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, uniform, x, b, dinv, r,
                                                                           st, pr.buf, (int)mode, ch, kz, pr.fs,
                                                                           bc);
}
void launch_apply64(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* x,
                    double* y, Partials pr, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    launch_absmax(g, x, uniform, nullptr, 0, pr, s);
    ECMG_VARIANT(k_apply, double)<<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, uniform, x, y, kz,
                                                                              pr.fs);
}
void launch_apply32(const Grid& g, const Op& op, const float* beta, const float* x, double* y, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    ECMG_VARIANT(k_apply, float)<<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, nullptr, x, y, kz,
                                                                             nullptr);
}
void launch_fh2(const Grid& g, const Op& op, const double* beta, const double* x, const double* b, SolveState* st,
                Partials pr, cudaStream_t s, const int* uniform, double* bc, int max_blocks)
{
    FhBox B;
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const bool dlo = op.bc[2 * a] == 0, dhi = op.bc[2 * a + 1] == 0;
        B.lo[a] = dlo ? 1 : 0;
        B.hi[a] = dhi ? n[a] - 1 : n[a];
        B.nlo[a] = dlo ? 2 : 0;           // fh_at: within one step of a Dirichlet face
        B.nhi[a] = dhi ? n[a] - 2 : n[a];
    }
    (has_robin(op) ? (op.cube ? k_fh2<true, true> : k_fh2<true, false>)
                   : (op.cube ? k_fh2<false, true> : k_fh2<false, false>))<<<
        max_blocks > 0 ? std::min(update_blocks(g.total), max_blocks) : update_blocks(g.total), UPD_TPB, 0, s>>>(
        g, op, B, beta, x, b, st, pr.buf, uniform, uniform && constant_coefficient_shape(g, op) ? bc : nullptr);
}
void launch_update64(const Grid& g, double* r, const double* q, const double* dinv, SolveState* st,
                     Partials pr, CondHandles ch, cudaStream_t s)
{
    k_update<double, false><<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, r, q, dinv, st, pr.buf, ch,
                                                                        nullptr, nullptr,
                                                                        RingArgs{nullptr, nullptr, 0}, nullptr);
}
void launch_update32(const Grid& g, const Op& op, const int* uniform, float* r, const float* q, const float* dinv,
                     SolveState* st, Partials pr, CondHandles ch, cudaStream_t s, const RingArgs* ring, float* e)
{
    bool diri = uniform != nullptr;
    for (int f = 0; f < 6; ++f) diri &= op.bc[f] == 0;
    // an interior node: free whenever every face is Dirichlet (levels >= 2 have >= 4 elements per axis)
    const float* cdiag = diri && g.nx >= 2 && g.ny >= 2 && g.nz >= 2 ? dinv + g.off(1, 1, 1) : nullptr;
    const RingArgs rg = ring ? *ring : RingArgs{nullptr, nullptr, 0};
    k_update<float, true><<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, r, q, dinv, st, pr.buf, ch, uniform,
                                                                      cdiag, rg, e);
}
void launch_final64(const Grid& g, double* x, const double* pA, const double* pB, SolveState* st,
                    cudaStream_t s)
{
    k_final64<<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, x, pA, pB, st);
}
void launch_fold32(const Grid& g, double* x, float* e, const float* p, const int* uniform, SolveState* st,
                   Partials pr, cudaStream_t s, const float* p_b)
{
    k_fold32<<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, x, e, p, p_b, uniform, st, pr.fs,
                                                        reinterpret_cast<unsigned long long*>(pr.buf));
}
void launch_state_init(SolveState* st, double rtol, double inner_rtol, int max_iters, int fixed, cudaStream_t s,
                       int pring)
{
    k_state_init<<<1, 1, 0, s>>>(st, rtol, inner_rtol, max_iters, fixed, pring);
}
void launch_fold_ring(const Grid& g, double* x, const RingArgs& ring, float* e, const int* uniform, SolveState* st,
                      Partials pr, cudaStream_t s)
{
    k_fold_ring<<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, x, ring.base, ring.alpha, ring.R, e, uniform, st,
                                                           pr.fs, reinterpret_cast<unsigned long long*>(pr.buf));
}

unsigned long long launches_jcg()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
