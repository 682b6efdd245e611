// march_fx.cuh -- the operator of a level with cubic elements and variable beta in fixed-point
// integers (batch.cu, jcg.cu).
//
// For a cube element of side h the element matrix is beta_e h times the unit-cube matrix:
// 1/3 on the diagonal, 0 between two nodes on an element edge, -1/12 between two nodes on a
// face diagonal or on the body diagonal. Every row sums to zero, so at node i
//     (A x)_i = -(h / 12) sum_e beta_e I_e,   I_e = sum_{j far from i in e} (x_j - x_i),
// the inner sum running over the three face-diagonal nodes and the body-diagonal node of
// element e. With the iterate in fixed point, x = X 2^-s (64-bit X < 2^53, the scale of
// fixed.cuh), each I_e is an exact integer below 2^56. beta is put in fixed point too,
// B_e = beta_e 2^t with t from the largest beta the block reads (B_e < 2^62; a beta more than
// 2^9 below that max loses its bits under 2^-t, far below one rounding of the result), and the
// eight products B_e I_e are summed exactly in 128-bit integers; the sum is rounded to FP64 once.
// The scale only has to be common to the eight elements of one node, so each block takes its
// own from a first pass over the betas it will stage (no level-wide reduction). That leaves
// about five FP64 operations per node for the residual instead of twenty (FP64 runs at 1/64 of
// the FP32 rate on GB300; the 64 x 64 -> 128-bit products run on the integer pipe). Elements
// outside the box carry beta = 0 in the padded layout, so nodes on a Neumann face need no special
// case. A Robin face F adds alpha_F (h^2 / 36) (S (x) S) x on its nodes, S = [1 4 1] ([2 1] at a
// face edge): an exact integer sum of the face neighbours (ghost nodes hold 0) times one FP64
// weight.
#pragma once

#include "fixed.cuh"
#include "march.cuh"

namespace ecmg {

// Signed 128-bit accumulator of 64 x 64-bit products (two's complement in hi:lo).
struct Acc128 {
    long long hi = 0;
    unsigned long long lo = 0ull;
    __device__ __forceinline__ void add_prod(long long a, long long b)
    {
        const unsigned long long pl = (unsigned long long)a * (unsigned long long)b;
        const long long ph = __mul64hi(a, b);
        const unsigned long long nl = lo + pl;
        hi += ph + (nl < lo ? 1ll : 0ll);
        lo = nl;
    }
    // hi 2^64 + lo, rounded to FP64 (about one rounding of the result)
    __device__ __forceinline__ double value() const
    {
        return fma(__ll2double_rn(hi), 18446744073709551616.0, __ull2double_rn(lo));
    }
};

// Fixed-point shift t of beta from the bits of the largest beta in use: max beta 2^t < 2^62.
__device__ __forceinline__ int beta_shift(unsigned long long bits)
{
    const int E = (int)((bits >> 52) & 0x7ff);
    return bits == 0ull ? 0 : 1084 - E;
}

// The z-march of march_range (march.cuh) with the operand staged as fixed-point integers:
// body(i, j, k, offset, A x) for every node of the range. x: the level vector (FP64, padded).
template <bool ROBIN, typename BODY>
__device__ __forceinline__ void march_range_fxv(const Grid& g, const double* __restrict__ beta,
                                                const double* __restrict__ x, const NodeRange& rg, int bx, int by,
                                                int bz, int kz, const fx::FixedFrame& fr, const Op& op, BODY body)
{
    const int op_robin_mask = op.robin_mask;
    const double* rw = op.rw64;
    constexpr int NT = mt::NT;
    constexpr int PC = (BX + 2) * (BY + 2), SC = (BX + 1) * (BY + 1);  // plane and slab cells
    constexpr int NP = (PC + NT - 1) / NT, NS = (SC + NT - 1) / NT;    // cells per thread
    __shared__ long long sv[3][BY + 2][BX + 2];
    __shared__ long long sb[2][BY + 1][BX + 1];  // beta in fixed point, B = beta 2^tb
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int i0 = rg.ilo + bx * BX, j0 = rg.jlo + by * BY;
    const int kb = rg.klo + bz * kz;
    const int ke = min(kb + kz, rg.khi + 1);
    const double cA = -g.h[0] / 12.0 * fr.inv;

    int pofs[NP], sofs[NS];
#pragma unroll
    for (int c = 0; c < NP; ++c) {
        const int cell = tid + c * NT;
        const int i = i0 - 1 + cell % (BX + 2), j = j0 - 1 + cell / (BX + 2);
        pofs[c] = (cell < PC && i <= g.nx + 1 && j <= g.ny + 1) ? g.in_plane(i, j) : -1;
    }
#pragma unroll
    for (int c = 0; c < NS; ++c) {
        const int cell = tid + c * NT;
        const int ex = i0 - 1 + cell % (BX + 1), ey = j0 - 1 + cell / (BX + 1);
        sofs[c] = (cell < SC && ex <= g.nx + 1 && ey <= g.ny + 1) ? g.in_plane(ex, ey) : -1;
    }
    // the block's beta scale: max beta over the element slabs kb-1 .. ke-1 it stages (bit
    // patterns of nonnegative doubles order like the values)
    __shared__ unsigned long long smax[NT / 32];
    unsigned long long bm = 0ull;
    for (int ez = kb - 1; ez < ke; ++ez) {
        const int64_t base = g.plane_base(ez);
#pragma unroll
        for (int c = 0; c < NS; ++c)
            if (sofs[c] >= 0) bm = max(bm, (unsigned long long)__double_as_longlong(beta[base + sofs[c]]));
    }
    for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    if ((tid & 31) == 0) smax[tid >> 5] = bm;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) bm = max(bm, smax[w]);
    const int tb = beta_shift(bm);
    // A x = -(h / 12) 2^-(s + tb) sum_e B_e I_e, the power of two applied in two steps so that
    // neither factor leaves the FP64 range
    const double cB = ldexp(1.0, -tb);
    double rp[NP], rb[NS];
    auto fetch_plane = [&](int k) {
        const int64_t base = g.plane_base(k);
#pragma unroll
        for (int c = 0; c < NP; ++c)
            if (pofs[c] >= 0) rp[c] = x[base + pofs[c]];
    };
    auto fetch_slab = [&](int ez) {
        const int64_t base = g.plane_base(ez);
#pragma unroll
        for (int c = 0; c < NS; ++c)
            if (sofs[c] >= 0) rb[c] = beta[base + sofs[c]];
    };
    auto store_plane = [&](int k) {
        long long* dst = &sv[(k + 3) % 3][0][0];
#pragma unroll
        for (int c = 0; c < NP; ++c)
            if (tid + c * NT < PC) dst[tid + c * NT] = pofs[c] >= 0 ? fx::to_fixed(rp[c], fr.s) : 0ll;
    };
    auto store_slab = [&](int ez) {
        long long* dst = &sb[(ez + 2) % 2][0][0];
#pragma unroll
        for (int c = 0; c < NS; ++c)
            if (tid + c * NT < SC) dst[tid + c * NT] = sofs[c] >= 0 ? fx::to_fixed(rb[c], tb) : 0ll;
    };

    fetch_plane(kb - 1);
    store_plane(kb - 1);
    fetch_plane(kb);
    store_plane(kb);
    fetch_slab(kb - 1);
    store_slab(kb - 1);
    if (kb < ke) {
        fetch_plane(kb + 1);
        fetch_slab(kb);
    }
    for (int k = kb; k < ke; ++k) {
        store_plane(k + 1);
        store_slab(k);
        if (k + 1 < ke) {
            fetch_plane(k + 2);
            fetch_slab(k + 1);
        }
        __syncthreads();
        const int i = i0 + tx, j = j0 + ty;
        if (i <= rg.ihi && j <= rg.jhi) {
            const int pl[3] = {(k + 2) % 3, k % 3, (k + 1) % 3};  // planes k-1, k, k+1
            auto X = [&](int dx, int dy, int dz) -> long long { return sv[pl[dz + 1]][ty + 1 + dy][tx + 1 + dx]; };
            const long long x4 = 4 * X(0, 0, 0);
            Acc128 S;
#pragma unroll
            for (int ez = 0; ez < 2; ++ez)
#pragma unroll
                for (int ey = 0; ey < 2; ++ey)
#pragma unroll
                    for (int ex = 0; ex < 2; ++ex) {
                        // element (i-1+ex, j-1+ey, k-1+ez); its other nodes lie towards (ox, oy, oz)
                        const int ox = ex ? 1 : -1, oy = ey ? 1 : -1, oz = ez ? 1 : -1;
                        const long long I = (X(ox, oy, 0) + X(ox, 0, oz)) + (X(0, oy, oz) + X(ox, oy, oz)) - x4;
                        S.add_prod(sb[ez ? k % 2 : (k + 1) % 2][ty + ey][tx + ex], I);
                    }
            double Av = cA * (S.value() * cB);
            if (ROBIN && (i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz)) {
                // S_a S_b X over the face through the node, in-face axes (a, b); the centre
                // weight is 2 at the face's edge (end of that axis) and 4 inside
                const long long sx0 = (i == 0 || i == g.nx) ? 2 : 4, sy0 = (j == 0 || j == g.ny) ? 2 : 4,
                                sz0 = (k == 0 || k == g.nz) ? 2 : 4;
                auto face = [&](int an) -> long long {
                    long long I = 0;
#pragma unroll
                    for (int u = -1; u <= 1; ++u)
#pragma unroll
                        for (int v = -1; v <= 1; ++v) {
                            long long w;
                            long long xv;
                            if (an == 0) {
                                w = (u ? 1 : sy0) * (v ? 1 : sz0);
                                xv = X(0, u, v);
                            } else if (an == 1) {
                                w = (u ? 1 : sx0) * (v ? 1 : sz0);
                                xv = X(u, 0, v);
                            } else {
                                w = (u ? 1 : sx0) * (v ? 1 : sy0);
                                xv = X(u, v, 0);
                            }
                            I += w * xv;
                        }
                    return I;
                };
                const int pos[3] = {i, j, k}, nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const int an = f / 2;
                    if (((op_robin_mask >> f) & 1) && pos[an] == ((f & 1) ? nn[an] : 0))
                        Av = fma(rw[f] * fr.inv, (double)face(an), Av);
                }
            }
            body(i, j, k, g.plane_base(k) + g.in_plane(i, j), Av);
        }
        __syncthreads();
    }
}

}  // namespace ecmg
