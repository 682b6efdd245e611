// march.cuh -- the tiled z-march of the matrix-free operator, shared by the single-problem
// kernels (jcg.cu) and the batched ones (batch.cu).
#pragma once

#include <type_traits>
#include <utility>

#include "ecmg_internal.cuh"
#include "stencil_core.cuh"

namespace ecmg {
namespace mt {
constexpr int BX = 32, BY = 8, NT = BX * BY;  // block: 32 x 8 nodes of a plane
}  // namespace mt

using mt::BX;
using mt::BY;

// ---- the tiled z-march -------------------------------------------------------------------
// Each block owns the BX x BY column of nodes of tile (bx, by) over planes [kb, ke), kb = bz kz.
// Three node planes of the operand (k-1, k, k+1) and two element slabs of beta (k-1, k) live in
// shared memory; the operand of a plane is produced by src(offset), so K1 can form p on the fly.
// Nodes a march visits: the box [ilo, ihi] x [jlo, jhi] x [klo, khi] of node indices.
struct NodeRange {
    int ilo, ihi, jlo, jhi, klo, khi;
};
__host__ __device__ inline NodeRange all_nodes(const Grid& g) { return NodeRange{0, g.nx, 0, g.ny, 0, g.nz}; }
// Every node off the Dirichlet faces: kernels whose result vanishes on Dirichlet nodes need
// no more, and grids of 2^k + 1 nodes then fill their 32-wide tiles.
__host__ __device__ inline NodeRange free_nodes(const Grid& g, const Op& op)
{
    return NodeRange{op.bc[0] == 0 ? 1 : 0, op.bc[1] == 0 ? g.nx - 1 : g.nx, op.bc[2] == 0 ? 1 : 0,
                     op.bc[3] == 0 ? g.ny - 1 : g.ny, op.bc[4] == 0 ? 1 : 0, op.bc[5] == 0 ? g.nz - 1 : g.nz};
}
// Tiles of a range: BX x BY columns of kz planes; at least one per axis, so that a kernel with
// a reduction has a block for an empty range too.
__host__ __device__ inline int range_tiles_x(const NodeRange& r) { return max((r.ihi - r.ilo + BX) / BX, 1); }
__host__ __device__ inline int range_tiles_y(const NodeRange& r) { return max((r.jhi - r.jlo + BY) / BY, 1); }
__host__ __device__ inline int range_tiles_z(const NodeRange& r, int kz) { return max((r.khi - r.klo + kz) / kz, 1); }

// Operand source of a march: a callable v(offset), or an object with fetch(offset) -> Raw
// (global loads only) and make(Raw) -> value, so that the loads for the next plane can be in
// flight while the current plane is computed.
template <typename S, typename = void>
struct has_fetch : std::false_type {
};
template <typename S>
struct has_fetch<S, std::void_t<decltype(&S::fetch)>> : std::true_type {
};
template <typename S, typename VT, bool F = has_fetch<S>::value>
struct SourceOf;
template <typename S, typename VT>
struct SourceOf<S, VT, true> {
    using Raw = decltype(std::declval<const S&>().fetch(int64_t(0)));
    static __device__ __forceinline__ Raw fetch(const S& s, int64_t o) { return s.fetch(o); }
    static __device__ __forceinline__ VT make(const S& s, const Raw& r) { return s.make(r); }
};
template <typename S, typename VT>
struct SourceOf<S, VT, false> {
    using Raw = VT;
    static __device__ __forceinline__ Raw fetch(const S& s, int64_t o) { return s(o); }
    static __device__ __forceinline__ VT make(const S&, const Raw& r) { return r; }
};

// The JCG search direction p = D^-1 r + beta p_old, formed as each cell is staged.
template <typename T>
struct PSource {
    const T* __restrict__ dinv;
    const T* __restrict__ r;
    const T* __restrict__ pold;
    T bcg;
    struct Raw {
        T d, r, p;
    };
    __device__ __forceinline__ Raw fetch(int64_t o) const { return Raw{dinv[o], r[o], pold[o]}; }
    __device__ __forceinline__ T make(const Raw& v) const { return v.d * v.r + bcg * v.p; }
    __device__ __forceinline__ T operator()(int64_t o) const { return make(fetch(o)); }
};

// Tile (bx, by, bz) of a node range starts at node (ilo + bx BX, jlo + by BY, klo + bz kz); body
// runs for the nodes of the range only. Each thread owns fixed cells of the staged plane and
// slab; the loads of plane k+2 and slab k+1 are issued before plane k is computed and written
// to shared memory after it (a register double buffer), so the march does not wait for HBM.
template <bool ROBIN, bool CUBE, typename VT, typename BT, typename SRC, typename BODY>
__device__ __forceinline__ void march_range(const Grid& g, const Op& op, const BT* __restrict__ beta,
                                            const NodeRange& rg, int bx, int by, int bz, int kz, SRC src, BODY body)
{
    using S = SourceOf<SRC, VT>;
    using Raw = typename S::Raw;
    constexpr int NT = mt::NT;
    constexpr int PC = (BX + 2) * (BY + 2), SC = (BX + 1) * (BY + 1);  // plane and slab cells
    constexpr int NP = (PC + NT - 1) / NT, NS = (SC + NT - 1) / NT;    // cells per thread
    __shared__ VT sv[3][BY + 2][BX + 2];
    __shared__ VT sb[2][BY + 1][BX + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int i0 = rg.ilo + bx * BX, j0 = rg.jlo + by * BY;
    const int kb = rg.klo + bz * kz;
    const int ke = min(kb + kz, rg.khi + 1);
    const Weights<VT> wts(op);

    // this thread's cells: in-plane offsets, or -1 outside the padded layout (value 0)
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
    Raw rp[NP];
    BT rb[NS];
    auto fetch_plane = [&](int k) {
        const int64_t base = g.plane_base(k);
#pragma unroll
        for (int c = 0; c < NP; ++c)
            if (pofs[c] >= 0) rp[c] = S::fetch(src, base + pofs[c]);
    };
    auto fetch_slab = [&](int ez) {
        const int64_t base = g.plane_base(ez);
#pragma unroll
        for (int c = 0; c < NS; ++c)
            if (sofs[c] >= 0) rb[c] = beta[base + sofs[c]];
    };
    auto store_plane = [&](int k) {
        VT* dst = &sv[(k + 3) % 3][0][0];
#pragma unroll
        for (int c = 0; c < NP; ++c)
            if (tid + c * NT < PC) dst[tid + c * NT] = pofs[c] >= 0 ? S::make(src, rp[c]) : VT(0);
    };
    auto store_slab = [&](int ez) {
        VT* dst = &sb[(ez + 2) % 2][0][0];
#pragma unroll
        for (int c = 0; c < NS; ++c)
            if (tid + c * NT < SC) dst[tid + c * NT] = sofs[c] >= 0 ? (VT)rb[c] : VT(0);
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
            const int pm = (k + 2) % 3, p0 = k % 3, pp = (k + 1) % 3;
            const int s0 = (k + 1) % 2, s1 = k % 2;
            auto V = [&](int dx, int dy, int dz) -> VT {
                return sv[dz < 0 ? pm : (dz > 0 ? pp : p0)][ty + 1 + dy][tx + 1 + dx];
            };
            const VT xc = V(0, 0, 0);
            const VT Av = q1_apply<true, ROBIN, CUBE, VT>(V, sb[s0][ty][tx], sb[s0][ty][tx + 1], sb[s0][ty + 1][tx],
                                                          sb[s0][ty + 1][tx + 1], sb[s1][ty][tx], sb[s1][ty][tx + 1],
                                                          sb[s1][ty + 1][tx], sb[s1][ty + 1][tx + 1], i, j, k, g, op, wts);
            body(i, j, k, g.plane_base(k) + g.in_plane(i, j), Av, xc);
        }
        __syncthreads();
    }
}

// The whole grid, every node.
template <bool ROBIN, bool CUBE, typename VT, typename BT, typename SRC, typename BODY>
__device__ __forceinline__ void march_tile(const Grid& g, const Op& op, const BT* __restrict__ beta, int bx, int by,
                                           int bz, int kz, SRC src, BODY body)
{
    march_range<ROBIN, CUBE, VT, BT>(g, op, beta, all_nodes(g), bx, by, bz, kz, src, body);
}

}  // namespace ecmg
