// k1_body.cuh -- the FP32 JCG step kernel body shared by the two-pass kernels (pq_tma.cu) and
// the single-pass ones (pq_sp.cu): TMA-staged z-march, formation of the search direction, the
// 27-point stencil, the deferred iterate update and the last-block reduction.
//
// Per block: a TBX x TBY column of nodes over a range of planes. A ring of shared memory
// buffers receives, for every node plane k, boxes of r, p_old, D^-1 (plane k) and beta
// (element slab k-1) by cp.async.bulk.tensor, each stage completing on its own mbarrier.
// One elected thread issues the copies several planes ahead, so HBM latency is hidden behind
// the stencil of the current plane. For each staged plane the block forms the new search
// direction p = D^-1 r + beta p_old once per node (tile plus halo) into a small plane buffer;
// every thread then keeps a 3x3x3 window of p and the 2x2x2 element betas of its node in
// registers while marching in z, so the 27-point stencil reads only 9 new values of p and 4
// new betas per node from shared memory. On a constant-coefficient level (one beta, every face
// Dirichlet) the body stages r and p_old only and keeps three plane sums per node column
// instead of the window.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records ECMG status 5 in the
// level state, finishes the level, waits (bounded) for its own copies still in flight and
// returns.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "jcg.cuh"
#include "jcg_core.cuh"
#include "pq_tma.cuh"
#include "stencil_core.cuh"
#include "tma.cuh"

namespace ecmg {
// Internal linkage on purpose: each translation unit that includes the body (the two-pass and
// the single-pass kernels) compiles its own copy, and no device symbol crosses units.
namespace {

using namespace tma;

constexpr int TBX = 32, TBY = 8, NT = TBX * TBY;
constexpr int SX = 40;                     // staged columns: from the 16-byte boundary at or below node i0-1
constexpr int EX = 36;                     // staged columns of e (no halo needed; 16-byte multiple)
constexpr int NSTAGE = 4;                  // ring stages of the general path (4 staged arrays each)
constexpr int NSTAGE_CC = 6;               // constant-coefficient path (2 staged arrays each; 4 and 8 measured slower)
constexpr int NSTAGE_CC_SP = 4;            // constant-coefficient single-pass path (3 staged arrays each)

// Sizes of a tile whose threads compute RY node rows each.
template <int RY>
struct Shape {
    static constexpr int NY = TBY * RY;                   // node rows of the tile
    static constexpr int SY = NY + 2;                     // staged rows: from node j0-1
    static constexpr int BOXF = SX * SY;                  // floats per staged vector
    static constexpr int BOXF_PAD = (BOXF + 31) / 32 * 32;  // 128 B multiple: TMA destinations stay aligned
    static constexpr int PX = TBX + 2, PY = NY + 2;       // formed plane of p: tile plus one-node halo
    static constexpr int NCELL = PX * PY;
    static constexpr int NFORM = (NCELL + NT - 1) / NT;   // formed cells per thread (at most)
    static constexpr int EBOXF = EX * NY;                 // floats of the staged e (own rows only)
    static constexpr int EBOXF_PAD = (EBOXF + 31) / 32 * 32;
};

// Staged arrays per stage with a halo: r and p_old; D^-1 and beta on the general path; q_old
// in the single-pass form. Then ring stages per block.
template <bool CC, bool SP>
constexpr int k1_arrays()
{
    return (CC ? 2 : 4) + (SP ? 1 : 0);
}
template <bool CC, bool SP>
constexpr int k1_stages()
{
    return CC ? (SP ? NSTAGE_CC_SP : NSTAGE_CC) : NSTAGE;
}

// Dynamic shared memory of a block: the stage ring (the staged arrays, then e of the tile's
// own rows unless NOE: the kernels of a ring of search directions move no e) plus slack to
// align it to 128 B (TMA destinations must be 128-byte aligned; the runtime only guarantees 16).
template <int RY, bool CC, bool SP, bool NOE = false>
constexpr size_t stage_smem()
{
    return (size_t)k1_stages<CC, SP>() *
               (k1_arrays<CC, SP>() * Shape<RY>::BOXF_PAD + (NOE ? 0 : Shape<RY>::EBOXF_PAD)) * sizeof(float) +
           128;
}

// Nodes K1 visits: every node not on a Dirichlet face (those keep p = q = 0).
struct Range {
    int ilo, ihi, jlo, jhi, klo, khi;
};
__host__ __device__ inline Range k1_range(const Grid& g, const Op& op)
{
    return Range{op.bc[0] == 0 ? 1 : 0, op.bc[1] == 0 ? g.nx - 1 : g.nx,
                 op.bc[2] == 0 ? 1 : 0, op.bc[3] == 0 ? g.ny - 1 : g.ny,
                 op.bc[4] == 0 ? 1 : 0, op.bc[5] == 0 ? g.nz - 1 : g.nz};
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Tile shape of the step kernel on one level: ry node rows per thread, kz planes per block.
inline dim3 k1_grid(const Range& rg, const K1Config& c)
{
    return dim3(cdiv(max(rg.ihi - rg.ilo + 1, 1), TBX), cdiv(max(rg.jhi - rg.jlo + 1, 1), TBY * c.ry),
                cdiv(max(rg.khi - rg.klo + 1, 1), c.kz));
}

inline int ry_index(int ry) { return ry == 1 ? 0 : 1; }

// compensated FP32 accumulation (TwoProduct + TwoSum); the block and grid stages merge the
// pairs in FP32 (block_merge) and widen each total to FP64 once
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float x, float y)
    {
        const float p = __fmul_rn(x, y);
        const float e = __fmaf_rn(x, y, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    // plain FP32 term (TwoSum only)
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        s = t;
        c = __fadd_rn(c, err);
    }
    __device__ __forceinline__ void merge(float2 p) { twosum_merge(s, c, p.x, p.y); }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
static_assert(NT == 256, "block_merge takes 256-thread blocks");

// Constant-coefficient operator by plane sums. With one beta bu on the level, every node the
// kernel visits interior, and the 27-point stencil of q1_interior written per plane: for the
// node column (i, j) and plane z let X(z) be p at the column, Fx(z) and Fy(z) the sums of the
// differences p - X(z) over the two x and the two y neighbours in that plane, and D(z) the sum
// of the differences over the four diagonal neighbours. Then, with dm = X(k-1) - X(k) and
// dp = X(k+1) - X(k),
//   (A p)(k) = bu [ 4 wf0 Fx(k) + 4 wf1 Fy(k) + 2 we0 (Fy(k-1) + Fy(k+1))
//                   + 2 we1 (Fx(k-1) + Fx(k+1)) + 2 we2 D(k) + wc (D(k-1) + D(k+1))
//                   + 4 (wf2 + we0 + we1 + wc) (dm + dp) ],
// since every neighbour difference splits into an in-plane difference plus dm or dp. The
// plane sums of a new plane are formed once and reused by the three nodes that need them, so
// the stencil costs about half the arithmetic of the element form; every term is still a
// difference of neighbouring values (the FP32 accuracy of the difference form). For cubic
// elements wf = 0 and we = wc, and Fx + Fy is kept as one sum.
template <int RY>
struct PlaneSums {
    float x[RY], fx[RY], fy[RY], d[RY];
};
struct CCWeights {
    float fx0, fy0, ey, ex, d0, c, z;  // the coefficients above, times bu
    float e_cube, z_cube;              // cubic elements: 2 wc bu and 12 wc bu
    __device__ __forceinline__ CCWeights(const Weights<float>& w, float bu)
        : fx0(4.f * w.wf0 * bu), fy0(4.f * w.wf1 * bu), ey(2.f * w.we0 * bu), ex(2.f * w.we1 * bu),
          d0(2.f * w.we2 * bu), c(w.wc * bu), z(4.f * (w.wf2 + w.we0 + w.we1 + w.wc) * bu),
          e_cube(2.f * w.wc * bu), z_cube(12.f * w.wc * bu)
    {
    }
};

// CC: constant coefficient -- one beta on the whole level and every face Dirichlet, so every
// node the kernel visits is interior with the same diagonal: beta and D^-1 are not streamed
// (bu and cdinv hold their values) and the operator takes the plane-sum form above.
// Where a block sits: its tile (bx, by, bz) in the level's tile grid, and its index among the
// nb blocks whose partial sums the last of them reduces. The single-problem kernels take both
// from blockIdx and gridDim (k1_block_of_grid); a batched launch decodes them from the block
// range of the block's (problem, level) item.
struct K1Block {
    int bx, by, bz;
    int bid, nb;
};
__device__ __forceinline__ K1Block k1_block_of_grid()
{
    return K1Block{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                   (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)),
                   (int)(gridDim.x * gridDim.y * gridDim.z)};
}

// Scalars a K1 block needs before its first plane, loaded together at kernel entry so that the
// block pays one global-memory round trip for them.
struct K1Scalars {
    int done;     // the level has finished: nothing to do
    float bcg;    // beta of the CG recurrence
    float ap;     // alpha of the previous step (deferred correction e += ap p_old)
    float cdinv;  // CC: the constant D^-1
    float bu;     // CC: the constant beta
    int pw = -1;  // ring slot of p_old (ring of search directions; -1: p_old is its own vector)
    int skip = 0; // a step behind one that asked for a replacement: return, conditions untouched
};

// Last block of a single-pass step. alpha comes from the measured r.z (this step's r) and p.q;
// the residual of the step, r' = r - alpha q, is not formed until the next step, so its norms
// are expanded in the dots of this pass:
//   r'.D^-1 r' = r.z - 2 alpha r.D^-1 q + alpha^2 q.D^-1 q,   r'.r' = r.r - 2 alpha r.q + alpha^2 q.q,
// and the test and recurrence of a two-pass step (update_epilogue) take them. Should the
// expansion cancel to a value that is not positive, the FP64 residual is taken at once.
__device__ __forceinline__ void sp_epilogue(SolveState* st, double pq, double rz, double rzq, double qzq, double rr,
                                            double rq, double qq, int pidx, CondHandles ch)
{
    st->alpha_prev = 0.0;  // applied to e by every block above
    st->p_latest = pidx;
    st->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
        st->status = 4;
        st->done = 1;
    } else {
        const double a = rz / pq;
        st->alpha = a;
        st->rho = rz;
        const double rz1 = rz - 2.0 * a * rzq + a * a * qzq;
        const double rr1 = rr - 2.0 * a * rq + a * a * qq;
        if (rz1 > 0.0 && rr1 > 0.0) {
            update_epilogue<true>(st, rz1, rr1);
        } else {
            st->iters += 1;
            st->alpha_prev = a;
            st->rr = 0.0;
            st->need_update = 1;
        }
    }
    if (ch.use) {
        cudaGraphSetConditional(ch.loop, st->done ? 0u : 1u);
        cudaGraphSetConditional(ch.update, st->need_update ? 1u : 0u);
    }
}

// One block of the step kernel. Two-pass form (SP false): p = D^-1 r + beta p_old, q = A p,
// e += alpha_prev p_old and p.q; the residual kernel follows. Single-pass form (SP true): the
// residual update of the previous step, r = r_old - alpha_prev q_old, is applied to every
// staged value of r (tile and halo) before p is formed; the block stores the new r into rnew
// and also sums r.r, r.q, q.q (and, on the general path, r.D^-1 r, D^-1 r.q, q.D^-1 q) for
// sp_epilogue. The old r and q come from one buffer of a pair and the new ones go to the
// other, since neighbouring blocks read the old values in their halo.
template <bool ROBIN, bool CUBE, int RY, bool CC, bool SP, bool NOE = false>
__device__ __forceinline__ void k1_body(const CUtensorMap& m_r, const CUtensorMap& m_pold, const CUtensorMap& m_dinv,
                                        const CUtensorMap& m_beta, const CUtensorMap& m_qold, const CUtensorMap& m_e,
                                        const Grid& g, const Op& op, const Range& rg, float* __restrict__ pnew,
                                        float* __restrict__ q, float* __restrict__ rnew, float* __restrict__ e,
                                        SolveState* st, double* partials, int pidx, CondHandles ch, int kz,
                                        KTimer* tm, const K1Scalars sc, const K1Block kb,
                                        double* ring_alpha = nullptr, int ring_R = 0)
{
    using S = Shape<RY>;
    extern __shared__ __align__(128) unsigned char k1_smem[];
    // the ring of staged boxes: NS stages of NA arrays (r, p_old[, D^-1, beta][, q_old]) and e
    constexpr int NA = k1_arrays<CC, SP>(), NS = k1_stages<CC, SP>();
    constexpr int NB = CC ? 2 : 4;                           // arrays staged at every step
    constexpr int AQ = NB;                                   // array index of q_old
    constexpr int NP = SP ? (CC ? 4 : 7) : 1;                // block sums
    constexpr int STAGEF = NA * S::BOXF_PAD + (NOE ? 0 : S::EBOXF_PAD);  // floats per stage
    float* ring = reinterpret_cast<float*>(k1_smem + ((128u - (smem_u32(k1_smem) & 127u)) & 127u));
    // array a (NA = e) of ring slot `slot`
    auto box = [&](int slot, int a) -> float* { return ring + slot * STAGEF + a * S::BOXF_PAD; };
    __shared__ float P[2][S::PY][S::PX];
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ float2 red[8 * NP], red_out[NP];
    __shared__ int bad;
    __shared__ int issued_hi;              // highest staged plane index issued so far
    __shared__ unsigned int ticket;

    if (sc.skip) return;
    if (sc.done) {
        // single pass: no residual kernel follows, so the loop's conditions are cleared here
        if (SP && ch.use && kb.bid == 0 && (threadIdx.x | threadIdx.y) == 0) {
            cudaGraphSetConditional(ch.loop, 0);
            cudaGraphSetConditional(ch.update, 0);
        }
        return;
    }
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TBX * ty;
    if (tm && tid == 0) atomicMin(&tm->t0, global_ns());
    const int i0 = rg.ilo + kb.bx * TBX, j0 = rg.jlo + kb.by * S::NY;
    const int k0 = rg.klo + kb.bz * kz;
    const int ke = min(k0 + kz, rg.khi + 1);
    const int P0 = k0 - 1;                 // first staged node plane
    const int nplanes = ke - k0 + 2;       // planes k0-1 .. ke
    // NOE: no e box in the stages, so no deferred correction (the caller passes ap = 0)
    const float bcg = sc.bcg, ap = NOE ? 0.f : sc.ap, cdinv = sc.cdinv, bu = sc.bu;
    // Node i sits in column i + XL of the padded layout. The box starts at the 16-byte
    // boundary bx at or below node i0-1's column, and node i0-1 is staged column sh.
    const int bx = (i0 + XL - 1) & ~3;
    const int sh = i0 + XL - 1 - bx;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
    }
    __syncthreads();

    // Stage t (ring slot t mod NS) holds node plane P0+t (memory plane P0+t+1) and element
    // slab P0+t-1 (memory plane P0+t); row 0 of a box is node row j0-1 (memory row j0). Its e
    // box holds the tile's own node rows j0.. of plane P0+t (memory row j0+1); it is staged only
    // when the deferred correction is live (ap != 0), and so is q_old of the single-pass form.
    const uint32_t stage_bytes =
        (uint32_t)sizeof(float) * (NB * S::BOXF + (ap != 0.f ? (SP ? S::BOXF : 0) + S::EBOXF : 0));
    auto issue = [&](int t, int slot) {
        uint64_t* b = &bar[slot];
        const int kk = P0 + t;
        mbar_expect_tx(b, stage_bytes);
        tma_load_3d(box(slot, 0), &m_r, bx, j0, kk + 1, b);
        if (sc.pw >= 0) tma_load_4d(box(slot, 1), &m_pold, bx, j0, kk + 1, sc.pw, b);
        else tma_load_3d(box(slot, 1), &m_pold, bx, j0, kk + 1, b);
        if (!CC) {
            tma_load_3d(box(slot, 2), &m_dinv, bx, j0, kk + 1, b);
            tma_load_3d(box(slot, 3), &m_beta, bx, j0, kk, b);
        }
        if (SP && ap != 0.f) tma_load_3d(box(slot, AQ), &m_qold, bx, j0, kk + 1, b);
        if (ap != 0.f) tma_load_3d(box(slot, NA), &m_e, bx, j0 + 1, kk + 1, b);
    };
    if (tid == 0) {
        for (int t = 0; t < NS && t < nplanes; ++t) issue(t, t);
        issued_hi = min(NS, nplanes) - 1;
    }

    // this thread: column i, node rows jt .. jt+RY-1, of which the first nown are in range
    const int i = i0 + tx, jt = j0 + ty * RY;
    const int nown = i <= rg.ihi ? min(RY, rg.jhi - jt + 1) : 0;
    const Weights<float> wts(op);
    const int pitch = g.pitch;

    // offset of the thread's first node on the plane computed next (plane k0 at step t = 2)
    int64_t o = g.plane_base(P0 - 1) + g.in_plane(min(i, g.nx + 1), min(jt, g.ny + 1));
    // the cells of the formed plane this thread fills, as staged offsets
    int sidx[S::NFORM];
#pragma unroll
    for (int f = 0; f < S::NFORM; ++f) {
        const int c = tid + f * NT;
        sidx[f] = c < S::NCELL ? (c / S::PX) * SX + (c % S::PX) + sh : -1;
    }

    float wA[RY + 2][3], wB[RY + 2][3], wC[RY + 2][3];  // three planes of the p window, [y][x]
    float bA[RY + 1][2], bB[RY + 1][2];                 // element betas of two slabs, [ey][ex]
    float pown_prev[RY], e_cur[RY];                     // p_old and e of the own nodes, plane k
    float r_cur[RY], d_cur[RY];                         // SP: new r and D^-1 of the own nodes, plane k
    PlaneSums<RY> sA, sB, sC;                           // CC: plane sums of three planes
    const CCWeights cw(wts, bu);
#pragma unroll
    for (int r = 0; r < RY; ++r) pown_prev[r] = e_cur[r] = r_cur[r] = d_cur[r] = 0.f;
    KSum acc;
    KSum a_rr, a_rq, a_qq, a_rz, a_zq, a_qzq;  // SP sums (the last three on the general path)
    int t_done = -1;                     // last stage waited for
    int t = 0;
    int slot = 0;                        // ring slot of stage t
    uint32_t phase = 0;                  // mbarrier phase parity of stage t
    bool stop = false;

    // One plane: stage t brings node plane kk = P0 + t into wp and beta slab kk-1 into bn;
    // then node plane kk-1 is computed from the window (wm, w0, wp) = planes (kk-2, kk-1, kk)
    // and the slabs (bo, bn) = (kk-2, kk-1). The caller rotates the arrays instead of moving
    // values, so the unrolled loop below needs no register copies. Jc is the step's position
    // J = t mod 6 in that loop: with a 6-stage ring (the two-pass constant-coefficient path) the
    // ring slot is J and the formed-plane buffer J mod 2, both known at compile time, so every
    // shared-memory address below is a register plus a constant.
    auto step = [&](auto Jc, float(&wm)[RY + 2][3], float(&w0)[RY + 2][3], float(&wp)[RY + 2][3],
                    float(&bo)[RY + 1][2], float(&bn)[RY + 1][2], PlaneSums<RY>& sm, PlaneSums<RY>& s0,
                    PlaneSums<RY>& sp) {
        constexpr int J = decltype(Jc)::value;
        constexpr bool FS = NS == 6;
        const int cs = FS ? J : slot;
        const int kk = P0 + t;
        const float* Sr = box(cs, 0);
        const float* Sp = box(cs, 1);
        const float* Sd = box(cs, 2);
        const float* Sbeta = box(cs, 3);
        const float* Sq = box(cs, AQ);
        const float* Se = box(cs, NA);
        if (!mbar_wait(&bar[cs], phase)) bad = 1;
        t_done = t;
        // e of the nodes computed at the next step (plane kk), from this stage: read before the
        // next step's barrier, after which the slot may be refilled
        float e_next[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) e_next[r] = ap != 0.f ? Se[(ty * RY + r) * EX + tx + 1 + sh] : 0.f;
        // form p of plane kk for the tile plus halo
        float* Pk = &P[FS ? (J & 1) : (kk & 1)][0][0];
#pragma unroll
        for (int f = 0; f < S::NFORM; ++f) {
            const int s = sidx[f];
            if ((f + 1) * NT <= S::NCELL || s >= 0) {
                float rv = Sr[s];
                if (SP && ap != 0.f) rv = fmaf(-ap, Sq[s], rv);
                Pk[tid + f * NT] = fmaf(CC ? cdinv : Sd[s], rv, bcg * Sp[s]);
            }
        }
        float pown_new[RY], r_new[RY], d_new[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int so = (ty * RY + r + 1) * SX + tx + 1 + sh;
            pown_new[r] = ap != 0.f ? Sp[so] : 0.f;  // only the correction e += ap p_old reads it
            if (SP) {
                float rv = Sr[so];
                if (ap != 0.f) rv = fmaf(-ap, Sq[so], rv);  // as the formed value of this node
                r_new[r] = rv;
                d_new[r] = CC ? cdinv : Sd[so];
            }
        }
        __syncthreads();
        if (bad) {
            stop = true;
            return;
        }
        if (tid == 0 && t >= 1 && t - 1 + NS < nplanes) {
            issue(t - 1 + NS, FS ? (J + NS - 1) % NS : (slot == 0 ? NS - 1 : slot - 1));  // the slot of stage t-1
            issued_hi = t - 1 + NS;
        }
        const float(*Pp)[S::PX] = P[FS ? (J & 1) : (kk & 1)];
        if (CC) {
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const float* c0 = &Pp[ty * RY + r + 1][tx + 1];
                const float c = c0[0];
                const float fx = (c0[-1] - c) + (c0[1] - c);
                const float fy = (c0[-S::PX] - c) + (c0[S::PX] - c);
                sp.x[r] = c;
                sp.fx[r] = CUBE ? fx + fy : fx;
                sp.fy[r] = fy;
                sp.d[r] = ((c0[-S::PX - 1] - c) + (c0[-S::PX + 1] - c)) + ((c0[S::PX - 1] - c) + (c0[S::PX + 1] - c));
            }
        } else {
#pragma unroll
            for (int yy = 0; yy < RY + 2; ++yy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) wp[yy][dx] = Pp[ty * RY + yy][tx + dx];
            const float* Sb = Sbeta + ty * RY * SX + tx + sh;
#pragma unroll
            for (int yy = 0; yy < RY + 1; ++yy)
#pragma unroll
                for (int ex = 0; ex < 2; ++ex) bn[yy][ex] = Sb[yy * SX + ex];
        }

        if (t >= 2) {
            const int k = kk - 1;
            float pq_plane = 0.f;  // two-pass: p.q of this plane's own nodes, one TwoSum per plane
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                if (r < nown) {
                    auto V = [&](int dx, int dy, int dz) -> float {
                        return dz < 0 ? wm[r + 1 + dy][dx + 1]
                                      : (dz > 0 ? wp[r + 1 + dy][dx + 1] : w0[r + 1 + dy][dx + 1]);
                    };
                    float xc, Av;
                    if (CC) {
                        xc = s0.x[r];
                        const float dz = (sm.x[r] - xc) + (sp.x[r] - xc);
                        if (CUBE) {
                            Av = fmaf(cw.z_cube, dz,
                                      fmaf(cw.c, sm.d[r] + sp.d[r], cw.e_cube * ((sm.fx[r] + sp.fx[r]) + s0.d[r])));
                        } else {
                            Av = fmaf(cw.z, dz,
                                      fmaf(cw.c, sm.d[r] + sp.d[r],
                                           fmaf(cw.d0, s0.d[r],
                                                fmaf(cw.ex, sm.fx[r] + sp.fx[r],
                                                     fmaf(cw.ey, sm.fy[r] + sp.fy[r],
                                                          fmaf(cw.fy0, s0.fy[r], cw.fx0 * s0.fx[r]))))));
                        }
                    } else {
                        xc = w0[r + 1][1];
                        Av = q1_apply<false, ROBIN, CUBE, float>(V, bo[r][0], bo[r][1], bo[r + 1][0], bo[r + 1][1],
                                                                 bn[r][0], bn[r][1], bn[r + 1][0], bn[r + 1][1], i,
                                                                 jt + r, k, g, op, wts);
                    }
                    const int64_t orr = o + r * pitch;
                    pnew[orr] = xc;
                    q[orr] = Av;
                    if (ap != 0.f) e[orr] = fmaf(ap, pown_prev[r], e_cur[r]);
                    if (SP) acc.add_prod(xc, Av);
                    else pq_plane = fmaf(xc, Av, pq_plane);
                    if (SP) {
                        const float rc = r_cur[r];
                        rnew[orr] = rc;
                        a_rr.add_prod(rc, rc);
                        a_rq.add_prod(rc, Av);
                        a_qq.add_prod(Av, Av);
                        if (!CC) {
                            const float d = d_cur[r], zc = d * rc;
                            a_rz.add_prod(rc, zc);
                            a_zq.add_prod(zc, Av);
                            a_qzq.add_prod(Av, d * Av);
                        }
                    }
                }
            }
            if (!SP) acc.add(pq_plane);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            pown_prev[r] = pown_new[r];
            e_cur[r] = e_next[r];
            if (SP) {
                r_cur[r] = r_new[r];
                d_cur[r] = d_new[r];
            }
        }
        o += g.plane;
        if (++slot == NS) {
            slot = 0;
            phase ^= 1u;
        }
        if (++t >= nplanes) stop = true;
    };
    // period 6 = lcm(3 window planes, 2 beta slabs)
    using std::integral_constant;
    for (;;) {
        step(integral_constant<int, 0>{}, wA, wB, wC, bA, bB, sA, sB, sC);
        if (stop) break;
        step(integral_constant<int, 1>{}, wB, wC, wA, bB, bA, sB, sC, sA);
        if (stop) break;
        step(integral_constant<int, 2>{}, wC, wA, wB, bA, bB, sC, sA, sB);
        if (stop) break;
        step(integral_constant<int, 3>{}, wA, wB, wC, bB, bA, sA, sB, sC);
        if (stop) break;
        step(integral_constant<int, 4>{}, wB, wC, wA, bA, bB, sB, sC, sA);
        if (stop) break;
        step(integral_constant<int, 5>{}, wC, wA, wB, bB, bA, sC, sA, sB);
        if (stop) break;
    }

    if (bad) {
        // a copy never arrived: record it, finish the level, drain what is still in flight
        if (tid == 0) {
            st->status = 5;
            st->done = 1;
            if (SP && ch.use) {
                cudaGraphSetConditional(ch.loop, 0);
                cudaGraphSetConditional(ch.update, 0);
            }
            for (int t = t_done; t <= issued_hi; ++t)
                (void)mbar_wait(&bar[t % NS], (uint32_t)((t / NS) & 1));
        }
        return;
    }

    // grid reduction of p.q (and the single-pass sums), last block advances the recurrence;
    // partials holds the compensated pair of sum c of block b at c * nb + b (a float2 per double
    // slot), and the last block merges them in the same FP32 arithmetic before the one widening
    // to FP64 of each sum
    KSum kv[NP];
    kv[0] = acc;
    if constexpr (SP) {
        kv[1] = a_rr;
        kv[2] = a_rq;
        kv[3] = a_qq;
        if constexpr (!CC) {
            kv[4] = a_rz;
            kv[5] = a_zq;
            kv[6] = a_qzq;
        }
    }
    const int nb = kb.nb, bid = kb.bid;
    float2* pp = reinterpret_cast<float2*>(partials);
    block_merge<NP>(kv, red, red_out);
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NP; ++c) pp[c * nb + bid] = red_out[c];
        __threadfence();
        ticket = atomicAdd(&st->arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return;
    __threadfence();
#pragma unroll
    for (int c = 0; c < NP; ++c) kv[c] = KSum{};
    for (int b = tid; b < nb; b += NT)
#pragma unroll
        for (int c = 0; c < NP; ++c) kv[c].merge(__ldcg(&pp[c * nb + b]));
    block_merge<NP>(kv, red, red_out);
    if (tid == 0) {
        double v[NP];
#pragma unroll
        for (int c = 0; c < NP; ++c) v[c] = (double)red_out[c].x + (double)red_out[c].y;
        if (tm) {
            tm->ns += global_ns() - tm->t0;
            tm->n += 1;
            tm->t0 = ~0ull;
        }
        st->arrive = 0u;
        if constexpr (SP) {
            // constant coefficient: D^-1 is the constant cdinv on every node summed
            const double cd = (double)cdinv;
            if constexpr (CC) sp_epilogue(st, v[0], cd * v[1], cd * v[2], cd * v[3], v[1], v[2], v[3], pidx, ch);
            else sp_epilogue(st, v[0], v[4], v[5], v[6], v[1], v[2], v[3], pidx, ch);
            return;
        }
        const double pq = v[0];
        st->alpha_prev = 0.0;
        st->p_latest = pidx;
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->status = 4;
            st->done = 1;
            if (ch.use) cudaGraphSetConditional(ch.loop, 0);
        } else {
            st->alpha = st->rho / pq;
            if (ring_alpha) {
                // the new direction is pending in the next ring slot with its step alpha
                const int jn = (sc.pw + 1) % ring_R;
                ring_alpha[jn] = st->alpha;
                st->pj = jn;
                st->pend += 1;
            }
        }
    }
}


}  // namespace
}  // namespace ecmg
