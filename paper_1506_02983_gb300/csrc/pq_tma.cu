// pq_tma.cu -- K1 of the FP32 JCG iteration with TMA-staged planes.
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
// Dirichlet) a kernel of its own stages r and p_old only and keeps three plane sums per node
// column instead of the window.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records ECMG status 5 in the
// level state, finishes the level, waits (bounded) for its own copies still in flight and
// returns.
#include <cuda.h>

#include "jcg.cuh"
#include "pq_tma.cuh"
#include "stencil_core.cuh"
#include "tma.cuh"

namespace ecmg {
namespace {

using namespace tma;

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TBX = 32, TBY = 8, NT = TBX * TBY;
constexpr int SX = 40;                     // staged columns: from the 16-byte boundary at or below node i0-1
constexpr int EX = 36;                     // staged columns of e (no halo needed; 16-byte multiple)
constexpr int NSTAGE = 4;                  // ring stages of the general path (4 staged arrays each)
constexpr int NSTAGE_CC = 6;               // constant-coefficient path (2 staged arrays each; 4 and 8 measured slower)

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

// Dynamic shared memory of a block: the stage ring (NA staged arrays per stage: r, p_old and,
// on the general path, D^-1 and beta; then e of the tile's own rows) plus slack to align it to
// 128 B (TMA destinations must be 128-byte aligned; the runtime only guarantees 16).
template <int RY, int NA>
constexpr size_t stage_smem()
{
    return (size_t)(NA == 2 ? NSTAGE_CC : NSTAGE) * (NA * Shape<RY>::BOXF_PAD + Shape<RY>::EBOXF_PAD) * sizeof(float) +
           128;
}

// Nodes K1 visits: every node not on a Dirichlet face (those keep p = q = 0).
struct Range {
    int ilo, ihi, jlo, jhi, klo, khi;
};
inline Range k1_range(const Grid& g, const Op& op)
{
    return Range{op.bc[0] == 0 ? 1 : 0, op.bc[1] == 0 ? g.nx - 1 : g.nx,
                 op.bc[2] == 0 ? 1 : 0, op.bc[3] == 0 ? g.ny - 1 : g.ny,
                 op.bc[4] == 0 ? 1 : 0, op.bc[5] == 0 ? g.nz - 1 : g.nz};
}

// compensated FP32 accumulation (TwoProduct + TwoSum), promoted to FP64 per thread
struct CSum {
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
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <int NP>
__device__ __forceinline__ void block_sum(double (&v)[NP], double* sh)
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = NT / 32;
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
// Scalars a K1 block needs before its first plane, loaded together at kernel entry so that the
// block pays one global-memory round trip for them.
struct K1Scalars {
    int done;     // the level has finished: nothing to do
    float bcg;    // beta of the CG recurrence
    float ap;     // alpha of the previous step (deferred correction e += ap p_old)
    float cdinv;  // CC: the constant D^-1
    float bu;     // CC: the constant beta
};

template <bool ROBIN, bool CUBE, int RY, bool CC>
__device__ __forceinline__ void k1_body(const CUtensorMap& m_r, const CUtensorMap& m_pold, const CUtensorMap& m_dinv,
                                        const CUtensorMap& m_beta, const CUtensorMap& m_e, const Grid& g, const Op& op,
                                        const Range& rg, float* __restrict__ pnew, float* __restrict__ q,
                                        float* __restrict__ e, SolveState* st, double* partials, int pidx,
                                        CondHandles ch, int kz, KTimer* tm, const K1Scalars sc)
{
    using S = Shape<RY>;
    extern __shared__ __align__(128) unsigned char k1_smem[];
    // the ring of staged boxes: NS stages of NA arrays (r, p_old[, D^-1, beta]) and e
    constexpr int NA = CC ? 2 : 4, NS = CC ? NSTAGE_CC : NSTAGE;
    constexpr int STAGEF = NA * S::BOXF_PAD + S::EBOXF_PAD;  // floats per stage
    float* ring = reinterpret_cast<float*>(k1_smem + ((128u - (smem_u32(k1_smem) & 127u)) & 127u));
    // array a (NA = e) of ring slot `slot`
    auto box = [&](int slot, int a) -> float* { return ring + slot * STAGEF + a * S::BOXF_PAD; };
    __shared__ float P[2][S::PY][S::PX];
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ double red[32];
    __shared__ int bad;
    __shared__ int issued_hi;              // highest staged plane index issued so far
    __shared__ unsigned int ticket;

    if (sc.done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TBX * ty;
    if (tm && tid == 0) atomicMin(&tm->t0, global_ns());
    const int i0 = rg.ilo + blockIdx.x * TBX, j0 = rg.jlo + blockIdx.y * S::NY;
    const int kb = rg.klo + blockIdx.z * kz;
    const int ke = min(kb + kz, rg.khi + 1);
    const int P0 = kb - 1;                 // first staged node plane
    const int nplanes = ke - kb + 2;       // planes kb-1 .. ke
    const float bcg = sc.bcg, ap = sc.ap, cdinv = sc.cdinv, bu = sc.bu;
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
    // when the deferred correction is live (ap != 0).
    const uint32_t stage_bytes = (uint32_t)sizeof(float) * (NA * S::BOXF + (ap != 0.f ? S::EBOXF : 0));
    auto issue = [&](int t, int slot) {
        uint64_t* b = &bar[slot];
        const int kk = P0 + t;
        mbar_expect_tx(b, stage_bytes);
        tma_load_3d(box(slot, 0), &m_r, bx, j0, kk + 1, b);
        tma_load_3d(box(slot, 1), &m_pold, bx, j0, kk + 1, b);
        if (!CC) {
            tma_load_3d(box(slot, 2), &m_dinv, bx, j0, kk + 1, b);
            tma_load_3d(box(slot, 3), &m_beta, bx, j0, kk, b);
        }
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

    // offset of the thread's first node on the plane computed next (plane kb at step t = 2)
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
    PlaneSums<RY> sA, sB, sC;                           // CC: plane sums of three planes
    const CCWeights cw(wts, bu);
#pragma unroll
    for (int r = 0; r < RY; ++r) pown_prev[r] = e_cur[r] = 0.f;
    CSum acc;
    int t_done = -1;                     // last stage waited for
    int t = 0;
    int slot = 0;                        // ring slot of stage t
    uint32_t phase = 0;                  // mbarrier phase parity of stage t
    bool stop = false;

    // One plane: stage t brings node plane kk = P0 + t into wp and beta slab kk-1 into bn;
    // then node plane kk-1 is computed from the window (wm, w0, wp) = planes (kk-2, kk-1, kk)
    // and the slabs (bo, bn) = (kk-2, kk-1). The caller rotates the arrays instead of moving
    // values, so the unrolled loop below needs no register copies.
    auto step = [&](float(&wm)[RY + 2][3], float(&w0)[RY + 2][3], float(&wp)[RY + 2][3],
                    float(&bo)[RY + 1][2], float(&bn)[RY + 1][2], PlaneSums<RY>& sm, PlaneSums<RY>& s0,
                    PlaneSums<RY>& sp) {
        const int kk = P0 + t;
        const float* Sr = box(slot, 0);
        const float* Sp = box(slot, 1);
        const float* Sd = box(slot, 2);
        const float* Sbeta = box(slot, 3);
        const float* Se = box(slot, NA);
        if (!mbar_wait(&bar[slot], phase)) bad = 1;
        t_done = t;
        // e of the nodes computed at the next step (plane kk), from this stage: read before the
        // next step's barrier, after which the slot may be refilled
        float e_next[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) e_next[r] = ap != 0.f ? Se[(ty * RY + r) * EX + tx + 1 + sh] : 0.f;
        // form p of plane kk for the tile plus halo
        float* Pk = &P[kk & 1][0][0];
#pragma unroll
        for (int f = 0; f < S::NFORM; ++f) {
            const int s = sidx[f];
            if ((f + 1) * NT <= S::NCELL || s >= 0)
                Pk[tid + f * NT] = fmaf(CC ? cdinv : Sd[s], Sr[s], bcg * Sp[s]);
        }
        float pown_new[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) pown_new[r] = Sp[(ty * RY + r + 1) * SX + tx + 1 + sh];
        __syncthreads();
        if (bad) {
            stop = true;
            return;
        }
        if (tid == 0 && t >= 1 && t - 1 + NS < nplanes) {
            issue(t - 1 + NS, slot == 0 ? NS - 1 : slot - 1);  // the slot of stage t-1
            issued_hi = t - 1 + NS;
        }
        const float(*Pp)[S::PX] = P[kk & 1];
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
                    acc.add_prod(xc, Av);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            pown_prev[r] = pown_new[r];
            e_cur[r] = e_next[r];
        }
        o += g.plane;
        if (++slot == NS) {
            slot = 0;
            phase ^= 1u;
        }
        if (++t >= nplanes) stop = true;
    };
    // period 6 = lcm(3 window planes, 2 beta slabs)
    for (;;) {
        step(wA, wB, wC, bA, bB, sA, sB, sC);
        if (stop) break;
        step(wB, wC, wA, bB, bA, sB, sC, sA);
        if (stop) break;
        step(wC, wA, wB, bA, bB, sC, sA, sB);
        if (stop) break;
        step(wA, wB, wC, bB, bA, sA, sB, sC);
        if (stop) break;
        step(wB, wC, wA, bA, bB, sB, sC, sA);
        if (stop) break;
        step(wC, wA, wB, bB, bA, sC, sA, sB);
        if (stop) break;
    }

    if (bad) {
        // a copy never arrived: record it, finish the level, drain what is still in flight
        if (tid == 0) {
            st->status = 5;
            st->done = 1;
            for (int t = t_done; t <= issued_hi; ++t)
                (void)mbar_wait(&bar[t % NS], (uint32_t)((t / NS) & 1));
        }
        return;
    }

    // grid reduction of p.q, last block advances the recurrence
    double v[1] = {acc.value()};
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_sum<1>(v, red);
    if (tid == 0) {
        partials[bid] = v[0];
        __threadfence();
        ticket = atomicAdd(&st->arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return;
    __threadfence();
    v[0] = 0.0;
    for (int b = tid; b < nb; b += NT) v[0] += __ldcg(&partials[b]);
    block_sum<1>(v, red);
    if (tid == 0) {
        if (tm) {
            tm->ns += global_ns() - tm->t0;
            tm->n += 1;
            tm->t0 = ~0ull;
        }
        st->arrive = 0u;
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
        }
    }
}

// General path: beta and D^-1 streamed with r and p_old.
template <bool ROBIN, bool CUBE, int RY>
__global__ void __launch_bounds__(NT, RY == 1 ? (ROBIN ? 3 : 4) : 2)
k_pq32_tma(const __grid_constant__ CUtensorMap m_r, const __grid_constant__ CUtensorMap m_pold,
           const __grid_constant__ CUtensorMap m_dinv, const __grid_constant__ CUtensorMap m_beta,
           const __grid_constant__ CUtensorMap m_e, const Grid g, const Op op, const Range rg,
           float* __restrict__ pnew, float* __restrict__ q, float* __restrict__ e, SolveState* st,
           double* partials, int pidx, CondHandles ch, int kz, KTimer* tm)
{
    COUNT_LAUNCH();
    const K1Scalars sc{st->done, (float)st->beta, (float)st->alpha_prev, 0.f, 0.f};
    k1_body<ROBIN, CUBE, RY, false>(m_r, m_pold, m_dinv, m_beta, m_e, g, op, rg, pnew, q, e, st, partials, pidx, ch,
                                    kz, tm, sc);
}

// Constant-coefficient path (every face Dirichlet, one beta on the level): r, p_old and e only,
// and about half the registers of the general path, so six blocks fit on an SM instead of four
// (one node row per thread; four blocks with two rows, which an autotuned 512^3 level
// prefers). The host picks it from the level's uniform flag after the set-up; should a later
// set-up clear the flag (new beta data under a recorded graph), the kernel computes nothing
// and records status 6 so that the host records the solve again with the general path.
template <bool CUBE, int RY>
__global__ void __launch_bounds__(NT, RY == 1 ? 6 : 4)
k_pq32_cc(const __grid_constant__ CUtensorMap m_r, const __grid_constant__ CUtensorMap m_pold,
          const __grid_constant__ CUtensorMap m_e, const Grid g, const Op op, const Range rg,
          float* __restrict__ pnew, float* __restrict__ q, float* __restrict__ e, SolveState* st, double* partials,
          int pidx, CondHandles ch, int kz, KTimer* tm, const int* __restrict__ uniform,
          const float* __restrict__ beta32, const float* __restrict__ dinv32)
{
    COUNT_LAUNCH();
    const int uni = *uniform;
    const K1Scalars sc{st->done, (float)st->beta, (float)st->alpha_prev, dinv32[g.off(1, 1, 1)],
                       beta32[g.off(0, 0, 0)]};
    if (!uni) {
        if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0 && !sc.done) {
            st->status = 6;
            st->done = 1;
            if (ch.use) cudaGraphSetConditional(ch.loop, 0);
        }
        return;
    }
    k1_body<false, CUBE, RY, true>(m_r, m_pold, m_r, m_r, m_e, g, op, rg, pnew, q, e, st, partials, pidx, ch, kz, tm,
                                   sc);
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

inline dim3 k1_grid(const Range& rg, const K1Config& c)
{
    return dim3(cdiv(max(rg.ihi - rg.ilo + 1, 1), TBX), cdiv(max(rg.jhi - rg.jlo + 1, 1), TBY * c.ry),
                cdiv(max(rg.khi - rg.klo + 1, 1), c.kz));
}

int ry_index(int ry) { return ry == 1 ? 0 : 1; }

bool make_plane_map(CUtensorMap* map, const float* base, const Grid& g, int sy, int sx = SX)
{
    return encode_level_map(map, false, base, g, sx, sy);
}

template <bool ROBIN, bool CUBE, int RY>
cudaError_t prepare_one()
{
    return cudaFuncSetAttribute(k_pq32_tma<ROBIN, CUBE, RY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem<RY, 4>());
}
template <bool CUBE, int RY>
cudaError_t prepare_cc()
{
    return cudaFuncSetAttribute(k_pq32_cc<CUBE, RY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem<RY, 2>());
}

template <int RY>
cudaError_t prepare_ry()
{
    cudaError_t e = prepare_one<false, false, RY>();
    if (e == cudaSuccess) e = prepare_one<false, true, RY>();
    if (e == cudaSuccess) e = prepare_one<true, false, RY>();
    if (e == cudaSuccess) e = prepare_one<true, true, RY>();
    if (e == cudaSuccess) e = prepare_cc<false, RY>();
    if (e == cudaSuccess) e = prepare_cc<true, RY>();
    return e;
}

template <int RY>
void launch_ry(const PlaneMaps& m, int pold_is_b, const K1Config& c, const Grid& g, const Op& op, bool cc,
               const int* uniform, const float* beta32, const float* dinv32, float* pnew, float* q, float* e,
               SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm, cudaStream_t s)
{
    const int v = ry_index(RY);
    const Range rg = k1_range(g, op);
    const CUtensorMap& pold = pold_is_b ? m.pB[v] : m.pA[v];
    if (cc) {
        auto kern = op.cube ? k_pq32_cc<true, RY> : k_pq32_cc<false, RY>;
        kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, 2>(), s>>>(m.r[v], pold, m.e[v], g, op, rg, pnew, q, e,
                                                                         st, pr.buf, pidx, ch, c.kz, tm, uniform,
                                                                         beta32, dinv32);
        return;
    }
    bool robin = false;
    for (int f = 0; f < 6; ++f) robin |= op.alpha[f] != 0.0;
    auto kern = robin ? (op.cube ? k_pq32_tma<true, true, RY> : k_pq32_tma<true, false, RY>)
                      : (op.cube ? k_pq32_tma<false, true, RY> : k_pq32_tma<false, false, RY>);
    kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, 4>(), s>>>(m.r[v], pold, m.dinv[v], m.beta[v], m.e[v], g,
                                                                     op, rg, pnew, q, e, st, pr.buf, pidx, ch, c.kz,
                                                                     tm);
}

}  // namespace

bool make_plane_maps(PlaneMaps* m, const float* r, const float* pA, const float* pB, const float* dinv,
                     const float* beta, const float* e, const Grid& g)
{
    for (int v = 0; v < K1_NRY; ++v) {
        const int sy = TBY * K1_RY[v] + 2;
        if (!make_plane_map(&m->r[v], r, g, sy) || !make_plane_map(&m->pA[v], pA, g, sy) ||
            !make_plane_map(&m->pB[v], pB, g, sy) || !make_plane_map(&m->dinv[v], dinv, g, sy) ||
            !make_plane_map(&m->beta[v], beta, g, sy) || !make_plane_map(&m->e[v], e, g, TBY * K1_RY[v], EX))
            return false;
    }
    return true;
}

cudaError_t k1_prepare()
{
    cudaError_t e = prepare_ry<1>();
    if (e == cudaSuccess) e = prepare_ry<2>();
    return e;
}

bool k1_valid(const K1Config& c)
{
    return (c.ry == 1 || c.ry == 2) && c.kz >= 4 && c.kz <= 1024;
}

// One node row per thread, and enough blocks for about three per SM (152 SMs) with 4 to 128
// planes per block (small levels are latency bound: short columns spread them over more SMs).
// Levels of at least 2^18 nodes are autotuned after a solve.
K1Config k1_default(const Grid& g, const Op& op)
{
    K1Config c{1, 128};
    const Range rg = k1_range(g, op);
    const dim3 d = k1_grid(rg, K1Config{c.ry, 1 << 30});
    const int nk = max(rg.khi - rg.klo + 1, 1);
    const int gz = cdiv(152 * 3, (int)(d.x * d.y));
    c.kz = min(max(cdiv(nk, gz), 4), 128);
    return c;
}

int k1_candidates(const Grid& g, K1Config* out, int cap)
{
    (void)g;
    // planes per block; the in-between values let a level end close to a whole number of waves
    const int kzs[8] = {8, 12, 16, 24, 32, 48, 64, 128};
    int n = 0;
    for (int v = 0; v < K1_NRY; ++v)
        for (int z = 0; z < 8; ++z)
            if (n < cap) out[n++] = K1Config{K1_RY[v], kzs[z]};
    return n;
}

int64_t k1_nodes(const Grid& g, const Op& op)
{
    const Range rg = k1_range(g, op);
    return (int64_t)max(rg.ihi - rg.ilo + 1, 0) * max(rg.jhi - rg.jlo + 1, 0) * max(rg.khi - rg.klo + 1, 0);
}

int max_tma_blocks(const Grid& g)
{
    // largest grid of any valid shape: ry = 1, kz = 4, all nodes in range
    return cdiv(g.nx + 1, TBX) * cdiv(g.ny + 1, TBY) * cdiv(g.nz + 1, 4);
}

void launch_pq32_tma(const PlaneMaps& m, int pold_is_b, const K1Config& c, const Grid& g, const Op& op, bool cc,
                     const int* uniform, const float* beta32, const float* dinv32, float* pnew, float* q, float* e,
                     SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm, cudaStream_t s)
{
    if (c.ry == 1)
        launch_ry<1>(m, pold_is_b, c, g, op, cc, uniform, beta32, dinv32, pnew, q, e, st, pr, pidx, ch, tm, s);
    else launch_ry<2>(m, pold_is_b, c, g, op, cc, uniform, beta32, dinv32, pnew, q, e, st, pr, pidx, ch, tm, s);
}

unsigned long long launches_pq_tma()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
