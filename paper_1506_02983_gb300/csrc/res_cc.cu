// res_cc.cu -- the residual of the MIXED iteration on a constant-coefficient level, exact in
// 64-bit fixed point, with the iterate staged by TMA.
//
// On a level with one beta, every face Dirichlet and cubic elements, every free node is
// interior, and with the iterate in fixed point, x = X 2^-s, the assembled operator there is
// A x = c 2^-s I, c = -beta h / 36, with the integer 27-point sum of the tensor form
// (Sy Sz Dx + Sx Sz Dy + Sx Sy Dz) X, D = [1 -2 1], S = [1 4 1]. Its weights are 6 on the twelve
// edge neighbours, 3 on the eight corners, 0 on the six face neighbours and -96 at the centre,
// so with the per-plane sums F(z) (the four in-plane axis neighbours of the node column in
// plane z) and D(z) (the four in-plane diagonals),
//     I = 3 (2 (F(k-1) + F(k+1) + D(k)) + D(k-1) + D(k+1) - 32 X(k)),
// the same exact integer as the tensor form in jcg.cu, at a third of its integer work: each
// plane's sums are formed once and serve the three nodes of the column that need them. With
// B = b / c on the same scale, r = c 2^-s (B - I) is exact before its single rounding to FP32.
//
// A ring of shared-memory stages receives, per node plane, the FP64 box of x for the tile plus
// halo and the box of b / c for the tile's own nodes by cp.async.bulk.tensor; one elected
// thread issues the copies several planes ahead. Every wait is bounded: on expiry the kernel
// records status 5 in the level state, finishes the level and drains its own copies.
#include <cuda.h>

#include "fixed.cuh"
#include "jcg_core.cuh"
#include "res_cc.cuh"
#include "tma.cuh"

namespace ecmg {
namespace {

using namespace fx;
using namespace tma;

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TBX = 32, TBY = 8, NT = TBX * TBY;
constexpr int SX = 40;                 // staged x columns: from the 16-byte boundary at or below node i0-1
constexpr int SY = TBY + 2;            // staged x rows: node rows j0-1 .. j0+8
constexpr int EX = 36;                 // staged b / c columns (the tile's own rows only)
constexpr int PX = TBX + 2, PY = TBY + 2, NCELL = PX * PY;
constexpr int NFORM = (NCELL + NT - 1) / NT;
constexpr int XBOX = SX * SY;          // doubles
constexpr int BBOX = EX * TBY;         // doubles
constexpr int STAGE = XBOX + BBOX;     // doubles per stage (5504 bytes, a 128-byte multiple)
constexpr int NS = 4;
constexpr int KZ_MAX = 32;             // planes per block at most
static_assert((STAGE * 8) % 128 == 0 && (XBOX * 8) % 128 == 0, "TMA destinations stay 128-byte aligned");

constexpr size_t smem_bytes() { return (size_t)NS * STAGE * sizeof(double) + 128; }

// plane sums of one node column: X, the axis-neighbour sum F and the diagonal sum D
struct Col {
    long long x, f, d;
};

__global__ void __launch_bounds__(NT, 5)
k_res_cc(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mbc, const Grid g,
         float* __restrict__ ra, float* __restrict__ rb, SolveState* st, double* partials, int mode, CondHandles ch,
         int kz, const FixedScale* fs, const int* __restrict__ uniform, const double* __restrict__ beta,
         const float* __restrict__ dinv32)
{
    COUNT_LAUNCH();
    // rb: the single-pass buffer pair from the level state: r goes where the next step reads it
    float* __restrict__ r = (rb && st->p_latest) ? rb : ra;
    extern __shared__ __align__(128) unsigned char rc_smem[];
    __shared__ long long P[2][PY][PX];
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ float2 red[8], red_out[1];
    __shared__ int bad;
    __shared__ int issued_hi;
    __shared__ unsigned int ticket;

    // everything the block needs before its first plane, in one round trip
    const int uni = *uniform;
    const int done = st->done;
    const unsigned long long bits = max(fs->bits, st->bcbits);
    const double bu = beta[g.off(0, 0, 0)];
    const float dd = dinv32[g.off(1, 1, 1)];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TBX * ty;
    const bool first_block = (blockIdx.x | blockIdx.y | blockIdx.z) == 0;
    if (mode == RES_REPLACE && done) return;
    if (!uni) {
        // the host chose this kernel from a flag a later set-up has cleared: do nothing, ask
        // for a new recording (status 6)
        if (first_block && tid == 0 && !done) {
            st->status = 6;
            st->done = 1;
            if (ch.use) cudaGraphSetConditional(ch.loop, 0);
        }
        return;
    }
    const FixedFrame fr = fixed_frame(bits);
    Acc<float> rr;

    if (fr.finite) {
        double* ring = reinterpret_cast<double*>(rc_smem + ((128u - (smem_u32(rc_smem) & 127u)) & 127u));
        // free nodes 1 .. n-1 on every axis
        const int i0 = 1 + blockIdx.x * TBX, j0 = 1 + blockIdx.y * TBY;
        const int kb = 1 + blockIdx.z * kz;
        const int ke = min(kb + kz, g.nz);
        const int P0 = kb - 1;
        const int nplanes = ke - kb + 2;
        const int bx = (i0 + XL - 1) & ~3;  // 16-byte boundary at or below node i0-1's column
        const int sh = i0 + XL - 1 - bx;    // node i0-1 is staged column sh
        if (tid == 0) {
            for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            bad = 0;
        }
        __syncthreads();
        // stage t (slot t mod NS): x of node plane P0+t (memory plane P0+t+1, rows from node
        // row j0-1 = memory row j0) and b / c of the tile's own rows of that plane
        auto issue = [&](int t, int slot) {
            uint64_t* b = &bar[slot];
            const int kk = P0 + t;
            double* dst = ring + slot * STAGE;
            mbar_expect_tx(b, (uint32_t)(STAGE * sizeof(double)));
            tma_load_3d(dst, &mx, bx, j0, kk + 1, b);
            tma_load_3d(dst + XBOX, &mbc, bx, j0 + 1, kk + 1, b);
        };
        if (tid == 0) {
            for (int t = 0; t < NS && t < nplanes; ++t) issue(t, t);
            issued_hi = min(NS, nplanes) - 1;
        }
        const int i = i0 + tx, j = j0 + ty;
        const bool own = i <= g.nx - 1 && j <= g.ny - 1;
        const float fscale = (float)(-bu * g.h[0] / 36.0 * fr.inv);
        int64_t o = g.plane_base(P0 - 1) + g.in_plane(min(i, g.nx + 1), min(j, g.ny + 1));
        int sidx[NFORM];
#pragma unroll
        for (int f = 0; f < NFORM; ++f) {
            const int c = tid + f * NT;
            sidx[f] = c < NCELL ? (c / PX) * SX + (c % PX) + sh : -1;
        }
        const int bidx = ty * EX + tx + 1 + sh;  // own node in the b / c box
        Col cA{0, 0, 0}, cB{0, 0, 0}, cC{0, 0, 0};
        long long Bcur = 0;
        int t = 0, slot = 0, t_done = -1;
        uint32_t phase = 0;
        bool stop = false;

        // stage t brings plane kk = P0 + t; node plane kk-1 is computed from the column sums of
        // planes (kk-2, kk-1, kk) = (cm, c0, cp)
        auto step = [&](Col& cm, Col& c0, Col& cp) {
            const int kk = P0 + t;
            const double* Sx = ring + slot * STAGE;
            const double* Sb = Sx + XBOX;
            if (!mbar_wait(&bar[slot], phase)) bad = 1;
            t_done = t;
            // b / c of the node computed at the next step (plane kk), read before the next
            // step's barrier, after which the slot may be refilled
            const long long Bnext = to_fixed(Sb[bidx], fr.s);
            long long* Pk = &P[kk & 1][0][0];
#pragma unroll
            for (int f = 0; f < NFORM; ++f) {
                const int s = sidx[f];
                if ((f + 1) * NT <= NCELL || s >= 0) Pk[tid + f * NT] = to_fixed(Sx[s], fr.s);
            }
            __syncthreads();
            if (bad) {
                stop = true;
                return;
            }
            if (tid == 0 && t >= 1 && t - 1 + NS < nplanes) {
                issue(t - 1 + NS, slot == 0 ? NS - 1 : slot - 1);  // the slot of stage t-1
                issued_hi = t - 1 + NS;
            }
            {
                const long long(*Pp)[PX] = P[kk & 1];
                const long long c = Pp[ty + 1][tx + 1];
                cp.x = c;
                cp.f = (Pp[ty][tx + 1] + Pp[ty + 2][tx + 1]) + (Pp[ty + 1][tx] + Pp[ty + 1][tx + 2]);
                cp.d = (Pp[ty][tx] + Pp[ty][tx + 2]) + (Pp[ty + 2][tx] + Pp[ty + 2][tx + 2]);
            }
            if (t >= 2 && own) {
                const long long e2 = cm.f + cp.f + c0.d;
                const long long I = 3 * (2 * e2 + (cm.d + cp.d) - 32 * c0.x);
                const float ro = __ll2float_rn(Bcur - I) * fscale;
                r[o] = ro;
                rr.add_prod(ro, ro);
            }
            Bcur = Bnext;
            o += g.plane;
            if (++slot == NS) {
                slot = 0;
                phase ^= 1u;
            }
            if (++t >= nplanes) stop = true;
        };
        for (;;) {
            step(cA, cB, cC);
            if (stop) break;
            step(cB, cC, cA);
            if (stop) break;
            step(cC, cA, cB);
            if (stop) break;
        }
        if (bad) {
            // a copy never arrived: record it, finish the level, drain what is still in flight
            if (tid == 0) {
                st->status = 5;
                st->done = 1;
                if (ch.use) cudaGraphSetConditional(ch.loop, 0);
                for (int u = t_done; u <= issued_hi; ++u)
                    (void)mbar_wait(&bar[u % NS], (uint32_t)((u / NS) & 1));
            }
            return;
        }
    }

    // ||r||^2: compensated FP32 products, merged in FP32 pairs over the block and the grid
    // (block_merge; partials hold a float2 per double slot) and widened to FP64 once; r.z = D^-1 r.r
    CSum pr[1] = {rr.v};
    if (!fr.finite) pr[0] = CSum{(tid == 0 && first_block) ? __int_as_float(0x7fc00000) : 0.f, 0.f};  // NaN
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    float2* pp = reinterpret_cast<float2*>(partials);
    block_merge<1>(pr, red, red_out);
    if (tid == 0) {
        pp[bid] = red_out[0];
        __threadfence();
        ticket = atomicAdd(&st->arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return;
    __threadfence();
    pr[0] = CSum{0.f, 0.f};
    for (int b = tid; b < nb; b += NT) {
        const float2 p = __ldcg(&pp[b]);
        twosum_merge(pr[0].s, pr[0].c, p.x, p.y);
    }
    block_merge<1>(pr, red, red_out);
    if (tid == 0) {
        const double s = (double)red_out[0].x + (double)red_out[0].y;
        st->arrive = 0u;
        res_epilogue(st, s, (double)dd * s, mode, ch);
    }
}

bool make_map(CUtensorMap* map, const double* base, const Grid& g, int sx, int sy)
{
    return encode_level_map(map, true, base, g, sx, sy);
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// planes per block: about four blocks per SM (152 SMs), 2 .. KZ_MAX planes
inline int res_kz(const Grid& g)
{
    const int gxy = cdiv(max(g.nx - 1, 1), TBX) * cdiv(max(g.ny - 1, 1), TBY);
    const int gz = cdiv(152 * 4, gxy);
    return min(max(cdiv(max(g.nz - 1, 1), gz), 2), KZ_MAX);
}

}  // namespace

bool make_res_maps(ResMaps* m, const double* x, const double* bc, const Grid& g)
{
    return make_map(&m->x, x, g, SX, SY) && make_map(&m->bc, bc, g, EX, TBY);
}

cudaError_t res_cc_prepare()
{
    return cudaFuncSetAttribute(k_res_cc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
}

int res_cc_blocks(const Grid& g)
{
    return cdiv(max(g.nx - 1, 1), TBX) * cdiv(max(g.ny - 1, 1), TBY) * cdiv(max(g.nz - 1, 1), res_kz(g));
}

void launch_res32_cc(const ResMaps& m, const Grid& g, const int* uniform, const double* beta, const float* dinv32,
                     float* r, SolveState* st, Partials pr, ResMode mode, CondHandles ch, cudaStream_t s, float* r_b)
{
    const int kz = res_kz(g);
    const dim3 grid(cdiv(max(g.nx - 1, 1), TBX), cdiv(max(g.ny - 1, 1), TBY), cdiv(max(g.nz - 1, 1), kz));
    k_res_cc<<<grid, dim3(TBX, TBY), smem_bytes(), s>>>(m.x, m.bc, g, r, r_b, st, pr.buf, (int)mode, ch, kz, pr.fs,
                                                        uniform, beta, dinv32);
}

unsigned long long launches_res_cc()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
