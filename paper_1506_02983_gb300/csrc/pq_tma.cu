// pq_tma.cu -- K1 of the FP32 JCG iteration with TMA-staged planes.
//
// Per block: a TBX x TBY column of nodes over a range of planes. A 4-stage ring of shared
// memory buffers receives, for every node plane k, boxes of r, p_old, D^-1 (plane k) and beta
// (element slab k-1) by cp.async.bulk.tensor, each stage completing on its own mbarrier.
// One elected thread issues the copies NSTAGE planes ahead, so HBM latency is hidden behind
// the stencil of the current plane. For each staged plane the block forms the new search
// direction p = D^-1 r + beta p_old once per node (tile plus halo) into a small plane buffer;
// every thread then keeps a 3x3x3 window of p and the 2x2x2 element betas of its node in
// registers while marching in z, so the 27-point stencil reads only 9 new values of p and 4
// new betas per node from shared memory.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records ECMG status 5 in the
// level state, finishes the level, waits (bounded) for its own copies still in flight and
// returns.
#include <cuda.h>

#include "jcg.cuh"
#include "pq_tma.cuh"
#include "stencil_core.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int TBX = 32, TBY = 8, NT = TBX * TBY;
constexpr int SX = 40, SY = 10;            // staged box: columns from node i0-4, rows from j0-1
constexpr int BOXF = SX * SY;              // floats per staged vector
constexpr int BOXF_PAD = 416;              // 1664 B: keeps every TMA destination 128 B aligned
constexpr int NSTAGE = 4;
constexpr int PX = TBX + 2, PY = TBY + 2;  // formed plane of p: tile plus one-node halo
constexpr uint32_t STAGE_BYTES = 4u * BOXF * sizeof(float);
constexpr long long WAIT_LIMIT = 1ll << 22; // polls before a wait is declared lost
constexpr int KZ_TARGET = 64;

struct __align__(128) Stage {
    float r[BOXF_PAD];
    float pold[BOXF_PAD];
    float dinv[BOXF_PAD];
    float beta[BOXF_PAD];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (long long it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
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

template <bool ROBIN, bool CUBE>
__global__ void __launch_bounds__(NT, ROBIN ? 3 : 4)
k_pq32_tma(const __grid_constant__ CUtensorMap m_r, const __grid_constant__ CUtensorMap m_pold,
           const __grid_constant__ CUtensorMap m_dinv, const __grid_constant__ CUtensorMap m_beta,
           const Grid g, const Op op, float* __restrict__ pnew, float* __restrict__ q,
           float* __restrict__ e, SolveState* st, double* partials, int pidx, CondHandles ch, int kz)
{
    COUNT_LAUNCH();
    __shared__ Stage stage[NSTAGE];
    __shared__ float P[2][PY][PX];
    __shared__ __align__(8) uint64_t bar[NSTAGE];
    __shared__ double red[32];
    __shared__ int bad;
    __shared__ int issued_hi;              // highest staged plane index issued so far
    __shared__ unsigned int ticket;

    if (st->done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TBX * ty;
    const int i0 = blockIdx.x * TBX, j0 = blockIdx.y * TBY;
    const int kb = blockIdx.z * kz;
    const int ke = min(kb + kz, g.nz + 1);
    const int P0 = kb - 1;                 // first staged node plane
    const int nplanes = ke - kb + 2;       // planes kb-1 .. ke
    const float bcg = (float)st->beta;
    const float ap = (float)st->alpha_prev;

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
    }
    __syncthreads();

    // Stage t holds node plane P0+t (memory plane P0+t+1) and element slab P0+t-1 (memory
    // plane P0+t). Column i0 of the padded layout is node i0-4, row j0 is node j0-1.
    auto issue = [&](int t) {
        Stage& S = stage[t % NSTAGE];
        uint64_t* b = &bar[t % NSTAGE];
        const int kk = P0 + t;
        mbar_expect_tx(b, STAGE_BYTES);
        tma_load_3d(S.r, &m_r, i0, j0, kk + 1, b);
        tma_load_3d(S.pold, &m_pold, i0, j0, kk + 1, b);
        tma_load_3d(S.dinv, &m_dinv, i0, j0, kk + 1, b);
        tma_load_3d(S.beta, &m_beta, i0, j0, kk, b);
    };
    if (tid == 0) {
        for (int t = 0; t < NSTAGE && t < nplanes; ++t) issue(t);
        issued_hi = min(NSTAGE, nplanes) - 1;
    }

    const int i = i0 + tx, j = j0 + ty;
    const bool owned = (i <= g.nx) && (j <= g.ny);
    const Weights<float> wts(op);

    // offset of this thread's node on the plane computed next (plane kb at step t = 2)
    int64_t o = g.plane_base(P0 - 1) + g.in_plane(min(i, g.nx + 1), min(j, g.ny + 1));
    // the cells this thread forms in every plane (PX*PY = 340 cells, at most 2 per thread)
    const int c1 = tid + NT;
    const bool has1 = c1 < PX * PY;
    const int sidx0 = (tid / PX) * SX + (tid % PX) + 3;
    const int sidx1 = has1 ? (c1 / PX) * SX + (c1 % PX) + 3 : 0;
    // the i, j part of the Dirichlet test is fixed for the thread's column
    const bool dir_ij = (i == 0 && op.bc[0] == 0) || (i == g.nx && op.bc[1] == 0) ||
                        (j == 0 && op.bc[2] == 0) || (j == g.ny && op.bc[3] == 0);
    const bool dir_k0 = op.bc[4] == 0, dir_kn = op.bc[5] == 0;

    float wA[3][3], wB[3][3], wC[3][3];  // three planes of the p window, [y][x]
    float bA[2][2], bB[2][2];            // element betas of two slabs, [ey][ex]
    float pown_prev = 0.f;               // p_old of this thread's node, plane k
    float e_cur = 0.f;
    CSum acc;
    int t_done = -1;                     // last stage waited for
    int t = 0;
    bool stop = false;

    // One plane: stage t brings node plane kk = P0 + t into wp and beta slab kk-1 into bn;
    // then node plane kk-1 is computed from the window (wm, w0, wp) = planes (kk-2, kk-1, kk)
    // and the slabs (bo, bn) = (kk-2, kk-1). The caller rotates the arrays instead of moving
    // values, so the unrolled loop below needs no register copies.
    auto step = [&](float(&wm)[3][3], float(&w0)[3][3], float(&wp)[3][3], float(&bo)[2][2], float(&bn)[2][2]) {
        const int kk = P0 + t;
        Stage& S = stage[t % NSTAGE];
        // prefetch e of the node computed at the next step (plane kk), one step ahead
        float e_next = 0.f;
        if (ap != 0.f && owned && t >= 1) e_next = e[o + g.plane];
        if (!mbar_wait(&bar[t % NSTAGE], (uint32_t)((t / NSTAGE) & 1))) bad = 1;
        t_done = t;
        // form p of plane kk for the tile plus halo (stage column = node column - (i0 - 4))
        float* Pk = &P[kk & 1][0][0];
        Pk[tid] = fmaf(S.dinv[sidx0], S.r[sidx0], bcg * S.pold[sidx0]);
        if (has1) Pk[c1] = fmaf(S.dinv[sidx1], S.r[sidx1], bcg * S.pold[sidx1]);
        const float pown_new = S.pold[(ty + 1) * SX + tx + 4];
        __syncthreads();
        if (bad) {
            stop = true;
            return;
        }
        if (tid == 0 && t >= 1 && t - 1 + NSTAGE < nplanes) {
            issue(t - 1 + NSTAGE);
            issued_hi = t - 1 + NSTAGE;
        }
        const float(*Pp)[PX] = P[kk & 1];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) wp[dy][dx] = Pp[ty + dy][tx + dx];
#pragma unroll
        for (int ey = 0; ey < 2; ++ey)
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) bn[ey][ex] = S.beta[(ty + ey) * SX + tx + 3 + ex];

        if (t >= 2 && owned) {
            const int k = kk - 1;
            const float xc = w0[1][1];
            auto V = [&](int dx, int dy, int dz) -> float {
                return dz < 0 ? wm[dy + 1][dx + 1] : (dz > 0 ? wp[dy + 1][dx + 1] : w0[dy + 1][dx + 1]);
            };
            const float Av = q1_apply<false, ROBIN, CUBE, float>(V, bo[0][0], bo[0][1], bo[1][0], bo[1][1], bn[0][0],
                                                                 bn[0][1], bn[1][0], bn[1][1], i, j, k, g, op, wts);
            const bool dir = dir_ij || (k == 0 && dir_k0) || (k == g.nz && dir_kn);
            const float qv = dir ? 0.f : Av;
            pnew[o] = xc;
            q[o] = qv;
            if (ap != 0.f) e[o] = fmaf(ap, pown_prev, e_cur);
            acc.add_prod(xc, qv);
        }
        pown_prev = pown_new;
        e_cur = e_next;
        o += g.plane;
        if (++t >= nplanes) stop = true;
    };
    // period 6 = lcm(3 window planes, 2 beta slabs)
    for (;;) {
        step(wA, wB, wC, bA, bB);
        if (stop) break;
        step(wB, wC, wA, bB, bA);
        if (stop) break;
        step(wC, wA, wB, bA, bB);
        if (stop) break;
        step(wA, wB, wC, bB, bA);
        if (stop) break;
        step(wB, wC, wA, bA, bB);
        if (stop) break;
        step(wC, wA, wB, bB, bA);
        if (stop) break;
    }

    if (bad) {
        // a copy never arrived: record it, finish the level, drain what is still in flight
        if (tid == 0) {
            st->status = 5;
            st->done = 1;
            for (int t = t_done; t <= issued_hi; ++t)
                (void)mbar_wait(&bar[t % NSTAGE], (uint32_t)((t / NSTAGE) & 1));
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

inline int tma_kz(const Grid& g)
{
    const int gx = (g.nx + 1 + TBX - 1) / TBX, gy = (g.ny + 1 + TBY - 1) / TBY;
    int gz = (152 * 3 + gx * gy - 1) / (gx * gy);
    int kz = (g.nz + 1 + gz - 1) / gz;
    if (kz < 8) kz = 8;
    if (kz > KZ_TARGET) kz = KZ_TARGET;
    return kz;
}

inline dim3 tma_grid(const Grid& g, int kz)
{
    return dim3((g.nx + 1 + TBX - 1) / TBX, (g.ny + 1 + TBY - 1) / TBY, (g.nz + 1 + kz - 1) / kz);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace

bool make_plane_map(CUtensorMap* map, const float* base, const Grid& g)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 3), (cuuint64_t)(g.nz + 3)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    const cuuint32_t box[3] = {SX, SY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int max_tma_blocks(const Grid& g)
{
    const dim3 d = tma_grid(g, tma_kz(g));
    return (int)(d.x * d.y * d.z);
}

void launch_pq32_tma(const PlaneMaps& m, int pold_is_b, const Grid& g, const Op& op, float* pnew, float* q,
                     float* e, SolveState* st, Partials pr, int pidx, CondHandles ch, cudaStream_t s)
{
    const int kz = tma_kz(g);
    bool robin = false;
    for (int f = 0; f < 6; ++f) robin |= op.alpha[f] != 0.0;
    (robin ? (op.cube ? k_pq32_tma<true, true> : k_pq32_tma<true, false>)
           : (op.cube ? k_pq32_tma<false, true> : k_pq32_tma<false, false>))<<<tma_grid(g, kz), dim3(TBX, TBY), 0, s>>>(m.r, pold_is_b ? m.pB : m.pA, m.dinv, m.beta, g, op, pnew,
                                                        q, e, st, pr.buf, pidx, ch, kz);
}

unsigned long long launches_pq_tma()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
