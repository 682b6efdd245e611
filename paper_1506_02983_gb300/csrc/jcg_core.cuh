// jcg_core.cuh -- device pieces of JCG (Alg. 4 lines 7-9) shared by the single-problem kernels
// (jcg.cu) and the batched ones (batch.cu): compensated FP32 sums and the scalar recurrence the
// last block of each reducing kernel advances.
#pragma once

#include "ecmg_internal.cuh"
#include "jcg.cuh"

namespace ecmg {

// ---- compensated FP32 accumulation ------------------------------------------------------
// Products are split exactly (TwoProduct with an FMA) and summed with TwoSum, so a thread's
// sum of FP32 products carries about 48 significant bits; the block and grid stages merge such
// pairs the same way (block_merge) and widen each total to FP64 once. Intrinsics keep the
// compiler from contracting the steps.
struct CSum {
    float s, c;
};
__device__ __forceinline__ void csum_add(CSum& a, float x)
{
    float t = __fadd_rn(a.s, x);
    float bp = __fsub_rn(t, a.s);
    float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, e);
}
__device__ __forceinline__ void csum_add_prod(CSum& a, float x, float y)
{
    float p = __fmul_rn(x, y);
    float e = __fmaf_rn(x, y, -p);
    csum_add(a, p);
    a.c = __fadd_rn(a.c, e);
}
__device__ __forceinline__ double csum_value(const CSum& a) { return (double)a.s + (double)a.c; }

// Merge the compensated pair (s2, c2) into (s, c): TwoSum of the leading parts, and the
// compensations and the rounding error of that sum added in FP32.
__device__ __forceinline__ void twosum_merge(float& s, float& c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, err));
}

// Block sums of NP compensated pairs (any type with float members s and c) of a 256-thread
// block, in FP32 arithmetic throughout: this part's FP64 pipe runs at a small fraction of its
// FP32 rate, and an FP64 tree here held every block for microseconds. The lanes of each warp
// merge their pairs by shuffles, then warp 0 merges the eight warps' pairs, eight lanes per sum.
// Sum c goes to out[c]; sh holds 8 NP pairs. Every thread may read out after the return.
template <int NP, typename P>
__device__ __forceinline__ void block_merge(P (&k)[NP], float2* sh, float2* out)
{
    constexpr int NW = 8;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int c = 0; c < NP; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, k[c].s, o);
            const float c2 = __shfl_down_sync(0xffffffffu, k[c].c, o);
            twosum_merge(k[c].s, k[c].c, s2, c2);
        }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NP; ++c) sh[c * NW + warp] = make_float2(k[c].s, k[c].c);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 4) {
            const int c = c0 + (lane >> 3);
            float ms = 0.f, mc = 0.f;
            if (c < NP) {
                const float2 p = sh[c * NW + (lane & 7)];
                ms = p.x;
                mc = p.y;
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                const float s2 = __shfl_down_sync(0xffffffffu, ms, o, 8);
                const float c2 = __shfl_down_sync(0xffffffffu, mc, o, 8);
                twosum_merge(ms, mc, s2, c2);
            }
            if ((lane & 7) == 0 && c < NP) out[c] = make_float2(ms, mc);
        }
    }
    __syncthreads();
}

// Accumulator selection: FP64 for FP64 data, compensated FP32 for FP32 data.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add_prod(double x, double y) { v = fma(x, y, v); }
    __device__ __forceinline__ double value() const { return v; }
};
template <> struct Acc<float> {
    CSum v{0.f, 0.f};
    __device__ __forceinline__ void add_prod(float x, float y) { csum_add_prod(v, x, y); }
    __device__ __forceinline__ double value() const { return csum_value(v); }
};

// What the last block of a residual evaluation does with ||r||^2 and r.z (ResMode).
__device__ __forceinline__ void res_epilogue(SolveState* st, double rr, double rz, int mode, CondHandles ch)
{
    switch (mode) {
    case RES_FH2:
        st->fh2 = rr;
        st->thresh2 = st->rtol2 * rr;
        break;
    case RES_INIT:
        st->rr = rr;
        st->rr_true = rr;
        st->rr_ref = rr;
        st->rho = rz;
        st->beta = 0.0;
        st->alpha_prev = 0.0;
        st->need_update = 0;
        if (st->pring) {  // the ring starts empty after the newest (zero) direction
            st->pbase = (st->pj + 1) % st->pring;
            st->pend = 0;
            st->espill = 0;
        }
        if (!isfinite(rr) || !isfinite(rz)) {
            st->status = 4;
            st->done = 1;
        } else if (rr <= st->thresh2) {
            st->done = 1;
        }
        if (ch.use) cudaGraphSetConditional(ch.loop, st->done ? 0u : 1u);
        break;
    case RES_REPLACE:
        st->updates += 1;
        st->rr_true = rr;
        st->alpha_prev = 0.0;
        st->need_update = 0;
        if (st->pring) {  // the fold before this residual added every pending direction and e
            st->pbase = (st->pj + 1) % st->pring;
            st->pend = 0;
            st->espill = 0;
        }
        if (!isfinite(rr) || !isfinite(rz)) {
            st->status = 4;
            st->done = 1;
        } else if (rr <= st->thresh2) {
            st->rr = rr;
            st->done = 1;
        } else if (st->stop_after_update) {
            st->rr = rr;
            st->status = st->fixed ? 0 : 3;  // the step count of a fixed schedule is the goal
            st->done = 1;
        } else {
            st->beta = rz / st->rho;
            st->rho = rz;
            st->rr = rr;
            st->rr_ref = rr;
        }
        break;
    default:
        st->rr_true = rr;
        break;
    }
}

// After K2 (r -= alpha q, rho_new = r.z, rrv = r.r): iteration count, stopping test (FP64) or
// replacement request (MIXED: FP32 inner reduction reached, tolerance reached, or the cap).
template <bool MIXED>
__device__ __forceinline__ void update_epilogue(SolveState* st, double rho_new, double rrv)
{
    st->iters += 1;
    st->alpha_prev = st->alpha;
    st->rr = rrv;
    if (!isfinite(rho_new) || !isfinite(rrv)) {
        st->status = 4;
        st->done = 1;
    } else if (!MIXED) {
        if (rrv <= st->thresh2) {
            st->done = 1;
        } else if (st->iters >= st->max_iters) {
            st->status = st->fixed ? 0 : 3;  // the step count of a fixed schedule is the goal
            st->done = 1;
        } else {
            st->beta = rho_new / st->rho;
            st->rho = rho_new;
        }
    } else {
        if (rrv <= st->thresh2 || rrv <= st->inner2 * st->rr_ref) {
            st->need_update = 1;
        } else if (st->iters >= st->max_iters) {
            st->need_update = 1;
            st->stop_after_update = 1;
        } else {
            st->beta = rho_new / st->rho;
            st->rho = rho_new;
        }
    }
}

// After K1 (p.q): the step alpha, or breakdown when p.q is not positive and finite.
__device__ __forceinline__ void pq_epilogue(SolveState* st, double pq, int pidx, CondHandles ch)
{
    st->alpha_prev = 0.0;  // applied by every block above
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

}  // namespace ecmg
