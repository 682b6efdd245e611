// jcg_core.cuh -- device pieces of JCG (Alg. 4 lines 7-9) shared by the single-problem kernels
// (jcg.cu) and the batched ones (batch.cu): compensated FP32 sums and the scalar recurrence the
// last block of each reducing kernel advances.
#pragma once

#include "ecmg_internal.cuh"
#include "jcg.cuh"

namespace ecmg {

// ---- compensated FP32 accumulation ------------------------------------------------------
// Products are split exactly (TwoProduct with an FMA) and summed with TwoSum, so a thread's
// sum of FP32 products carries about 48 significant bits before it is promoted to FP64 for
// the block and grid stages. Intrinsics keep the compiler from contracting the steps.
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
