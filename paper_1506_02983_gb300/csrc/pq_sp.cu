// pq_sp.cu -- the single-pass FP32 JCG step (ECMG_CG_SINGLE_PASS; body in k1_body.cuh): one
// kernel per step applies the previous step's residual update while staging r, forms p, applies
// the stencil and sums everything the recurrence needs, so the residual kernel of the two-pass
// form (one read of r and q and one write of r per node) is not run. Per node and step on a
// constant-coefficient level it moves r, q, p_old, e in and r, q, p, e out: 8 FP32 words
// against 9 for the two kernels of the two-pass form.
#include <cuda.h>

#include "k1_body.cuh"
#include "pq_tma.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

// General path: beta and D^-1 streamed with r, p_old and q_old.
template <bool ROBIN, bool CUBE, int RY>
__global__ void __launch_bounds__(NT, RY == 1 ? 3 : 2)
k_step32_tma(const __grid_constant__ CUtensorMap m_r, const __grid_constant__ CUtensorMap m_pold,
             const __grid_constant__ CUtensorMap m_dinv, const __grid_constant__ CUtensorMap m_beta,
             const __grid_constant__ CUtensorMap m_qold, const __grid_constant__ CUtensorMap m_e, const Grid g,
             const Op op, const Range rg, float* __restrict__ pnew, float* __restrict__ q, float* __restrict__ rnew,
             float* __restrict__ e, SolveState* st, double* partials, int pidx, CondHandles ch, int kz, KTimer* tm)
{
    COUNT_LAUNCH();
    const K1Scalars sc{st->done, (float)st->beta, (float)st->alpha_prev, 0.f, 0.f};
    k1_body<ROBIN, CUBE, RY, false, true>(m_r, m_pold, m_dinv, m_beta, m_qold, m_e, g, op, rg, pnew, q, rnew, e, st,
                                          partials, pidx, ch, kz, tm, sc, k1_block_of_grid());
}

// Constant-coefficient path (every face Dirichlet, one beta on the level); a stale host choice
// (the level's uniform flag clear when the kernel runs) is recorded as status 6, as in the
// two-pass kernel.
// With `pf` (buffer sets from the level state) the maps and pointers of both sets are given, the
// step reads set st->p_latest (the one the previous step or the residual wrote) and writes the
// other, and returns at once while a replacement is pending.
template <bool CUBE, int RY>
__global__ void __launch_bounds__(NT, RY == 1 ? (CUBE ? 6 : 5) : 4)
k_step32_cc(const __grid_constant__ CUtensorMap m_rA, const __grid_constant__ CUtensorMap m_pA,
            const __grid_constant__ CUtensorMap m_qA, const __grid_constant__ CUtensorMap m_rB,
            const __grid_constant__ CUtensorMap m_pB, const __grid_constant__ CUtensorMap m_qB,
            const __grid_constant__ CUtensorMap m_e, const Grid g, const Op op, const Range rg, const SpSets out,
            int in_b, int pf, float* __restrict__ e, SolveState* st, double* partials, CondHandles ch, int kz,
            KTimer* tm, const int* __restrict__ uniform, const float* __restrict__ beta32,
            const float* __restrict__ dinv32)
{
    COUNT_LAUNCH();
    const int uni = *uniform;
    const int in = pf ? st->p_latest : in_b;
    K1Scalars sc{st->done, (float)st->beta, (float)st->alpha_prev, dinv32[g.off(1, 1, 1)], beta32[g.off(0, 0, 0)]};
    sc.skip = pf ? st->need_update : 0;
    if (!uni) {
        if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) {
            if (!sc.done) {
                st->status = 6;
                st->done = 1;
            }
            if (ch.use) {
                cudaGraphSetConditional(ch.loop, 0);
                cudaGraphSetConditional(ch.update, 0);
            }
        }
        return;
    }
    const int o = in ^ 1;
    k1_body<false, CUBE, RY, true, true>(in ? m_rB : m_rA, in ? m_pB : m_pA, m_rA, m_rA, in ? m_qB : m_qA, m_e, g, op,
                                         rg, o ? out.p[1] : out.p[0], o ? out.q[1] : out.q[0],
                                         o ? out.r[1] : out.r[0], e, st, partials, o, ch, kz, tm, sc,
                                         k1_block_of_grid());
}

template <bool ROBIN, bool CUBE, int RY>
cudaError_t prepare_one()
{
    return cudaFuncSetAttribute(k_step32_tma<ROBIN, CUBE, RY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem<RY, false, true>());
}
template <bool CUBE, int RY>
cudaError_t prepare_cc()
{
    return cudaFuncSetAttribute(k_step32_cc<CUBE, RY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem<RY, true, true>());
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
void launch_ry(const PlaneMaps& m, int in_b, const K1Config& c, const Grid& g, const Op& op, bool cc,
               const int* uniform, const float* beta32, const float* dinv32, float* pnew, float* qnew, float* rnew,
               float* e, SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm, cudaStream_t s,
               const SpSets* sets)
{
    const int v = ry_index(RY);
    const Range rg = k1_range(g, op);
    const CUtensorMap& rin = in_b ? m.rB[v] : m.r[v];
    const CUtensorMap& qin = in_b ? m.qB[v] : m.qA[v];
    const CUtensorMap& pold = in_b ? m.pB[v] : m.pA[v];
    if (cc) {
        // the output set: either as given (pidx, the set written) or both sets for the state to pick
        SpSets out{};
        if (sets) {
            out = *sets;
        } else {
            out.p[pidx] = pnew;
            out.q[pidx] = qnew;
            out.r[pidx] = rnew;
        }
        auto kern = op.cube ? k_step32_cc<true, RY> : k_step32_cc<false, RY>;
        kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, true, true>(), s>>>(
            m.r[v], m.pA[v], m.qA[v], m.rB[v], m.pB[v], m.qB[v], m.e[v], g, op, rg, out, in_b, sets ? 1 : 0, e, st,
            pr.buf, ch, c.kz, tm, uniform, beta32, dinv32);
        return;
    }
    bool robin = false;
    for (int f = 0; f < 6; ++f) robin |= op.alpha[f] != 0.0;
    auto kern = robin ? (op.cube ? k_step32_tma<true, true, RY> : k_step32_tma<true, false, RY>)
                      : (op.cube ? k_step32_tma<false, true, RY> : k_step32_tma<false, false, RY>);
    kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, false, true>(), s>>>(
        rin, pold, m.dinv[v], m.beta[v], qin, m.e[v], g, op, rg, pnew, qnew, rnew, e, st, pr.buf, pidx, ch, c.kz, tm);
}

}  // namespace

cudaError_t k1_sp_prepare()
{
    cudaError_t e = prepare_ry<1>();
    if (e == cudaSuccess) e = prepare_ry<2>();
    return e;
}

void launch_step32(const PlaneMaps& m, int in_b, const K1Config& c, const Grid& g, const Op& op, bool cc,
                   const int* uniform, const float* beta32, const float* dinv32, float* pnew, float* qnew,
                   float* rnew, float* e, SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm,
                   cudaStream_t s, const SpSets* sets)
{
    if (c.ry == 1)
        launch_ry<1>(m, in_b, c, g, op, cc, uniform, beta32, dinv32, pnew, qnew, rnew, e, st, pr, pidx, ch, tm, s,
                     sets);
    else launch_ry<2>(m, in_b, c, g, op, cc, uniform, beta32, dinv32, pnew, qnew, rnew, e, st, pr, pidx, ch, tm, s,
                      sets);
}

unsigned long long launches_pq_sp()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
