// pq_tma.cu -- K1 of the two-pass FP32 JCG step (the body is k1_body.cuh): p = D^-1 r +
// beta p_old, q = A p, the deferred iterate update and p.q; also the tensor maps, the tile
// heuristics and candidates shared with the single-pass kernels (pq_sp.cu).
#include <cuda.h>

#include "k1_body.cuh"
#include "pq_tma.cuh"

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

// With a ring of search directions (ring.base not null; m_pold is then the ring's 4D map): p_old
// from slot st->pj, p into the next slot, no deferred correction (ap = 0: e is neither read nor
// written; K2 and the fold of a replacement add the pending alpha p from the ring).
__device__ __forceinline__ float* ring_scalars(K1Scalars& sc, float* pnew, const SolveState* st, const Grid& g,
                                               const RingArgs& ring)
{
    if (!ring.base) return pnew;
    sc.pw = st->pj;
    sc.ap = 0.f;
    return ring.base + (int64_t)((sc.pw + 1) % ring.R) * ring_stride(g.total);
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
    k1_body<ROBIN, CUBE, RY, false, false>(m_r, m_pold, m_dinv, m_beta, m_r, m_e, g, op, rg, pnew, q, nullptr, e, st,
                                           partials, pidx, ch, kz, tm, sc, k1_block_of_grid());
}

// Constant-coefficient path (every face Dirichlet, one beta on the level): r, p_old and e only,
// and about half the registers of the general path, so six blocks fit on an SM instead of four
// (one node row per thread; four blocks with two rows, which an autotuned 512^3 level
// prefers). The host picks it from the level's uniform flag after the set-up; should a later
// set-up clear the flag (new beta data under a recorded graph), the kernel computes nothing
// and records status 6 so that the host records the solve again with the general path.
// RING: the ring form (p_old from the ring, no e): its stages hold no e box, so on cubic elements
// five blocks of two-row tiles fit an SM by shared memory and by registers.
template <bool CUBE, int RY, bool RING>
__global__ void __launch_bounds__(NT, RY == 1 ? 6 : (RING && CUBE ? 5 : 4))
k_pq32_cc(const __grid_constant__ CUtensorMap m_r, const __grid_constant__ CUtensorMap m_pold,
          const __grid_constant__ CUtensorMap m_e, const Grid g, const Op op, const Range rg,
          float* __restrict__ pnew, float* __restrict__ q, float* __restrict__ e, SolveState* st, double* partials,
          int pidx, CondHandles ch, int kz, KTimer* tm, const int* __restrict__ uniform,
          const float* __restrict__ beta32, const float* __restrict__ dinv32, const RingArgs ring)
{
    COUNT_LAUNCH();
    const int uni = *uniform;
    // ring form: a step behind one that asked for a replacement does nothing until it has run
    K1Scalars sc{RING ? (st->done | st->need_update) : st->done, (float)st->beta, (float)st->alpha_prev,
                 dinv32[g.off(1, 1, 1)], beta32[g.off(0, 0, 0)]};
    pnew = ring_scalars(sc, pnew, st, g, ring);
    if (!uni) {
        if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0 && !sc.done) {
            st->status = 6;
            st->done = 1;
            if (ch.use) cudaGraphSetConditional(ch.loop, 0);
        }
        return;
    }
    k1_body<false, CUBE, RY, true, false, RING>(m_r, m_pold, m_r, m_r, m_r, m_e, g, op, rg, pnew, q, nullptr, e, st,
                                                partials, pidx, ch, kz, tm, sc, k1_block_of_grid(), ring.alpha, ring.R);
}

bool make_plane_map(CUtensorMap* map, const float* base, const Grid& g, int sy, int sx = SX)
{
    return encode_level_map(map, false, base, g, sx, sy);
}

template <bool ROBIN, bool CUBE, int RY>
cudaError_t prepare_one()
{
    return cudaFuncSetAttribute(k_pq32_tma<ROBIN, CUBE, RY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_smem<RY, false, false>());
}
template <bool CUBE, int RY>
cudaError_t prepare_cc()
{
    cudaError_t e = cudaFuncSetAttribute(k_pq32_cc<CUBE, RY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stage_smem<RY, true, false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pq32_cc<CUBE, RY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stage_smem<RY, true, false, true>());
    return e;
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
               SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm, cudaStream_t s,
               const RingArgs* ring)
{
    const int v = ry_index(RY);
    const Range rg = k1_range(g, op);
    const CUtensorMap& pold = pold_is_b ? m.pB[v] : m.pA[v];
    if (cc) {
        if (ring) {
            auto kern = op.cube ? k_pq32_cc<true, RY, true> : k_pq32_cc<false, RY, true>;
            kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, true, false, true>(), s>>>(
                m.r[v], m.ring[v], m.e[v], g, op, rg, pnew, q, e, st, pr.buf, pidx, ch, c.kz, tm, uniform, beta32,
                dinv32, *ring);
        } else {
            auto kern = op.cube ? k_pq32_cc<true, RY, false> : k_pq32_cc<false, RY, false>;
            kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, true, false>(), s>>>(
                m.r[v], pold, m.e[v], g, op, rg, pnew, q, e, st, pr.buf, pidx, ch, c.kz, tm, uniform, beta32, dinv32,
                RingArgs{nullptr, nullptr, 0});
        }
        return;
    }
    bool robin = false;
    for (int f = 0; f < 6; ++f) robin |= op.alpha[f] != 0.0;
    auto kern = robin ? (op.cube ? k_pq32_tma<true, true, RY> : k_pq32_tma<true, false, RY>)
                      : (op.cube ? k_pq32_tma<false, true, RY> : k_pq32_tma<false, false, RY>);
    kern<<<k1_grid(rg, c), dim3(TBX, TBY), stage_smem<RY, false, false>(), s>>>(
        m.r[v], pold, m.dinv[v], m.beta[v], m.e[v], g, op, rg, pnew, q, e, st, pr.buf, pidx, ch, c.kz, tm);
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

bool make_ring_maps(PlaneMaps* m, const float* ring, int R, const Grid& g)
{
    for (int v = 0; v < K1_NRY; ++v)
        if (!encode_ring_map(&m->ring[v], ring, g, R, SX, TBY * K1_RY[v] + 2)) return false;
    return true;
}

bool make_plane_maps_sp(PlaneMaps* m, const float* rB, const float* qA, const float* qB, const Grid& g)
{
    for (int v = 0; v < K1_NRY; ++v) {
        const int sy = TBY * K1_RY[v] + 2;
        if (!make_plane_map(&m->rB[v], rB, g, sy) || !make_plane_map(&m->qA[v], qA, g, sy) ||
            !make_plane_map(&m->qB[v], qB, g, sy))
            return false;
    }
    return true;
}

cudaError_t k1_prepare()
{
    cudaError_t e = prepare_ry<1>();
    if (e == cudaSuccess) e = prepare_ry<2>();
    if (e == cudaSuccess) e = k1_sp_prepare();
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
    constexpr int NKZ = 13;
    const int kzs[NKZ] = {4, 6, 8, 10, 12, 14, 16, 20, 24, 32, 48, 64, 128};
    int n = 0;
    for (int v = 0; v < K1_NRY; ++v)
        for (int z = 0; z < NKZ; ++z)
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
                     SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm, cudaStream_t s,
                     const RingArgs* ring)
{
    if (c.ry == 1)
        launch_ry<1>(m, pold_is_b, c, g, op, cc, uniform, beta32, dinv32, pnew, q, e, st, pr, pidx, ch, tm, s, ring);
    else launch_ry<2>(m, pold_is_b, c, g, op, cc, uniform, beta32, dinv32, pnew, q, e, st, pr, pidx, ch, tm, s, ring);
}

unsigned long long launches_pq_tma()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
