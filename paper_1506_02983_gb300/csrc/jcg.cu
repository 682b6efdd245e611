// jcg.cu -- Jacobi-preconditioned CG of Alg. 4 (lines 7-9) on the matrix-free Q1 operator.
//
// One JCG iteration is two kernels:
//   K1 (k_pq):     p = D^-1 r + beta p_old, computed on the fly for a tile plus halo in shared
//                  memory; q = A p (27-point stencil, difference form); the iterate update
//                  x += alpha_prev p_old deferred from the previous iteration; p.q.
//   K2 (k_update): r -= alpha q; z = D^-1 r; r.z and r.r.
// The last block to finish each reducing kernel sums the per-block partials in a fixed order
// (deterministic) and advances the scalar recurrence in SolveState: alpha after K1, the
// stopping test of Alg. 4 line 7 and beta after K2. Inside a CUDA graph it also sets the
// condition of the level's WHILE node, so a level runs with no host round trip.
//
// The stencil: with S_d(i) the sum of beta over the elements that contain both node i and
// node i+d, and K(d) the beta=1 element matrix entry for that offset class,
//     (A v)_i = sum_{d != 0} K(d) S_d(i) (v_{i+d} - v_i) + Robin face terms,
// which holds because every element matrix has zero row sums (Sec. 2 bilinear form).
#include "jcg.cuh"

#include <cmath>

namespace ecmg {
namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

constexpr int BX = 32, BY = 8, NT = BX * BY;
constexpr int KZ_TARGET = 64;
constexpr int UPD_TPB = 256;
constexpr int UPD_MAX_BLOCKS = 152 * 8;

__device__ __forceinline__ bool on_dirichlet(const Grid& g, const Op& op, int i, int j, int k)
{
    return (i == 0 && op.bc[0] == 0) || (i == g.nx && op.bc[1] == 0) ||
           (j == 0 && op.bc[2] == 0) || (j == g.ny && op.bc[3] == 0) ||
           (k == 0 && op.bc[4] == 0) || (k == g.nz && op.bc[5] == 0);
}

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

// ---- block / grid reductions --------------------------------------------------------------
template <int NP>
__device__ __forceinline__ void block_sum(double (&v)[NP], double* sh)
{
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
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

// Sum v over the whole grid. Returns true in the last block to arrive, whose thread 0 then
// holds the totals in v; every other block returns false.
template <int NP>
__device__ __forceinline__ bool grid_sum(double (&v)[NP], double* partials, unsigned int* arrive)
{
    __shared__ double sh[NP * 32];
    __shared__ unsigned int ticket;
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_sum<NP>(v, sh);
    if (tid == 0) {
        for (int c = 0; c < NP; ++c) partials[bid * NP + c] = v[c];
        __threadfence();
        ticket = atomicAdd(arrive, 1u);
    }
    __syncthreads();
    if (ticket != (unsigned int)(nb - 1)) return false;
    __threadfence();
    for (int c = 0; c < NP; ++c) v[c] = 0.0;
    for (int b = tid; b < nb; b += nthr)
        for (int c = 0; c < NP; ++c) v[c] += __ldcg(&partials[b * NP + c]);
    block_sum<NP>(v, sh);
    if (tid == 0) *arrive = 0u;
    return tid == 0;
}

// ---- the tiled z-march -------------------------------------------------------------------
// Each block owns a BX x BY column of nodes over planes [kb, ke). Three node planes of the
// operand (k-1, k, k+1) and two element slabs of beta (k-1, k) live in shared memory; the
// operand of a plane is produced by src(offset), so K1 can form p on the fly.
template <typename VT, typename BT, typename SRC, typename BODY>
__device__ __forceinline__ void march(const Grid& g, const Op& op, const BT* __restrict__ beta,
                                      int kz, SRC src, BODY body)
{
    __shared__ VT sv[3][BY + 2][BX + 2];
    __shared__ VT sb[2][BY + 1][BX + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int kb = blockIdx.z * kz;
    const int ke = min(kb + kz, g.nz + 1);
    const VT wf0 = (VT)op.wf[0], wf1 = (VT)op.wf[1], wf2 = (VT)op.wf[2];
    const VT we0 = (VT)op.we[0], we1 = (VT)op.we[1], we2 = (VT)op.we[2], wc = (VT)op.wc;
    const bool any_robin = (op.alpha[0] != 0.0) | (op.alpha[1] != 0.0) | (op.alpha[2] != 0.0) |
                           (op.alpha[3] != 0.0) | (op.alpha[4] != 0.0) | (op.alpha[5] != 0.0);

    auto load_plane = [&](int k) {
        VT(*dst)[BX + 2] = sv[(k + 3) % 3];
        for (int c = tid; c < (BX + 2) * (BY + 2); c += NT) {
            const int ci = c % (BX + 2), cj = c / (BX + 2);
            const int i = i0 - 1 + ci, j = j0 - 1 + cj;
            VT v = VT(0);
            if (i <= g.nx + 1 && j <= g.ny + 1) v = src(g.off(i, j, k));
            dst[cj][ci] = v;
        }
    };
    auto load_slab = [&](int ez) {
        VT(*dst)[BX + 1] = sb[(ez + 2) % 2];
        for (int c = tid; c < (BX + 1) * (BY + 1); c += NT) {
            const int ci = c % (BX + 1), cj = c / (BX + 1);
            const int ex = i0 - 1 + ci, ey = j0 - 1 + cj;
            VT v = VT(0);
            if (ex <= g.nx + 1 && ey <= g.ny + 1) v = (VT)beta[g.off(ex, ey, ez)];
            dst[cj][ci] = v;
        }
    };

    load_plane(kb - 1);
    load_plane(kb);
    load_slab(kb - 1);
    for (int k = kb; k < ke; ++k) {
        load_plane(k + 1);
        load_slab(k);
        __syncthreads();
        const int i = i0 + tx, j = j0 + ty;
        if (i <= g.nx && j <= g.ny) {
            const int pl[3] = {(k + 2) % 3, k % 3, (k + 1) % 3};
            const int s0 = (k + 1) % 2, s1 = k % 2;
            auto V = [&](int dx, int dy, int dz) -> VT { return sv[pl[dz + 1]][ty + 1 + dy][tx + 1 + dx]; };
            const VT xc = V(0, 0, 0);
            // betas of the 8 elements around the node: b<ex><ey><ez>
            const VT b000 = sb[s0][ty][tx], b100 = sb[s0][ty][tx + 1];
            const VT b010 = sb[s0][ty + 1][tx], b110 = sb[s0][ty + 1][tx + 1];
            const VT b001 = sb[s1][ty][tx], b101 = sb[s1][ty][tx + 1];
            const VT b011 = sb[s1][ty + 1][tx], b111 = sb[s1][ty + 1][tx + 1];
            // pair sums over the axis the offset does not cross
            const VT sx00 = b000 + b100, sx01 = b010 + b110, sx10 = b001 + b101, sx11 = b011 + b111;  // [ez][ey]
            const VT sy00 = b000 + b010, sy01 = b100 + b110, sy10 = b001 + b011, sy11 = b101 + b111;  // [ez][ex]
            const VT sz00 = b000 + b001, sz01 = b100 + b101, sz10 = b010 + b011, sz11 = b110 + b111;  // [ey][ex]
            const VT fx = (sz01 + sz11) * (V(1, 0, 0) - xc) + (sz00 + sz10) * (V(-1, 0, 0) - xc);
            const VT fy = (sx01 + sx11) * (V(0, 1, 0) - xc) + (sx00 + sx10) * (V(0, -1, 0) - xc);
            const VT fz = (sx10 + sx11) * (V(0, 0, 1) - xc) + (sx00 + sx01) * (V(0, 0, -1) - xc);
            const VT ex = sx00 * (V(0, -1, -1) - xc) + sx01 * (V(0, 1, -1) - xc) +
                          sx10 * (V(0, -1, 1) - xc) + sx11 * (V(0, 1, 1) - xc);
            const VT ey = sy00 * (V(-1, 0, -1) - xc) + sy01 * (V(1, 0, -1) - xc) +
                          sy10 * (V(-1, 0, 1) - xc) + sy11 * (V(1, 0, 1) - xc);
            const VT ez = sz00 * (V(-1, -1, 0) - xc) + sz01 * (V(1, -1, 0) - xc) +
                          sz10 * (V(-1, 1, 0) - xc) + sz11 * (V(1, 1, 0) - xc);
            const VT cc = b000 * (V(-1, -1, -1) - xc) + b100 * (V(1, -1, -1) - xc) +
                          b010 * (V(-1, 1, -1) - xc) + b110 * (V(1, 1, -1) - xc) +
                          b001 * (V(-1, -1, 1) - xc) + b101 * (V(1, -1, 1) - xc) +
                          b011 * (V(-1, 1, 1) - xc) + b111 * (V(1, 1, 1) - xc);
            VT Av = wf0 * fx + wf1 * fy + wf2 * fz + we0 * ex + we1 * ey + we2 * ez + wc * cc;
            if (any_robin && (i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz)) {
                // alpha * (face mass matrix) on every Robin face through the node
                const int idx[3] = {i, j, k};
                const int nn[3] = {g.nx, g.ny, g.nz};
                for (int f = 0; f < 6; ++f) {
                    if (op.alpha[f] == 0.0) continue;
                    const int an = f / 2;
                    if (idx[an] != ((f & 1) ? nn[an] : 0)) continue;
                    const int aa = (an == 0) ? 1 : 0, ab = (an == 2) ? 1 : 2;
                    for (int db = -1; db <= 1; ++db)
                        for (int da = -1; da <= 1; ++da) {
                            const int ca = (da < 0) ? (idx[aa] >= 1) : (da > 0) ? (idx[aa] < nn[aa])
                                                                           : (idx[aa] >= 1) + (idx[aa] < nn[aa]);
                            const int cb = (db < 0) ? (idx[ab] >= 1) : (db > 0) ? (idx[ab] < nn[ab])
                                                                           : (idx[ab] >= 1) + (idx[ab] < nn[ab]);
                            if (!ca || !cb) continue;
                            const double w = op.alpha[f] * ca * g.h[aa] * (da ? 1.0 : 2.0) / 6.0 *
                                             cb * g.h[ab] * (db ? 1.0 : 2.0) / 6.0;
                            int o[3] = {0, 0, 0};
                            o[aa] = da;
                            o[ab] = db;
                            Av += (VT)w * V(o[0], o[1], o[2]);
                        }
                }
            }
            body(i, j, k, g.off(i, j, k), Av, xc);
        }
        __syncthreads();
    }
}

// ---- K1: search direction and operator ------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) k_pq(const Grid g, const Op op, const T* __restrict__ beta,
                                           const T* __restrict__ r, const T* __restrict__ dinv,
                                           const T* __restrict__ pold, T* __restrict__ pnew,
                                           T* __restrict__ q, T* __restrict__ x, SolveState* st,
                                           double* partials, int pidx, CondHandles ch, int kz)
{
    COUNT_LAUNCH();
    if (st->done) return;
    const T bcg = (T)st->beta;
    const T ap = (T)st->alpha_prev;
    Acc<T> acc;
    march<T, T>(
        g, op, beta, kz, [&](int64_t o) -> T { return dinv[o] * r[o] + bcg * pold[o]; },
        [&](int i, int j, int k, int64_t o, T Av, T pn) {
            const T qv = on_dirichlet(g, op, i, j, k) ? T(0) : Av;
            pnew[o] = pn;
            q[o] = qv;
            if (ap != T(0)) x[o] += ap * pold[o];
            acc.add_prod(pn, qv);
        });
    double v[1] = {acc.value()};
    if (grid_sum<1>(v, partials, &st->arrive)) {
        const double pq = v[0];
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
}

// ---- residual r = b - A x (FP64 arithmetic) -------------------------------------------------
__device__ void res_epilogue(SolveState* st, double rr, double rz, int mode, CondHandles ch)
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
        if (!isfinite(rr) || !isfinite(rz)) {
            st->status = 4;
            st->done = 1;
        } else if (rr <= st->thresh2) {
            st->rr = rr;
            st->done = 1;
        } else if (st->stop_after_update) {
            st->rr = rr;
            st->status = 3;
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

template <typename OT>
__global__ void __launch_bounds__(NT) k_res(const Grid g, const Op op, const double* __restrict__ beta,
                                            const double* __restrict__ x, const double* __restrict__ b,
                                            const OT* __restrict__ dinv, OT* __restrict__ r,
                                            SolveState* st, double* partials, int mode, CondHandles ch,
                                            int kz)
{
    COUNT_LAUNCH();
    if (mode == RES_REPLACE && st->done) return;
    double rr = 0.0, rz = 0.0;
    march<double, double>(
        g, op, beta, kz, [&](int64_t o) -> double { return x[o]; },
        [&](int i, int j, int k, int64_t o, double Av, double) {
            const double rv = on_dirichlet(g, op, i, j, k) ? 0.0 : b[o] - Av;
            const OT ro = (OT)rv;
            r[o] = ro;
            rr = fma(rv, rv, rr);
            const double rd = (double)ro;
            rz = fma(rd * (double)dinv[o], rd, rz);
        });
    double v[2] = {rr, rz};
    if (grid_sum<2>(v, partials, &st->arrive)) res_epilogue(st, v[0], v[1], mode, ch);
}

// ---- y = A x (full matrix, for operator checks) ---------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) k_apply(const Grid g, const Op op, const T* __restrict__ beta,
                                              const T* __restrict__ x, double* __restrict__ y, int kz)
{
    COUNT_LAUNCH();
    march<T, T>(
        g, op, beta, kz, [&](int64_t o) -> T { return x[o]; },
        [&](int, int, int, int64_t o, T Av, T) { y[o] = (double)Av; });
}

// ---- K2: residual update and stopping test ----------------------------------------------------
template <typename T, bool MIXED>
__global__ void __launch_bounds__(UPD_TPB) k_update(int64_t n, T* __restrict__ r, const T* __restrict__ q,
                                                    const T* __restrict__ dinv, SolveState* st,
                                                    double* partials, CondHandles ch)
{
    COUNT_LAUNCH();
    if (st->done) {
        if (ch.use && blockIdx.x == 0 && threadIdx.x == 0) {
            cudaGraphSetConditional(ch.loop, 0);
            if (MIXED) cudaGraphSetConditional(ch.update, 0);
        }
        return;
    }
    const T a = (T)st->alpha;
    Acc<T> rz, rr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride) {
        T rv = r[t] - a * q[t];
        r[t] = rv;
        const T zv = dinv[t] * rv;
        rz.add_prod(rv, zv);
        rr.add_prod(rv, rv);
    }
    double v[2] = {rz.value(), rr.value()};
    if (grid_sum<2>(v, partials, &st->arrive)) {
        const double rho_new = v[0], rrv = v[1];
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
                st->status = 3;
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
        if (ch.use) {
            cudaGraphSetConditional(ch.loop, st->done ? 0u : 1u);
            if (MIXED) cudaGraphSetConditional(ch.update, st->need_update ? 1u : 0u);
        }
    }
}

__global__ void k_final64(int64_t n, double* __restrict__ x, const double* __restrict__ pA,
                          const double* __restrict__ pB, const SolveState* st)
{
    COUNT_LAUNCH();
    const double a = st->alpha_prev;
    if (a == 0.0) return;
    const double* p = st->p_latest ? pB : pA;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride)
        x[t] = fma(a, p[t], x[t]);
}

__global__ void k_fold32(int64_t n, double* __restrict__ x, float* __restrict__ e,
                         const float* __restrict__ p, const SolveState* st)
{
    COUNT_LAUNCH();
    if (st->done) return;
    const double a = st->alpha_prev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride) {
        x[t] += (double)e[t] + a * (double)p[t];
        e[t] = 0.f;
    }
}

__global__ void k_state_init(SolveState* st, double rtol, double inner, int max_iters)
{
    COUNT_LAUNCH();
    SolveState s = {};
    s.rtol2 = rtol * rtol;
    s.inner2 = inner * inner;
    s.max_iters = max_iters;
    *st = s;
}

inline int stencil_kz(const Grid& g)
{
    const int gx = (g.nx + 1 + BX - 1) / BX, gy = (g.ny + 1 + BY - 1) / BY;
    const int want_blocks = 152 * 4;
    int gz = (want_blocks + gx * gy - 1) / (gx * gy);
    int kz = (g.nz + 1 + gz - 1) / gz;
    if (kz < 8) kz = 8;
    if (kz > KZ_TARGET) kz = KZ_TARGET;
    return kz;
}

inline dim3 stencil_grid(const Grid& g, int kz)
{
    return dim3((g.nx + 1 + BX - 1) / BX, (g.ny + 1 + BY - 1) / BY, (g.nz + 1 + kz - 1) / kz);
}

inline int update_blocks(int64_t n)
{
    int64_t b = (n + UPD_TPB * 4 - 1) / (UPD_TPB * 4);
    return (int)(b < UPD_MAX_BLOCKS ? (b > 0 ? b : 1) : UPD_MAX_BLOCKS);
}

}  // namespace

int max_stencil_blocks(const Grid& g)
{
    dim3 d = stencil_grid(g, stencil_kz(g));
    return (int)(d.x * d.y * d.z);
}
int max_stream_blocks() { return UPD_MAX_BLOCKS; }

void launch_pq64(const Grid& g, const Op& op, const double* beta, const double* r,
                 const double* dinv, const double* pold, double* pnew, double* q, double* x,
                 SolveState* st, Partials pr, int pidx, CondHandles ch, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    k_pq<double><<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, r, dinv, pold, pnew, q, x, st,
                                                            pr.buf, pidx, ch, kz);
}
void launch_pq32(const Grid& g, const Op& op, const float* beta, const float* r, const float* dinv,
                 const float* pold, float* pnew, float* q, float* e, SolveState* st, Partials pr,
                 int pidx, CondHandles ch, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    k_pq<float><<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, r, dinv, pold, pnew, q, e, st,
                                                           pr.buf, pidx, ch, kz);
}
void launch_res64(const Grid& g, const Op& op, const double* beta, const double* x, const double* b,
                  const double* dinv, double* r, SolveState* st, Partials pr, ResMode mode,
                  CondHandles ch, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    k_res<double><<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, x, b, dinv, r, st, pr.buf,
                                                             (int)mode, ch, kz);
}
void launch_res32(const Grid& g, const Op& op, const double* beta, const double* x, const double* b,
                  const float* dinv, float* r, SolveState* st, Partials pr, ResMode mode,
                  CondHandles ch, cudaStream_t s)
{
    const int kz = stencil_kz(g);
    k_res<float><<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, x, b, dinv, r, st, pr.buf,
                                                            (int)mode, ch, kz);
}
void launch_apply64(const Grid& g, const Op& op, const double* beta, const double* x, double* y,
                    cudaStream_t s)
{
    const int kz = stencil_kz(g);
    k_apply<double><<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, x, y, kz);
}
void launch_apply32(const Grid& g, const Op& op, const float* beta, const float* x, double* y,
                    cudaStream_t s)
{
    const int kz = stencil_kz(g);
    k_apply<float><<<stencil_grid(g, kz), dim3(BX, BY), 0, s>>>(g, op, beta, x, y, kz);
}
void launch_update64(const Grid& g, double* r, const double* q, const double* dinv, SolveState* st,
                     Partials pr, CondHandles ch, cudaStream_t s)
{
    k_update<double, false><<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, r, q, dinv, st, pr.buf, ch);
}
void launch_update32(const Grid& g, float* r, const float* q, const float* dinv, SolveState* st,
                     Partials pr, CondHandles ch, cudaStream_t s)
{
    k_update<float, true><<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, r, q, dinv, st, pr.buf, ch);
}
void launch_final64(const Grid& g, double* x, const double* pA, const double* pB, SolveState* st,
                    cudaStream_t s)
{
    k_final64<<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, x, pA, pB, st);
}
void launch_fold32(const Grid& g, double* x, float* e, const float* p, SolveState* st, cudaStream_t s)
{
    k_fold32<<<update_blocks(g.total), UPD_TPB, 0, s>>>(g.total, x, e, p, st);
}
void launch_state_init(SolveState* st, double rtol, double inner_rtol, int max_iters, cudaStream_t s)
{
    k_state_init<<<1, 1, 0, s>>>(st, rtol, inner_rtol, max_iters);
}

unsigned long long launches_jcg()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
