// jcg.cuh -- host-side launch interface of the JCG kernels (jcg.cu).
#pragma once

#include "ecmg_internal.cuh"

namespace ecmg {

// What the last block of a residual evaluation does with ||r||^2 and r.z.
enum ResMode : int {
    RES_FH2 = 0,      // store ||f_h||^2 (x = Dirichlet extension) and the stopping threshold
    RES_INIT = 1,     // initial residual of a level: start JCG (or finish with 0 iterations)
    RES_REPLACE = 2,  // MIXED: FP64 residual replacement after folding the FP32 correction
    RES_REPORT = 3    // report the true residual after JCG has stopped
};

struct CondHandles {
    cudaGraphConditionalHandle loop;   // WHILE node of the level's JCG loop
    cudaGraphConditionalHandle update; // MIXED: IF node of the residual replacement
    int use;                           // 0 when the kernels run outside a graph
};

// Tiled z-marching stencil launches. uniform: device flag of the level (1 = one beta
// everywhere, which selects the tensor-product evaluation in FP64), or nullptr.
// p_new = dinv r + beta p_old on the fly; q = A p_new; x += alpha_prev p_old; state.alpha.
void launch_pq64(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* r,
                 const double* dinv, const double* pold, double* pnew, double* q, double* x,
                 SolveState* st, Partials pr, int pnew_index, CondHandles ch, cudaStream_t s);
// r = b - A x on free nodes, 0 on Dirichlet nodes; r stored as double or float; ||r||^2 and
// r.dinv.r reduced; last block acts by ResMode. A x exactly in fixed point on a level with one
// beta, in fixed point up to the beta products with variable beta on cubic elements without
// Robin terms (march_fx.cuh), else in FP64 arithmetic (two launches: max |x|, then the residual).
void launch_res64(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* x,
                  const double* b, const double* dinv, double* r, SolveState* st, Partials pr,
                  ResMode mode, CondHandles ch, cudaStream_t s);
// bc: b / c from launch_fh2 (same level), or null. On a constant-coefficient level (one beta,
// every face Dirichlet, cubic elements) the residual is then exact in 64-bit integers.
void launch_res32(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* x,
                  const double* b, const float* dinv, float* r, SolveState* st, Partials pr,
                  ResMode mode, CondHandles ch, cudaStream_t s, const double* bc = nullptr);
// max |x| over the level vector into pr.fs (the fixed-point scale of the exact residual) when the
// level's uniform flag is set, or always with `always` (variable beta on cubic elements without
// Robin terms); skipped for a replacement (mode RES_REPLACE) of a finished level.
void launch_absmax(const Grid& g, const double* x, const int* uniform, const SolveState* st, int mode,
                   Partials pr, cudaStream_t s, bool always = false);
// y = A x with the full matrix (no boundary masking), FP64 or FP32 arithmetic.
void launch_apply64(const Grid& g, const Op& op, const double* beta, const int* uniform, const double* x,
                    double* y, Partials pr, cudaStream_t s);
void launch_apply32(const Grid& g, const Op& op, const float* beta, const float* x, double* y,
                    cudaStream_t s);

// ||f_h||^2 into the level state (x = Dirichlet extension), and the stopping threshold. On a
// MIXED level (uniform: the level's flag, bc: a level vector, else both null) that turns out to
// be a constant-coefficient one (one beta, every face Dirichlet, cubic elements), also
// bc = b / c (c = -beta h / 36) on the free nodes and max |bc| into st->bcbits: the exact
// residual's load and scale.
// max_blocks: a cap on the grid (0: the usual streaming grid); the pass strides over any grid.
void launch_fh2(const Grid& g, const Op& op, const double* beta, const double* x, const double* b, SolveState* st,
                Partials pr, cudaStream_t s, const int* uniform = nullptr, double* bc = nullptr, int max_blocks = 0);
// r -= alpha q; z = dinv r; r.z and r.r; last block: convergence / next beta.
void launch_update64(const Grid& g, double* r, const double* q, const double* dinv,
                     SolveState* st, Partials pr, CondHandles ch, cudaStream_t s);
// uniform: the level's device flag; with every face Dirichlet and the flag set, D^-1 is one
// constant on the free nodes and is not streamed. ring: the level's ring of search directions
// (or nullptr); when it is full this step also adds the pending alpha p to the correction vector e.
void launch_update32(const Grid& g, const Op& op, const int* uniform, float* r, const float* q, const float* dinv,
                     SolveState* st, Partials pr, CondHandles ch, cudaStream_t s, const RingArgs* ring = nullptr,
                     float* e = nullptr);

// x += alpha_prev p_latest (FP64 JCG exit).
void launch_final64(const Grid& g, double* x, const double* pA, const double* pB,
                    SolveState* st, cudaStream_t s);
// MIXED: x64 += e + alpha_prev p (combined in FP32, added in FP64); e = 0. With the level's
// uniform flag set, also max |x| of the new iterate into pr.fs (what launch_absmax computes).
// p_b: with the single-pass buffer pairs taken from the level state, the other p of the pair; the
// fold then takes the newest one (st->p_latest).
void launch_fold32(const Grid& g, double* x, float* e, const float* p, const int* uniform, SolveState* st,
                   Partials pr, cudaStream_t s, const float* p_b = nullptr);
// Reset the level state before a solve; fixed: run exactly max_iters steps (Alg. 3); pring: the
// slots of the level's ring of search directions (0: none).
void launch_state_init(SolveState* st, double rtol, double inner_rtol, int max_iters, int fixed,
                       cudaStream_t s, int pring = 0);
// MIXED with a ring of search directions: x64 += e + the pending alpha p (FP32 sum, one FP64 add;
// e only when a full ring was added to it, and then e = 0); with the level's uniform flag set,
// also max |x| of the new iterate into pr.fs.
void launch_fold_ring(const Grid& g, double* x, const RingArgs& ring, float* e, const int* uniform, SolveState* st,
                      Partials pr, cudaStream_t s);

int max_stencil_blocks(const Grid& g);
int max_stream_blocks();

}  // namespace ecmg
