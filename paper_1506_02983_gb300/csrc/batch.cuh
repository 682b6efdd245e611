// batch.cuh -- many independent problems in one launch per step (batch.cu).
//
// A batched solve runs Alg. 4 for every problem of the batch side by side. Levels are aligned
// at the finest: at stage s, a problem with L levels of a batch whose deepest problem has Lmax
// works on its level s - (Lmax - L), so every problem finishes its finest level at the last
// stage. Each step of a stage (state set-up, EXP_finite, the FP64 residual, one FP32 JCG
// iteration, the residual replacement, EXP_true) is ONE kernel launch over the blocks of all
// problems that take part; a block finds its (problem, level) item from the launch's block
// offsets and works on that item's grid alone. Reductions are per item (the item's last block
// advances that item's JCG recurrence); the kernels that steer the loop also count every block
// of the launch, and the launch's last block sets the CUDA-graph conditions from all items:
// keep looping while any item runs, replace residuals where any item asks for it.
#pragma once

#include "ecmg_internal.cuh"
#include "jcg.cuh"
#include "pq_tma.cuh"

namespace ecmg {

constexpr int BATCH_MAX = 128;  // problems per batch

// One (problem, level) of a batch.
struct BItem {
    Grid g;
    Op op;
    Grid g1, g0;          // levels l-1 and l-2 (EXP)
    Grid gf;              // level l+1 (set-up of a coarser level)
    int level, problem, depth, fmode;  // depth 0 = the problem's finest level
    // depth 0 of a problem with compact inputs: beta, the load b and g_D already assembled on the
    // device from them (separable f or g_D, one beta) before the batched set-up, which keeps them
    int pre_beta, pre_load, pre_gD;
    int kz;               // z-march depth of the register-prefetched stencil kernels
    int k1kz;             // planes per block of the TMA-staged FP32 stencil kernel (K1)
    double rtol;          // relative residual tolerance of this level
    int max_iters;        // step cap (the exact step count when fixed)
    int fixed;            // 1: exactly max_iters steps (the schedule of Alg. 3)
    int precond;          // 1: Jacobi (ECMG_jcg), 0: plain CG (ECMG_cg)
    // vectors of this level (padded layout)
    double *U, *W, *Ut, *b, *beta, *f, *gD, *gR;
    float *beta32, *dinv32, *r32, *pA32, *pB32, *q32, *e32;
    float *r32B, *q32B;   // single-pass step: the second residual and q buffers
    // solutions of levels l-1, l-2 (EXP)
    const double *U1, *U0;
    // level l+1 vectors (set-up of a coarser level)
    const double *fbeta, *ff, *fgD, *fgR, *fb;
    // the caller's finest arrays (dense layout; depth 0 only; gD, gR may be null)
    const double *in_beta, *in_f, *in_gD, *in_gR;
    SolveState* st;
    double* part;         // per-block partial sums of this item's reductions
};

// Blocks of one batched launch: slot s covers blocks [start[s], start[s+1]) and works on item
// id[s].
struct BLaunch {
    int n;
    int id[BATCH_MAX];
    int start[BATCH_MAX + 1];
};

// Launch-wide reduction state (device).
struct BCtl {
    unsigned int arrive;
};

// Block shapes of the batched kernels.
enum BGeom : int {
    BG_STENCIL = 0,  // 32 x 8 node tiles x kz planes (the z-march kernels)
    BG_FLAT,         // 4096 consecutive padded elements per block (whole-vector initialisation)
    BG_SPAN,         // node plane spans (0,0,k)..(nx,ny,k): whole planes, or chunks of one, per block (K2)
    BG_SPAN_FINE,    // one chunk of at most 1024 vectors of one plane span per block (fold, max |x|)
    BG_NODES,        // 32 x 8 nodes of one plane per block
    BG_ELEMS,        // 32 x 8 elements of one slab per block
    BG_EXPF,         // 128 level-(l-2) elements per block
    BG_EXPT,         // 128 level-(l-1) elements per block
    BG_ROWS,         // 32 rows (j, k) per block
    BG_ONE,          // one block per item
    BG_COUNT
};
constexpr int BFLAT_ELEMS = 4096;

// The owned nodes of node plane k lie in the span from node (0, 0, k) to node (nx, ny, k) of the
// padded layout (rows of pitch elements: the ghost rows and planes around it are skipped, the row
// padding in between is not). In 4-element vectors, rounded up (the span starts 16-byte
// aligned; the last vector ends inside row ny's padding).
__host__ __device__ inline int span_v4(const Grid& g) { return (int)(((int64_t)g.ny * g.pitch + g.nx + 1 + 3) / 4); }
// A BG_SPAN block covers about SPAN_BLOCK_V4 vectors: several whole planes of a small level, or
// a chunk of one plane of a large one, so that every block has enough work to pay for its
// reduction.
constexpr int SPAN_BLOCK_V4 = 4096;
// The fold and max |x| of a replacement usually run on one problem alone: their blocks take
// chunks of at most SPAN_FINE_V4 vectors of one plane, for more blocks on one problem.
constexpr int SPAN_FINE_V4 = 1024;
__host__ __device__ inline int span_planes_per_block(const Grid& g)
{
    const int v = span_v4(g);
    return v >= SPAN_BLOCK_V4 ? 1 : SPAN_BLOCK_V4 / v;
}
__host__ __device__ inline int span_chunks_per_plane(const Grid& g)
{
    const int v = span_v4(g);
    return v <= SPAN_BLOCK_V4 ? 1 : (v + SPAN_BLOCK_V4 - 1) / SPAN_BLOCK_V4;
}

// Blocks one item needs in a geometry (host).
int bgeom_blocks(BGeom geo, const BItem& it);
// Most per-block partial pairs any reducing launch needs for this item (host).
int bitem_partials(const BItem& it);

// Set-up of one depth (finest first): beta (packed or averaged) and its FP32 copy; f, g_D, g_R
// (packed or injected); the load vector; the FP32 Jacobi diagonal.
void blaunch_setup(const BItem* items, const BLaunch& nodes, const BLaunch& elems, cudaStream_t s);
// Start of a level: state reset, Dirichlet extension, ||f_h||^2.
void blaunch_level_start(const BItem* items, const BLaunch& one, const BLaunch& nodes, const BLaunch& rows,
                         int robin, int cube, double inner_rtol, cudaStream_t s);
// EXP_finite for levels >= 2 (x and W), W = x on the direct levels 0 and 1, and zeroed FP32
// search directions and corrections.
void blaunch_guess(const BItem* items, const BLaunch& expf, const BLaunch& flat_all, int variant, cudaStream_t s);
// FP64 residual r = b - A x (stored FP32 into r32, or r32B with r_to_b) with r.z and ||r||^2 per
// item; mode RES_INIT or
// RES_REPLACE (items that asked for a replacement only). Sets the loop condition. With cubic
// elements and no Robin term, A x is exact in fixed point up to the products with beta
// (march_fx.cuh), on the scale of max |x| that blaunch_absmax (before RES_INIT) or
// blaunch_fold (before RES_REPLACE) left in the item's state.
void blaunch_res(const BItem* items, const BLaunch& stencil, int robin, int cube, ResMode mode, BCtl* ctl,
                 CondHandles ch, cudaStream_t s, int r_to_b = 0);
// K2 of one FP32 JCG iteration (after K1, blaunch_pq_tma): r -= alpha q, r.z, r.r and the
// item's tests; sets the loop and replacement conditions.
void blaunch_update(const BItem* items, const BLaunch& flat, BCtl* ctl, CondHandles ch, cudaStream_t s);
// Fold the FP32 correction into the FP64 iterate for items that asked for a replacement, and
// take max |x| of the new iterate into the item's state (the scale of the exact residual).
// fine: a BG_SPAN_FINE launch.
void blaunch_fold(const BItem* items, const BLaunch& fine, int pnew_is_b, cudaStream_t s);
// max |x| of each running item's iterate into its state, before an initial residual (fine: a
// BG_SPAN_FINE launch).
void blaunch_absmax(const BItem* items, const BLaunch& fine, cudaStream_t s);
// EXP_true for levels >= 2.
void blaunch_exp_true(const BItem* items, const BLaunch& expt, cudaStream_t s);

// TMA-staged K1 (batch_tma.cu): p = D^-1 r + beta p_old, q = A p, e += alpha_prev p_old and
// the item's p.q, one launch over the items of L with tiles of 32 x 8 ry nodes and k1kz planes;
// maps: the items' tensor maps (device array indexed like items).
void blaunch_pq_tma(const BItem* items, const PlaneMaps* maps, const BLaunch& L, int ry, int robin, int cube,
                    int pin_is_b, int pidx, cudaStream_t s);
// The single-pass step over the items of L (buffer set in_b read, the other written), which
// also sets the loop and replacement conditions from all items (ctl: the launch-wide counter).
void blaunch_step_tma(const BItem* items, const PlaneMaps* maps, const BLaunch& L, int ry, int robin, int cube,
                      int in_b, int pidx, BCtl* ctl, CondHandles ch, cudaStream_t s);
// Blocks of one item in that launch, the most any tile shape needs, and the nodes it computes.
int bk1_blocks(const BItem& it, int ry);
int bk1_max_blocks(const BItem& it);
int64_t bk1_nodes(const BItem& it);
// Shared-memory limits of the batched K1 instantiations on the current device.
cudaError_t bk1_prepare();

unsigned long long launches_batch();
unsigned long long launches_batch_tma();

}  // namespace ecmg
