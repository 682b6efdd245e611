// api.cu -- host driver of ECMG_jcg (Alg. 4) behind the C ABI of include/ecmg.h.
//
// ecmg_solve records the whole method -- set-up of every level, DSOLVE on levels 0 and 1,
// then EXP_finite / JCG / EXP_true on every finer level -- into one CUDA graph on first use.
// Each level's JCG loop is a conditional WHILE node whose condition the kernels themselves
// set (see jcg.cu); in MIXED precision the FP64 residual replacement is a conditional IF node
// inside the loop body. A solve is therefore one graph launch and one stream synchronisation.
// With options.use_graph = 0 the same kernels run eagerly and the host reads the level state
// after every iteration (for debugging).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ecmg.h"
#include "batch.cuh"
#include "ecmg_internal.cuh"
#include "exp.cuh"
#include "jcg.cuh"
#include "pq_tma.cuh"
#include "res_cc.cuh"
#include "separable.cuh"

using namespace ecmg;

namespace {

// A batch of independent problems (ecmg_create_batched): one item per (problem, level).
struct Batch {
    int n = 0;
    int Lmax = 0;
    std::vector<int> L;            // levels of each problem
    std::vector<int> first;        // item index of (problem, level 0)
    std::vector<BItem> items;      // host copy of the item table
    BItem* d_items = nullptr;      // device item table
    SolveState* states = nullptr;  // device, one per item
    SolveState* host_states = nullptr;  // pinned
    BCtl* ctl = nullptr;
    int robin = 0, cube = 1;       // kernel variants: any Robin face in the batch; all elements cubic
    PlaneMaps* d_maps = nullptr;   // device, the tensor maps of every item's FP32 vectors
    std::vector<ecmg_problem> probs;  // the problems (device input pointers resolved)
    std::vector<double*> Hf;       // per problem: 1D hat integrals of separable f (else null)
    bool sp = false;               // FP32 steps in the single-pass form (one kernel per step)
    std::vector<int> stage_ry;     // node rows per thread of the TMA-staged K1 at each stage
    int item(int p, int l) const { return first[p] + l; }
};

thread_local std::string g_last_error;

struct CudaFail {
    cudaError_t e;
};

inline void ck(cudaError_t e)
{
    if (e != cudaSuccess) throw CudaFail{e};
}

struct Level {
    Grid g;
    Op op;
    // FP64 vectors
    double *U = nullptr, *W = nullptr, *Ut = nullptr, *b = nullptr, *beta = nullptr, *dinv = nullptr;
    double *f = nullptr, *gD = nullptr, *gR = nullptr;  // injected data (nodal mode); f = load (load mode)
    double *r = nullptr, *pA = nullptr, *pB = nullptr, *q = nullptr;
    // FP32 vectors (mixed precision)
    float *beta32 = nullptr, *dinv32 = nullptr, *r32 = nullptr, *pA32 = nullptr, *pB32 = nullptr,
          *q32 = nullptr, *e32 = nullptr;
    float *r32B = nullptr, *q32B = nullptr;  // single-pass form: second r and q buffers
    // two-pass form with a ring of search directions: R stored directions and their steps alpha
    float* ring = nullptr;
    double* ring_alpha = nullptr;
    int R = 0;
    PlaneMaps maps;  // TMA descriptors of the FP32 vectors
    ResMaps rmaps;   // TMA descriptors of U and of b / c (exact constant-coefficient residual)
    K1Config k1{1, 128};  // tile shape of the FP32 stencil kernel
    int* uniform = nullptr;  // device flag: one beta on the whole level
    bool cc = false;         // the FP32 stencil runs its constant-coefficient kernel (host choice)
    // 1D factors of separable data (ECMG_F_SEPARABLE load, separable g_D); Hg of the finest level
    // is the caller's array
    double *Hf = nullptr, *Hg = nullptr;
};

}  // namespace

struct ecmg_handle {
    ecmg_problem prob;
    ecmg_options opt;
    cudaStream_t user_stream = nullptr;
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};  // capture streams (graph + 2 nesting levels)
    int L = 0;
    Level lv[MAX_LEVELS];
    SolveState* states = nullptr;  // device, one per level
    KTimer* timers = nullptr;      // device, one per level: the FP32 stencil launches of the solves
    Partials part{nullptr, 0, nullptr};
    double* norm_part = nullptr;   // device, per-block norm partials
    std::vector<std::pair<void*, size_t>> allocs;  // device workspace blocks and their sizes
    ecmg_alloc_fn alloc_fn = nullptr;              // caller's allocator (ecmg_create_with_allocator)
    ecmg_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    unsigned long long* stamps = nullptr;       // device: global timer at the set-up, at each level's start, at the end
    unsigned long long* host_stamps = nullptr;  // pinned copy
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    SolveState* host_states = nullptr;  // pinned
    double* host_norms = nullptr;       // pinned
    int graph_first = -1;               // first level of the recorded graph
    Batch* batch = nullptr;             // batched handle (ecmg_create_batched), else null
    // the starts of the large levels (state, Dirichlet shell, ||f_h||) on a second stream while
    // the small levels solve (record_solve): the stream, its partials, one event per level it
    // completes; the same stream takes the copy of the solution beside the last EXP_true
    cudaStream_t side = nullptr;
    Partials part_side{nullptr, 0, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_level[MAX_LEVELS] = {};
    // the caller's output array of the running solve (device slot, null: none), and the fork and
    // join of its copy, which runs beside the finest level's EXP_true
    double** out_slot = nullptr;
    cudaEvent_t ev_out_fork = nullptr, ev_out_join = nullptr;
};

namespace {

ecmg_status fail(ecmg_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

// The library's kernels read and write caller arrays through the pointers they are given:
// device memory of the current device, managed memory and page-locked host memory
// (cudaHostAlloc / cudaHostRegister, which a GB300 reaches over its coherent chip-to-chip link)
// qualify, and *dev receives the address the kernels use. Any other pointer (pageable host
// memory, another device's memory, an invalid address) would fault the GPU, so it is refused.
bool kernel_accessible(const void* p, const void** dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return false;
    switch (a.type) {
    case cudaMemoryTypeDevice:
        if (a.device != cur) return false;
        *dev = p;
        return true;
    case cudaMemoryTypeManaged:
        *dev = p;
        return true;
    case cudaMemoryTypeHost:
        if (!a.devicePointer) return false;
        *dev = a.devicePointer;
        return true;
    default:
        return false;
    }
}

// The input arrays of a problem, each replaced by the address the kernels use; false if one of
// them is not reachable by the kernels.
bool resolve_inputs(ecmg_problem* p)
{
    for (const double** q : {&p->beta, &p->f, &p->g_D, &p->g_R}) {
        if (!*q) continue;
        const void* d = nullptr;
        if (!kernel_accessible(*q, &d)) return false;
        *q = static_cast<const double*>(d);
    }
    return true;
}

// An output (or input) array of a call, as the address the kernels use; null if not reachable.
template <typename T>
T* resolve_array(T* p)
{
    const void* d = nullptr;
    return kernel_accessible(p, &d) ? static_cast<T*>(const_cast<void*>(d)) : nullptr;
}

bool op_robin(const Op& op)
{
    for (int f = 0; f < 6; ++f)
        if (op.alpha[f] != 0.0) return true;
    return false;
}

Grid make_grid(const ecmg_problem& p, int l)
{
    Grid g;
    g.nx = p.n0[0] << l;
    g.ny = p.n0[1] << l;
    g.nz = p.n0[2] << l;
    g.pitch = ((g.nx + 1 + XL + 2) + 7) / 8 * 8;  // rows 32-byte aligned (FP32), 16-byte TMA strides
    g.plane = (int64_t)g.pitch * (g.ny + 3);
    g.total = g.plane * (g.nz + 3);
    for (int a = 0; a < 3; ++a) g.h[a] = (p.hi[a] - p.lo[a]) / (double)(p.n0[a] << l);
    return g;
}

ecmg_status validate(const ecmg_problem* p, const ecmg_options* o)
{
    if (!p || !o) return fail(ECMG_ERR_INVALID_ARG, "null problem or options");
    if (p->levels < 3 || p->levels > 12) return fail(ECMG_ERR_INVALID_ARG, "levels must be 3..12");
    for (int a = 0; a < 3; ++a) {
        if (p->n0[a] < 1) return fail(ECMG_ERR_INVALID_ARG, "n0 must be >= 1");
        if (!(p->hi[a] > p->lo[a])) return fail(ECMG_ERR_INVALID_ARG, "hi must exceed lo");
        int64_t nf = (int64_t)p->n0[a] << (p->levels - 1);
        if (nf > 16384) return fail(ECMG_ERR_INVALID_ARG, "finest grid too large");
    }
    if (!p->f) return fail(ECMG_ERR_INVALID_ARG, "f is required");
    if (!p->beta && !(p->beta_const > 0.0 && std::isfinite(p->beta_const)))
        return fail(ECMG_ERR_INVALID_ARG, "beta is NULL and beta_const is not a finite positive number");
    if (p->f_mode != ECMG_F_NODAL && p->f_mode != ECMG_F_LOAD && p->f_mode != ECMG_F_SEPARABLE &&
        p->f_mode != ECMG_F_GAUSS)
        return fail(ECMG_ERR_INVALID_ARG, "bad f_mode");
    if (p->f_mode == ECMG_F_SEPARABLE) {
        if (p->f_terms < 1 || p->f_terms > 64) return fail(ECMG_ERR_INVALID_ARG, "f_terms must be 1..64");
        if (p->g_R) return fail(ECMG_ERR_INVALID_ARG, "ECMG_F_SEPARABLE takes no g_R");
    }
    if (p->gD_terms < 0 || p->gD_terms > 64) return fail(ECMG_ERR_INVALID_ARG, "gD_terms must be 0..64");
    if (p->gD_terms > 0 && !p->g_D) return fail(ECMG_ERR_INVALID_ARG, "gD_terms > 0 needs g_D");
    bool dir = false, alpha = false;
    for (int f = 0; f < 6; ++f) {
        if (p->face_bc[f] != ECMG_BC_DIRICHLET && p->face_bc[f] != ECMG_BC_ROBIN)
            return fail(ECMG_ERR_INVALID_ARG, "bad face_bc");
        if (p->face_bc[f] == ECMG_BC_DIRICHLET) dir = true;
        else {
            if (!(p->robin_alpha[f] >= 0.0) || !std::isfinite(p->robin_alpha[f]))
                return fail(ECMG_ERR_INVALID_ARG, "robin_alpha must be finite and >= 0");
            if (p->robin_alpha[f] > 0.0) alpha = true;
        }
    }
    if (!dir && !alpha) return fail(ECMG_ERR_SINGULAR, "no Dirichlet face and every Robin alpha is 0");
    if (!(o->rtol > 0.0) || !(o->rtol < 1.0)) return fail(ECMG_ERR_INVALID_ARG, "rtol must be in (0,1)");
    if (o->precision != ECMG_FP64 && o->precision != ECMG_MIXED)
        return fail(ECMG_ERR_INVALID_ARG, "bad precision");
    if (o->precision == ECMG_MIXED && !(o->inner_rtol > 0.0 && o->inner_rtol < 1.0))
        return fail(ECMG_ERR_INVALID_ARG, "inner_rtol must be in (0,1)");
    if (o->max_iters < 1) return fail(ECMG_ERR_INVALID_ARG, "max_iters must be >= 1");
    if (!(o->dsolve_rtol > 0.0 && o->dsolve_rtol < 1.0))
        return fail(ECMG_ERR_INVALID_ARG, "dsolve_rtol must be in (0,1)");
    if (o->exp_variant != ECMG_EXP_SERENDIPITY20 && o->exp_variant != ECMG_EXP_LAGRANGE27)
        return fail(ECMG_ERR_INVALID_ARG, "bad exp_variant");
    if (o->autotune != 0 && o->autotune != 1) return fail(ECMG_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (o->preconditioner != ECMG_PREC_JACOBI && o->preconditioner != ECMG_PREC_NONE)
        return fail(ECMG_ERR_INVALID_ARG, "bad preconditioner");
    if (o->schedule != ECMG_SCHED_TOLERANCE && o->schedule != ECMG_SCHED_FIXED)
        return fail(ECMG_ERR_INVALID_ARG, "bad schedule");
    if (o->cg_form != ECMG_CG_TWO_PASS && o->cg_form != ECMG_CG_SINGLE_PASS && o->cg_form != ECMG_CG_AUTO)
        return fail(ECMG_ERR_INVALID_ARG, "bad cg_form");
    if (o->ring_slots != ECMG_RING_AUTO && o->ring_slots != 0 && (o->ring_slots < 4 || o->ring_slots > 64))
        return fail(ECMG_ERR_INVALID_ARG, "ring_slots must be ECMG_RING_AUTO, 0 or in [4, 64]");
    if (o->schedule == ECMG_SCHED_FIXED) {
        if (o->sched_mL < 1 || !(o->sched_beta >= 1.0 && o->sched_beta <= 64.0))
            return fail(ECMG_ERR_INVALID_ARG, "fixed schedule: sched_mL >= 1 and sched_beta in [1, 64]");
        if ((double)o->sched_mL * std::pow(o->sched_beta, (double)(p->levels - 3)) > 1e8)
            return fail(ECMG_ERR_INVALID_ARG, "fixed schedule: more than 1e8 steps on a level");
    }
    return ECMG_OK;
}

// Byte count of the per-level vectors (the same arithmetic ecmg_create performs).
uint64_t level_bytes(const Grid& g, bool mixed, bool single_pass, int ring_slots)
{
    const uint64_t n = (uint64_t)g.total;
    uint64_t b = n * 8ull * 14ull;  // U W Ut b beta dinv f gD gR r pA pB q (+1 spare alignment)
    if (mixed) b += n * 4ull * (single_pass ? 9ull : 7ull);
    if (ring_slots) b += ((uint64_t)ring_stride((int64_t)n) * 4ull + 8ull) * (uint64_t)ring_slots;
    return b;
}

// Partial sums per block of the reducing kernels: 3 (FP64 and residual kernels), 7 (the
// single-pass step on the general path); rounded up to 8.
int partials_per_block(const ecmg_options& o)
{
    return (o.precision == ECMG_MIXED && o.cg_form != ECMG_CG_TWO_PASS) ? 8 : 3;
}

// Whether MIXED level l (>= 2) runs the single-pass step: always, never, or (AUTO) on levels
// of fewer than ECMG_AUTO_SINGLE_PASS_NODES nodes.
// FP32 steps per replacement check in the loop body of a level with a ring of search directions.
constexpr int RING_STEPS = 4;

bool single_pass_level(const ecmg_options& o, const Grid& g, int l)
{
    if (o.precision != ECMG_MIXED || l < 2) return false;
    if (o.cg_form == ECMG_CG_SINGLE_PASS) return true;
    if (o.cg_form != ECMG_CG_AUTO) return false;
    return (int64_t)(g.nx + 1) * (g.ny + 1) * (g.nz + 1) < (int64_t)ECMG_AUTO_SINGLE_PASS_NODES;
}

// Slots of the ring of search directions on level l: the MIXED two-pass levels (>= 2) of a
// single-problem handle with every face Dirichlet, when the option asks for one. A solve uses the
// ring on such a level when it also has one beta: the constant-coefficient FP32 stencil kernel is
// bound by DRAM bandwidth, so the correction-vector bytes it no longer moves are time saved; the
// general kernel (beta and D^-1 streamed, Robin terms) runs below the bandwidth bound, and there
// the directions the ring reads back at a replacement would cost more than they save.
int ring_slots_level(const ecmg_problem& p, const ecmg_options& o, const Grid& g, int l)
{
    if (o.precision != ECMG_MIXED || l < 2 || single_pass_level(o, g, l)) return 0;
    for (int f = 0; f < 6; ++f)
        if (p.face_bc[f] != ECMG_BC_DIRICHLET) return 0;
    return o.ring_slots;
}

template <typename T>
T* dalloc(ecmg_handle* h, int64_t n)
{
    void* p = nullptr;
    const size_t bytes = (size_t)n * sizeof(T);
    if (bytes == 0) return nullptr;
    if (h->alloc_fn) {
        p = h->alloc_fn(bytes, (void*)h->user_stream, h->alloc_ctx);
        if (!p) throw CudaFail{cudaErrorMemoryAllocation};
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) throw CudaFail{e};
    }
    h->allocs.emplace_back(p, bytes);
    ck(cudaMemsetAsync(p, 0, (size_t)n * sizeof(T), h->cap[0]));
    return (T*)p;
}

// ---- recording: graph capture with conditional nodes, or eager execution ------------------
struct Rec {
    ecmg_handle* h;
    bool graph;
    int depth = 0;
    cudaStream_t s() const { return graph ? h->cap[depth] : h->user_stream; }

    // A conditional handle on the graph being captured on s(); its value is reset to 0 at every
    // graph launch and set by the kernels.
    cudaGraphConditionalHandle new_handle()
    {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg;
        ck(cudaStreamGetCaptureInfo(s(), &cs, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle hd;
        ck(cudaGraphConditionalHandleCreate(&hd, cg, 0, cudaGraphCondAssignDefault));
        return hd;
    }
    // Append a WHILE / IF node after everything captured so far on s() and continue capturing
    // into its body on the next stream until close().
    void open(cudaGraphConditionalHandle hd, cudaGraphConditionalNodeType type)
    {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* ed = nullptr;
        size_t nd = 0;
        ck(cudaStreamGetCaptureInfo(s(), &cs, nullptr, &cg, &deps, &ed, &nd));
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = hd;
        np.conditional.type = type;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        ck(cudaGraphAddNode(&node, cg, deps, ed, nd, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        ck(cudaStreamUpdateCaptureDependencies(s(), &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        ++depth;
        ck(cudaStreamBeginCaptureToGraph(s(), body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    }
    void close()
    {
        cudaGraph_t g;
        ck(cudaStreamEndCapture(s(), &g));
        --depth;
    }
};

void host_state(ecmg_handle* h, int l, SolveState* out)
{
    ck(cudaMemcpyAsync(out, h->states + l, sizeof(SolveState), cudaMemcpyDeviceToHost, h->user_stream));
    ck(cudaStreamSynchronize(h->user_stream));
}

bool constant_coefficient(ecmg_handle* h, const Level& v);
void drop_graph(ecmg_handle* h);

// FP64 residual of the MIXED iteration into r32 (or, in the single-pass form, into the residual
// buffer the next step reads): on a constant-coefficient level (the host's choice v.cc, cubic
// elements) the TMA-staged exact kernel, else the general one.
// r_b: the single-pass buffer pair taken from the level state (constant-coefficient cubes): the
// residual goes to rdst or r_b, whichever st->p_latest names.
void res32(ecmg_handle* h, Level& v, SolveState* st, ResMode mode, CondHandles ch, cudaStream_t s,
           float* rdst = nullptr, float* r_b = nullptr)
{
    float* r = rdst ? rdst : v.r32;
    if (v.cc && v.op.cube) {
        // a replacement follows the fold, which has taken max |U| already
        if (mode != RES_REPLACE) launch_absmax(v.g, v.U, v.uniform, st, (int)mode, h->part, s);
        launch_res32_cc(v.rmaps, v.g, v.uniform, v.beta, v.dinv32, r, st, h->part, mode, ch, s, r_b);
    } else {
        launch_res32(v.g, v.op, v.beta, v.uniform, v.U, v.b, v.dinv32, r, st, h->part, mode, ch, s, v.r);
    }
}

// ---- level set-up (finest to coarsest) -------------------------------------------------------
void record_setup(Rec& R)
{
    ecmg_handle* h = R.h;
    const ecmg_problem& p = h->prob;
    cudaStream_t s = R.s();
    const bool mixed = h->opt.precision == ECMG_MIXED;
    const int L = h->L;
    // MIXED with a dense beta: the finest beta, its FP32 copy, the uniform flag and the beta of the
    // level below in one pass over the caller's array (16-byte pairs: the array must be aligned)
    const bool fused_beta = mixed && p.beta && L >= 3 && reinterpret_cast<uintptr_t>(p.beta) % 16 == 0;
    for (int l = L - 1; l >= 0; --l) {
        Level& v = h->lv[l];
        if (l == L - 1) {
            if (fused_beta) beta_finest(v.g, h->lv[L - 2].g, p.beta, v.beta, v.beta32, v.uniform, h->lv[L - 2].beta, s);
            else if (p.beta) pack_elements(v.g, p.beta, v.beta, s);
            else fill_beta(v.g, p.beta_const, v.beta, s);
            if (p.g_R) pack_nodal(v.g, p.g_R, v.gR, s);
            if (p.f_mode == ECMG_F_SEPARABLE) sep_load_finest(v.g, p.f_terms, p.f, v.Hf, v.b, s);
            else if (p.f_mode == ECMG_F_GAUSS) gauss_load(v.g, v.op, p.f, p.g_R ? v.gR : nullptr, v.b, s);
            else pack_nodal(v.g, p.f, p.f_mode == ECMG_F_LOAD ? v.b : v.f, s);  // the load is b itself
            if (p.g_D && p.gD_terms > 0) sep_nodal(v.g, p.gD_terms, p.g_D, v.gD, s);
            else if (p.g_D) pack_dirichlet(v.g, v.op, p.g_D, v.gD, s);
        } else {
            Level& u = h->lv[l + 1];
            if (!(fused_beta && l == L - 2)) coarsen_beta(v.g, u.beta, u.g, v.beta, s);
            if (p.f_mode == ECMG_F_LOAD || p.f_mode == ECMG_F_GAUSS) restrict_load(v.g, u.b, u.g, v.b, s);
            else if (p.f_mode == ECMG_F_SEPARABLE) sep_coarsen(v.g, u.g, p.f_terms, u.Hf, v.Hf, true, v.b, s);
            else inject_nodal(v.g, u.f, u.g, v.f, s);
            if (p.g_D && p.gD_terms > 0)
                sep_coarsen(v.g, u.g, p.gD_terms, l + 1 == L - 1 ? p.g_D : u.Hg, v.Hg, false, v.gD, s);
            else if (p.g_D) inject_nodal(v.g, u.gD, u.g, v.gD, s);
            if (p.g_R) inject_nodal(v.g, u.gR, u.g, v.gR, s);
        }
        if (p.f_mode == ECMG_F_NODAL) {
            nodal_load(v.g, v.op, v.f, p.g_R ? v.gR : nullptr, v.b, s);
        }
        if (mixed && l >= 2) {
            if (!(fused_beta && l == L - 1)) beta32_uniform(v.g, v.beta, v.beta32, v.uniform, s);
        } else {
            uniform_check(v.g, v.beta, v.uniform, s);
        }
        // FP64 diagonal for FP64 JCG and the direct levels, FP32 for the FP32 iteration of MIXED
        jacobi_diag(v.g, v.op, v.beta, (!mixed || l < 2) ? v.dinv : nullptr, mixed ? v.dinv32 : nullptr,
                    mixed ? v.beta32 : nullptr, h->opt.preconditioner == ECMG_PREC_JACOBI, s,
                    l >= 2 ? v.uniform : nullptr);
    }
}

// Steps of level l (>= 2) of an L-level hierarchy in the fixed schedule of Alg. 3, eq. (ee): the
// paper numbers the levels above the two direct ones j = l - 1 = 1 .. L - 2 and sets
// m_j = ceil(m_L beta^(L_p - j)) with L_p = L - 2.
int schedule_steps(int L, int l, int mL, double beta)
{
    return (int)std::ceil((double)mL * std::pow(beta, (double)((L - 2) - (l - 1))));
}

// ---- one level of Alg. 4 ------------------------------------------------------------------------
// The start of level l: its state, the Dirichlet extension and ||f_h|| (Alg. 4 line 7's
// threshold). It needs only the set-up (b, beta, g_D of the level), not the coarser solutions,
// so after a full set-up the starts of the large levels run on a second stream while the small
// levels solve (record_solve); pr: the partials of the ||f_h|| reduction on that stream,
// fh_blocks: a cap on the blocks of that pass (0: none).
void level_start(ecmg_handle* h, bool graph, int l, cudaStream_t s, Partials pr, int fh_blocks = 0)
{
    Level& v = h->lv[l];
    SolveState* st = h->states + l;
    const ecmg_options& o = h->opt;
    const bool direct = l < 2;
    const bool mixed = o.precision == ECMG_MIXED && !direct;
    const bool fixed = o.schedule == ECMG_SCHED_FIXED && !direct;
    const double rtol = direct ? o.dsolve_rtol : (fixed ? 0.0 : o.rtol);
    const int max_iters = fixed ? schedule_steps(h->L, l, o.sched_mL, o.sched_beta) : o.max_iters;
    // eager: the set-up of this solve (or of the last one, for a solve from a finer level) has
    // run, so the level's flag can be read now; a graph takes the choice made before its recording
    if (mixed && !graph) v.cc = constant_coefficient(h, v);
    // the ring of search directions runs with the constant-coefficient stencil kernel only
    const bool ring_on = mixed && v.ring && v.cc;
    launch_state_init(st, rtol, o.inner_rtol, max_iters, fixed ? 1 : 0, s, ring_on ? v.R : 0);
    // levels >= 2: EXP_finite writes every free node below, so only the shell that ||f_h|| reads
    dirichlet_extension(v.g, v.op, h->prob.g_D ? v.gD : nullptr, v.U, s, /*shell=*/l >= 2);
    // MIXED: also b / c and its max on a constant-coefficient level, the exact residual's load
    // and scale, kept in the FP64 r vector, which the MIXED iteration does not use
    launch_fh2(v.g, v.op, v.beta, v.U, v.b, st, pr, s, mixed ? v.uniform : nullptr, mixed ? v.r : nullptr,
               fh_blocks);
}

// started: level_start has run for this level (on the side stream, joined before this call)
void record_level(Rec& R, int l, bool started = false)
{
    ecmg_handle* h = R.h;
    Level& v = h->lv[l];
    SolveState* st = h->states + l;
    const ecmg_options& o = h->opt;
    const bool direct = l < 2;
    const bool mixed = o.precision == ECMG_MIXED && !direct;
    CondHandles none{0, 0, 0};
    if (!started) level_start(h, R.graph, l, R.s(), h->part);
    else if (mixed && !R.graph) v.cc = constant_coefficient(h, v);
    const bool ring_on = mixed && v.ring && v.cc;
    if (!direct) {
        const Level& u1 = h->lv[l - 1];
        const Level& u0 = h->lv[l - 2];
        launch_exp_finite(o.exp_variant, v.g, v.op, u1.g, u1.U, u0.g, u0.U, v.U, v.W, R.s());
    } else {
        ck(cudaMemcpyAsync(v.W, v.U, (size_t)v.g.total * 8, cudaMemcpyDeviceToDevice, R.s()));
    }

    if (!mixed) {
        ck(cudaMemsetAsync(v.pA, 0, (size_t)v.g.total * 8, R.s()));
        ck(cudaMemsetAsync(v.pB, 0, (size_t)v.g.total * 8, R.s()));
        auto half = [&](CondHandles ch, const double* pin, double* pout, int idx) {
            launch_pq64(v.g, v.op, v.beta, v.uniform, v.r, v.dinv, pin, pout, v.q, v.U, st, h->part, idx, ch, R.s());
            launch_update64(v.g, v.r, v.q, v.dinv, st, h->part, ch, R.s());
        };
        if (R.graph) {
            const cudaGraphConditionalHandle loop = R.new_handle();
            const CondHandles ch{loop, 0, 1};
            launch_res64(v.g, v.op, v.beta, v.uniform, v.U, v.b, v.dinv, v.r, st, h->part, RES_INIT, ch, R.s());
            R.open(loop, cudaGraphCondTypeWhile);
            half(ch, v.pA, v.pB, 1);
            half(ch, v.pB, v.pA, 0);
            R.close();
        } else {
            launch_res64(v.g, v.op, v.beta, v.uniform, v.U, v.b, v.dinv, v.r, st, h->part, RES_INIT, none, R.s());
            SolveState hs;
            host_state(h, l, &hs);
            int parity = 0;
            while (!hs.done) {
                if (parity == 0) half(none, v.pA, v.pB, 1);
                else half(none, v.pB, v.pA, 0);
                parity ^= 1;
                host_state(h, l, &hs);
            }
        }
        launch_final64(v.g, v.U, v.pA, v.pB, st, R.s());
        if (o.true_residual)
            launch_res64(v.g, v.op, v.beta, v.uniform, v.U, v.b, v.dinv, v.r, st, h->part, RES_REPORT, none, R.s());
    } else {
        ck(cudaMemsetAsync(v.pA32, 0, (size_t)v.g.total * 4, R.s()));
        ck(cudaMemsetAsync(v.pB32, 0, (size_t)v.g.total * 4, R.s()));
        ck(cudaMemsetAsync(v.e32, 0, (size_t)v.g.total * 4, R.s()));
        // ring: slot 0 holds the zero direction the first step reads (its beta is 0 as well)
        if (ring_on) ck(cudaMemsetAsync(v.ring, 0, (size_t)v.g.total * 4, R.s()));
        const RingArgs ring{v.ring, v.ring_alpha, v.R};
        const RingArgs* rp = ring_on ? &ring : nullptr;
        // Step `half` of the loop body reads the buffers of set A (half 0) or B (half 1) and
        // writes the other set: p in both forms, r and q too in the single-pass form (which
        // keeps 0 in them on the nodes no step visits). The residual of the initial state and
        // of a replacement goes to the r buffer the next step reads.
        const bool single = v.r32B != nullptr;
        float* rbuf[2] = {v.r32, single ? v.r32B : v.r32};
        float* qbuf[2] = {v.q32, single ? v.q32B : v.q32};
        float* pbuf[2] = {v.pA32, v.pB32};
        // single pass on a constant-coefficient cube: the step picks its buffer set from the level
        // state, so the loop body needs no fixed alternation and can check for a replacement once
        // per several steps (a step behind the one that asked returns at once)
        const bool pf = single && v.cc && v.op.cube;
        SpSets sets{{v.pA32, v.pB32}, {v.q32, v.q32B}, {v.r32, v.r32B}};
        auto step = [&](CondHandles ch, int half) {
            const int o = half ^ 1;
            if (single) {
                launch_step32(v.maps, half, v.k1, v.g, v.op, v.cc, v.uniform, v.beta32, v.dinv32, pbuf[o], qbuf[o],
                              rbuf[o], v.e32, st, h->part, o, ch, h->timers + l, R.s(), pf ? &sets : nullptr);
            } else {
                launch_pq32_tma(v.maps, half, v.k1, v.g, v.op, v.cc, v.uniform, v.beta32, v.dinv32, pbuf[o], v.q32,
                                v.e32, st, h->part, o, ch, h->timers + l, R.s(), rp);
                launch_update32(v.g, v.op, v.uniform, v.r32, v.q32, v.dinv32, st, h->part, ch, R.s(),
                                rp, v.e32);
            }
        };
        auto replace = [&](int half) {
            const int o = half ^ 1;
            if (ring_on) launch_fold_ring(v.g, v.U, ring, v.e32, v.uniform, st, h->part, R.s());
            else if (pf) launch_fold32(v.g, v.U, v.e32, pbuf[0], v.uniform, st, h->part, R.s(), pbuf[1]);
            else launch_fold32(v.g, v.U, v.e32, pbuf[o], v.uniform, st, h->part, R.s());
            if (pf) res32(h, v, st, RES_REPLACE, none, R.s(), rbuf[0], rbuf[1]);
            else res32(h, v, st, RES_REPLACE, none, R.s(), rbuf[o]);
        };
        if (R.graph && (ring_on || pf)) {
            // with the ring every step reads and writes the same buffers (with pf the buffers come
            // from the level state), so one replacement check serves RING_STEPS steps: a step
            // after the one that asks for a replacement finds need_update set and returns at once
            const cudaGraphConditionalHandle loop = R.new_handle();
            res32(h, v, st, RES_INIT, CondHandles{loop, 0, 1}, R.s(), rbuf[0]);
            R.open(loop, cudaGraphCondTypeWhile);
            const cudaGraphConditionalHandle upd = R.new_handle();  // on the loop body
            for (int k = 0; k < RING_STEPS; ++k) step(CondHandles{loop, upd, 1}, 0);
            R.open(upd, cudaGraphCondTypeIf);
            replace(0);
            R.close();
            R.close();
        } else if (R.graph) {
            const cudaGraphConditionalHandle loop = R.new_handle();
            res32(h, v, st, RES_INIT, CondHandles{loop, 0, 1}, R.s(), rbuf[0]);
            R.open(loop, cudaGraphCondTypeWhile);
            for (int half = 0; half < 2; ++half) {
                const cudaGraphConditionalHandle upd = R.new_handle();  // on the loop body
                step(CondHandles{loop, upd, 1}, half);
                R.open(upd, cudaGraphCondTypeIf);
                replace(half);
                R.close();
            }
            R.close();
        } else {
            res32(h, v, st, RES_INIT, none, R.s(), rbuf[0]);
            SolveState hs;
            host_state(h, l, &hs);
            int half = 0;
            while (!hs.done) {
                step(none, half);
                host_state(h, l, &hs);
                if (hs.need_update && !hs.done) {
                    replace(half);
                    host_state(h, l, &hs);
                }
                half ^= 1;
            }
        }
    }
    if (!direct) {
        const Level& u1 = h->lv[l - 1];
        if (l == h->L - 1 && R.graph) {
            // the solution's copy into the caller's array reads only U: beside EXP_true
            ck(cudaEventRecord(h->ev_out_fork, R.s()));
            ck(cudaStreamWaitEvent(h->side, h->ev_out_fork, 0));
            unpack_out(v.g, v.U, h->out_slot, h->side);
            ck(cudaEventRecord(h->ev_out_join, h->side));
            launch_exp_true(v.g, v.U, u1.g, u1.U, v.Ut, R.s(), h->lv[l - 1].q);
            ck(cudaStreamWaitEvent(R.s(), h->ev_out_join, 0));
        } else {
            launch_exp_true(v.g, v.U, u1.g, u1.U, v.Ut, R.s(), h->lv[l - 1].q);
            if (l == h->L - 1) unpack_out(v.g, v.U, h->out_slot, R.s());
        }
    }
}

// Levels whose start goes to the side stream, and the blocks of its ||f_h|| pass (two per SM:
// enough warps for the FP64 pipe, room on every SM for the small levels' blocks).
constexpr int64_t SIDE_START_NODES = 1 << 22;
constexpr int SIDE_FH_BLOCKS = 2 * 152;

// The whole solve from level `first`, with a global-timer stamp before the set-up, before each
// level and at the end (the per-level seconds of ecmg_stats).
void record_solve(Rec& R, int first)
{
    ecmg_handle* h = R.h;
    // After a full set-up the starts of the levels of at least SIDE_START_NODES nodes depend on
    // nothing the coarser solves write. They are issued before level 2 (after the two direct
    // levels, whose FP64 kernels they would slow) and, in a graph, on the side stream, joined
    // level by level below: their FP64-bound ||f_h|| passes, on at most SIDE_FH_BLOCKS blocks,
    // then run beside the small levels, whose latency-bound steps leave most of the GPU idle.
    auto side = [&](int l) {
        const Level& v = h->lv[l];
        return first == 0 && l >= 2 && (int64_t)(v.g.nx + 1) * (v.g.ny + 1) * (v.g.nz + 1) >= SIDE_START_NODES;
    };
    if (first == 0) {
        launch_stamp(h->stamps, R.s());
        record_setup(R);
    }
    for (int l = first; l < h->L; ++l) {
        if (l == 2 && first == 0) {
            bool any = false;
            for (int m = 2; m < h->L; ++m) any |= side(m);
            if (any && R.graph) {
                ck(cudaEventRecord(h->ev_fork, R.s()));
                ck(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            }
            for (int m = 2; m < h->L; ++m) {
                if (!side(m)) continue;
                if (R.graph) {
                    level_start(h, true, m, h->side, h->part_side, SIDE_FH_BLOCKS);
                    ck(cudaEventRecord(h->ev_level[m], h->side));
                } else {
                    level_start(h, false, m, R.s(), h->part);
                }
            }
        }
        launch_stamp(h->stamps + 1 + l, R.s());
        if (side(l) && R.graph) ck(cudaStreamWaitEvent(R.s(), h->ev_level[l], 0));
        record_level(R, l, side(l));
    }
    launch_stamp(h->stamps + 1 + h->L, R.s());
}

ecmg_status run_solve(ecmg_handle* h, int first, double* u_out, ecmg_stats* stats, bool retried = false)
{
    if (u_out && !(u_out = resolve_array(u_out)))
        return fail(ECMG_ERR_INVALID_ARG, "u_out must be device memory of the current device or page-locked host memory");
    try {
        set_out(h->out_slot, u_out, h->user_stream);  // the finest level writes it (record_level)
        if (h->opt.use_graph) {
            if (!h->exec || h->graph_first != first) {
                // the FP32 stencil path of each level is fixed in the recording: run the set-up
                // once outside the graph so that the levels' uniform flags are current
                if (first == 0) {
                    Rec E{h, false, 0};
                    record_setup(E);
                }
                for (int l = std::max(first, 2); l < h->L; ++l)
                    h->lv[l].cc = h->opt.precision == ECMG_MIXED && constant_coefficient(h, h->lv[l]);
                if (h->exec) {
                    cudaGraphExecDestroy(h->exec);
                    h->exec = nullptr;
                }
                if (h->graph) {
                    cudaGraphDestroy(h->graph);
                    h->graph = nullptr;
                }
                Rec R{h, true, 0};
                ck(cudaStreamBeginCapture(h->cap[0], cudaStreamCaptureModeThreadLocal));
                try {
                    record_solve(R, first);
                } catch (...) {
                    cudaGraph_t junk;
                    cudaStreamEndCapture(h->cap[0], &junk);
                    if (junk) cudaGraphDestroy(junk);
                    throw;
                }
                ck(cudaStreamEndCapture(h->cap[0], &h->graph));
                ck(cudaGraphInstantiate(&h->exec, h->graph, 0));
                h->graph_first = first;
            }
            ck(cudaGraphLaunch(h->exec, h->user_stream));
        } else {
            Rec R{h, false, 0};
            record_solve(R, first);
        }
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(h->host_states, h->states, sizeof(SolveState) * h->L, cudaMemcpyDeviceToHost,
                           h->user_stream));
        ck(cudaMemcpyAsync(h->host_stamps, h->stamps, sizeof(unsigned long long) * (h->L + 2),
                           cudaMemcpyDeviceToHost, h->user_stream));
        ck(cudaStreamSynchronize(h->user_stream));
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(f.e));
    }
    // a level whose recorded constant-coefficient path no longer holds (its beta changed under
    // the graph) computed nothing: record again with the current flags and solve again
    bool stale = false;
    for (int l = first; l < h->L; ++l) stale |= h->host_states[l].status == 6;
    if (stale && !retried) {
        drop_graph(h);
        return run_solve(h, first, u_out, stats, true);
    }
    ecmg_status worst = ECMG_OK;
    ecmg_stats st;
    memset(&st, 0, sizeof(st));
    st.levels = h->L;
    const unsigned long long* t = h->host_stamps;
    if (first == 0) st.setup_seconds = 1e-9 * (double)(t[1] - t[0]);
    for (int l = 0; l < h->L; ++l) {
        const SolveState& s = h->host_states[l];
        if (l < first) continue;
        st.seconds[l] = 1e-9 * (double)(t[2 + l] - t[1 + l]);
        st.iters[l] = s.iters;
        st.updates[l] = s.updates;
        st.rhs_norm[l] = std::sqrt(s.fh2);
        const bool have_true = h->opt.true_residual || (h->opt.precision == ECMG_MIXED && l >= 2);
        const double rr = have_true ? s.rr_true : s.rr;
        st.rel_res[l] = s.fh2 > 0 ? std::sqrt(rr / s.fh2) : std::sqrt(rr);
        ecmg_status ls = ECMG_OK;
        if (s.status == 3) ls = ECMG_ERR_NO_CONVERGENCE;
        if (s.status == 4) ls = ECMG_ERR_BREAKDOWN;
        if (s.status == 5) ls = ECMG_ERR_CUDA;  // a staged copy of the FP32 stencil never arrived
        if (s.status == 6) ls = ECMG_ERR_CUDA;  // stale stencil path after a fresh recording (not expected)
        if (ls == ECMG_ERR_BREAKDOWN || (ls != ECMG_OK && worst == ECMG_OK)) worst = ls;
    }
    st.status = worst;
    if (stats) *stats = st;
    if (worst != ECMG_OK) g_last_error = ecmg_status_string(worst);
    return worst;
}

int resolve_level(ecmg_handle* h, int level) { return level < 0 ? h->L - 1 : level; }

// ---- batched solves ----------------------------------------------------------------------------
// Block table of one batched launch over the given items in one geometry.
BLaunch make_launch(const Batch& B, const std::vector<int>& ids, BGeom geo)
{
    BLaunch L{};
    L.n = (int)ids.size();
    int acc = 0;
    for (int s = 0; s < L.n; ++s) {
        L.id[s] = ids[s];
        L.start[s] = acc;
        acc += bgeom_blocks(geo, B.items[ids[s]]);
    }
    L.start[L.n] = acc;
    return L;
}

// Block table of one batched launch of the TMA-staged K1 (ry node rows per thread, each item's
// own planes per block).
BLaunch make_launch_k1(const Batch& B, const std::vector<int>& ids, int ry)
{
    BLaunch L{};
    L.n = (int)ids.size();
    int acc = 0;
    for (int s = 0; s < L.n; ++s) {
        L.id[s] = ids[s];
        L.start[s] = acc;
        acc += bk1_blocks(B.items[ids[s]], ry);
    }
    L.start[L.n] = acc;
    return L;
}

// Items of the set-up at depth d (d = 0: every problem's finest level).
std::vector<int> depth_items(const Batch& B, int d)
{
    std::vector<int> ids;
    for (int p = 0; p < B.n; ++p)
        if (B.L[p] - 1 - d >= 0) ids.push_back(B.item(p, B.L[p] - 1 - d));
    return ids;
}

// Items of stage s: problem p works on level s - (Lmax - L_p), levels aligned at the finest.
std::vector<int> stage_items(const Batch& B, int s, int lmin = 0)
{
    std::vector<int> ids;
    for (int p = 0; p < B.n; ++p) {
        const int l = s - (B.Lmax - B.L[p]);
        if (l >= lmin && l < B.L[p]) ids.push_back(B.item(p, l));
    }
    return ids;
}

bool any_state(ecmg_handle* h, const std::vector<int>& ids, bool need_update)
{
    Batch& B = *h->batch;
    ck(cudaMemcpyAsync(B.host_states, B.states, sizeof(SolveState) * B.items.size(), cudaMemcpyDeviceToHost,
                       h->user_stream));
    ck(cudaStreamSynchronize(h->user_stream));
    for (int id : ids) {
        const SolveState& st = B.host_states[id];
        if (!st.done && (!need_update || st.need_update)) return true;
    }
    return false;
}

void record_batched(Rec& R)
{
    ecmg_handle* h = R.h;
    Batch& B = *h->batch;
    const ecmg_options& o = h->opt;
    const BItem* items = B.d_items;
    // compact inputs: beta, the load and g_D of the finest level assembled per problem first
    for (int p = 0; p < B.n; ++p) {
        const ecmg_problem& pr = B.probs[p];
        const BItem& it = B.items[B.item(p, B.L[p] - 1)];
        if (!pr.beta) fill_beta(it.g, pr.beta_const, it.beta, R.s());
        if (pr.f_mode == ECMG_F_SEPARABLE) sep_load_finest(it.g, pr.f_terms, pr.f, B.Hf[p], it.b, R.s());
        if (pr.gD_terms > 0) sep_nodal(it.g, pr.gD_terms, pr.g_D, it.gD, R.s());
    }
    for (int d = 0; d < B.Lmax; ++d) {
        const std::vector<int> ids = depth_items(B, d);
        blaunch_setup(items, make_launch(B, ids, BG_NODES), make_launch(B, ids, BG_ELEMS), R.s());
    }
    for (int s = 0; s < B.Lmax; ++s) {
        const std::vector<int> ids = stage_items(B, s), ids2 = stage_items(B, s, 2);
        if (ids.empty()) continue;
        blaunch_level_start(items, make_launch(B, ids, BG_ONE), make_launch(B, ids, BG_NODES),
                            make_launch(B, ids, BG_ROWS), B.robin, B.cube, o.inner_rtol, R.s());
        blaunch_guess(items, make_launch(B, ids2, BG_EXPF), make_launch(B, ids, BG_FLAT), o.exp_variant, R.s());
        const BLaunch stencil = make_launch(B, ids, BG_STENCIL), flat = make_launch(B, ids, BG_SPAN),
                      fine = make_launch(B, ids, BG_SPAN_FINE);
        const int ry = B.stage_ry[s];
        const BLaunch k1 = make_launch_k1(B, ids, ry);
        if (B.sp) {
            // single-pass steps: step `half` reads buffer set `half` (A: r32, q32, pA32; B: r32B,
            // q32B, pB32) and writes the other; a replacement folds the other set's p and writes
            // its residual there, where the next step reads it
            if (R.graph) {
                const cudaGraphConditionalHandle loop = R.new_handle();
                blaunch_absmax(items, fine, R.s());
                blaunch_res(items, stencil, B.robin, B.cube, RES_INIT, B.ctl, CondHandles{loop, 0, 1}, R.s(), 0);
                R.open(loop, cudaGraphCondTypeWhile);
                for (int half = 0; half < 2; ++half) {
                    const int o = half ^ 1;
                    const cudaGraphConditionalHandle upd = R.new_handle();  // on the loop body
                    blaunch_step_tma(items, B.d_maps, k1, ry, B.robin, B.cube, half, o, B.ctl, CondHandles{loop, upd, 1},
                                     R.s());
                    R.open(upd, cudaGraphCondTypeIf);
                    blaunch_fold(items, fine, o, R.s());
                    blaunch_res(items, stencil, B.robin, B.cube, RES_REPLACE, B.ctl, CondHandles{loop, 0, 1}, R.s(), o);
                    R.close();
                }
                R.close();
            } else {
                const CondHandles none{0, 0, 0};
                blaunch_absmax(items, fine, R.s());
                blaunch_res(items, stencil, B.robin, B.cube, RES_INIT, B.ctl, none, R.s(), 0);
                int half = 0;
                while (any_state(h, ids, false)) {
                    const int o = half ^ 1;
                    blaunch_step_tma(items, B.d_maps, k1, ry, B.robin, B.cube, half, o, B.ctl, none, R.s());
                    if (any_state(h, ids, true)) {
                        blaunch_fold(items, fine, o, R.s());
                        blaunch_res(items, stencil, B.robin, B.cube, RES_REPLACE, B.ctl, none, R.s(), o);
                    }
                    half = o;
                }
            }
        } else if (R.graph) {
            const cudaGraphConditionalHandle loop = R.new_handle();
            blaunch_absmax(items, fine, R.s());
            blaunch_res(items, stencil, B.robin, B.cube, RES_INIT, B.ctl, CondHandles{loop, 0, 1}, R.s());
            R.open(loop, cudaGraphCondTypeWhile);
            for (int half = 0; half < 2; ++half) {
                const cudaGraphConditionalHandle upd = R.new_handle();  // on the loop body
                blaunch_pq_tma(items, B.d_maps, k1, ry, B.robin, B.cube, half, half ? 0 : 1, R.s());
                blaunch_update(items, flat, B.ctl, CondHandles{loop, upd, 1}, R.s());
                R.open(upd, cudaGraphCondTypeIf);
                blaunch_fold(items, fine, half ? 0 : 1, R.s());
                blaunch_res(items, stencil, B.robin, B.cube, RES_REPLACE, B.ctl, CondHandles{loop, 0, 1}, R.s());
                R.close();
            }
            R.close();
        } else {
            const CondHandles none{0, 0, 0};
            blaunch_absmax(items, fine, R.s());
            blaunch_res(items, stencil, B.robin, B.cube, RES_INIT, B.ctl, none, R.s());
            int half = 0;
            while (any_state(h, ids, false)) {
                blaunch_pq_tma(items, B.d_maps, k1, ry, B.robin, B.cube, half, half ? 0 : 1, R.s());
                blaunch_update(items, flat, B.ctl, none, R.s());
                if (any_state(h, ids, true)) {
                    blaunch_fold(items, fine, half ? 0 : 1, R.s());
                    blaunch_res(items, stencil, B.robin, B.cube, RES_REPLACE, B.ctl, none, R.s());
                }
                half ^= 1;
            }
        }
        blaunch_exp_true(items, make_launch(B, ids2, BG_EXPT), R.s());
    }
}

ecmg_status run_batched(ecmg_handle* h, double* const* u_out, ecmg_stats* stats)
{
    Batch& B = *h->batch;
    std::vector<double*> outs;
    if (u_out) {
        for (int p = 0; p < B.n; ++p) {
            outs.push_back(u_out[p] ? resolve_array(u_out[p]) : nullptr);
            if (u_out[p] && !outs.back())
                return fail(ECMG_ERR_INVALID_ARG,
                            "u_out entries must be device memory of the current device or page-locked host memory");
        }
    }
    try {
        if (h->opt.use_graph) {
            if (!h->exec) {
                Rec R{h, true, 0};
                ck(cudaStreamBeginCapture(h->cap[0], cudaStreamCaptureModeThreadLocal));
                try {
                    record_batched(R);
                } catch (...) {
                    cudaGraph_t junk;
                    cudaStreamEndCapture(h->cap[0], &junk);
                    if (junk) cudaGraphDestroy(junk);
                    throw;
                }
                ck(cudaStreamEndCapture(h->cap[0], &h->graph));
                ck(cudaGraphInstantiate(&h->exec, h->graph, 0));
            }
            ck(cudaGraphLaunch(h->exec, h->user_stream));
        } else {
            Rec R{h, false, 0};
            record_batched(R);
        }
        for (int p = 0; p < (int)outs.size(); ++p)
            if (outs[p]) {
                const BItem& it = B.items[B.item(p, B.L[p] - 1)];
                unpack_nodal(it.g, it.U, outs[p], h->user_stream);
            }
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(B.host_states, B.states, sizeof(SolveState) * B.items.size(), cudaMemcpyDeviceToHost,
                           h->user_stream));
        ck(cudaStreamSynchronize(h->user_stream));
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(f.e));
    }
    ecmg_status worst = ECMG_OK;
    for (int p = 0; p < B.n; ++p) {
        ecmg_stats st;
        memset(&st, 0, sizeof(st));
        st.levels = B.L[p];
        ecmg_status pw = ECMG_OK;
        for (int l = 0; l < B.L[p]; ++l) {
            const SolveState& s = B.host_states[B.item(p, l)];
            st.iters[l] = s.iters;
            st.updates[l] = s.updates;
            st.rhs_norm[l] = std::sqrt(s.fh2);
            st.rel_res[l] = s.fh2 > 0 ? std::sqrt(s.rr_true / s.fh2) : std::sqrt(s.rr_true);
            ecmg_status ls = ECMG_OK;
            if (s.status == 3) ls = ECMG_ERR_NO_CONVERGENCE;
            if (s.status == 4) ls = ECMG_ERR_BREAKDOWN;
            if (ls == ECMG_ERR_BREAKDOWN || (ls != ECMG_OK && pw == ECMG_OK)) pw = ls;
        }
        st.status = pw;
        if (stats) stats[p] = st;
        if (pw == ECMG_ERR_BREAKDOWN || (pw != ECMG_OK && worst == ECMG_OK)) worst = pw;
    }
    if (worst != ECMG_OK) g_last_error = ecmg_status_string(worst);
    return worst;
}


// True when the level has one beta (device flag of the last set-up) and every face Dirichlet:
// the FP32 stencil and update kernels then take their constant-coefficient paths.
bool constant_coefficient(ecmg_handle* h, const Level& v)
{
    for (int f = 0; f < 6; ++f)
        if (v.op.bc[f] != 0) return false;
    int flag = 0;
    ck(cudaMemcpyAsync(&flag, v.uniform, sizeof(int), cudaMemcpyDeviceToHost, h->user_stream));
    ck(cudaStreamSynchronize(h->user_stream));
    return flag != 0;
}

// Forget the recorded graph (it holds launch shapes that no longer apply).
void drop_graph(ecmg_handle* h)
{
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    h->graph_first = -1;
}

// Mean milliseconds of `reps` launches of one kernel on level l (CUDA events on the handle's
// stream, one untimed launch first), on a scratch level state that no solve uses.
double time_launches(ecmg_handle* h, int l, int which, int reps)
{
    Level& v = h->lv[l];
    SolveState* st = h->states + (MAX_LEVELS - 1);
    SolveState tmpl = {};
    tmpl.rho = 1.0;
    tmpl.beta = 0.5;
    tmpl.alpha = 1e-30;
    tmpl.alpha_prev = 1e-30;
    tmpl.max_iters = 1 << 30;
    tmpl.thresh2 = -1.0;
    tmpl.inner2 = -1.0;
    cudaStream_t s = h->user_stream;
    const CondHandles none{0, 0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double total = 0.0;
    try {
        // the fixed-point scale of the level's load (constant-coefficient residual) from its last solve
        SolveState last;
        ck(cudaMemcpyAsync(&last, h->states + l, sizeof(last), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        tmpl.bcbits = last.bcbits;
        const bool cc = (which == 0 || which == 2 || which == 9 || which == 11) && constant_coefficient(h, v);
        // a level that runs the ring: K1 reads p_old from slot 0 and writes slot 1; the fold adds
        // the largest pending set a solve can hold
        const bool ring_on = v.ring && cc && (which == 0 || which == 9);
        if (ring_on) {
            tmpl.pring = v.R;
            tmpl.pend = which == 9 ? ring_cap(v.R) : 0;
        }
        const RingArgs ring{v.ring, v.ring_alpha, v.R};
        ck(cudaEventCreate(&e0));
        ck(cudaEventCreate(&e1));
        for (int rep = 0; rep <= reps; ++rep) {
            ck(cudaMemcpyAsync(st, &tmpl, sizeof(tmpl), cudaMemcpyHostToDevice, s));
            ck(cudaEventRecord(e0, s));
            switch (which) {
            case 0:
                launch_pq32_tma(v.maps, 0, v.k1, v.g, v.op, cc, v.uniform, v.beta32, v.dinv32, v.pB32, v.q32, v.e32, st,
                                h->part, 1, none, nullptr, s, ring_on ? &ring : nullptr);
                break;
            case 1: launch_update32(v.g, v.op, v.uniform, v.r32, v.q32, v.dinv32, st, h->part, none, s); break;
            case 2: {
                Level lv = v;
                lv.cc = cc;
                res32(h, lv, st, RES_REPORT, none, s);
                break;
            }
            case 3: launch_pq64(v.g, v.op, v.beta, v.uniform, v.r, v.dinv, v.pA, v.pB, v.q, v.Ut, st, h->part, 1, none, s); break;
            case 4: launch_update64(v.g, v.r, v.q, v.dinv, st, h->part, none, s); break;
            case 5: launch_res64(v.g, v.op, v.beta, v.uniform, v.U, v.b, v.dinv, v.r, st, h->part, RES_REPORT, none, s); break;
            case 6: {
                const Level& u1 = h->lv[l - 1];
                const Level& u0 = h->lv[l - 2];
                launch_exp_finite(h->opt.exp_variant, v.g, v.op, u1.g, u1.U, u0.g, u0.U, v.r, v.q, s);
                break;
            }
            case 7: {
                const Level& u1 = h->lv[l - 1];
                launch_exp_true(v.g, v.U, u1.g, u1.U, v.Ut, s, h->lv[l - 1].q);
                break;
            }
            case 8:  // as a MIXED solve runs it: with b / c on a constant-coefficient level
                launch_fh2(v.g, v.op, v.beta, v.U, v.b, st, h->part, s, v.r32 ? v.uniform : nullptr, v.r32 ? v.r : nullptr);
                break;
            case 9:
                if (ring_on) launch_fold_ring(v.g, v.Ut, ring, v.e32, v.uniform, st, h->part, s);
                else launch_fold32(v.g, v.Ut, v.e32, v.pA32, v.uniform, st, h->part, s);
                break;
            case 11:
                launch_step32(v.maps, 0, v.k1, v.g, v.op, cc, v.uniform, v.beta32, v.dinv32, v.pB32, v.q32B, v.r32B,
                              v.e32, st, h->part, 1, none, nullptr, s);
                break;
            default: launch_absmax(v.g, v.U, v.uniform, nullptr, 0, h->part, s); break;
            }
            ck(cudaEventRecord(e1, s));
            ck(cudaEventSynchronize(e1));
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) total += ms;
        }
        ck(cudaGetLastError());
    } catch (CudaFail&) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return total / reps;
}

// Levels below this many nodes keep the heuristic shape: their stencil time is launch-bound.
constexpr int64_t AUTOTUNE_MIN_NODES = 1 << 18;

// Time every candidate tile shape of the FP32 stencil kernel on each MIXED level that is large
// enough, and keep the fastest (ties keep the earlier candidate, so the choice is repeatable
// when timings agree).
// ---- batched K1 tile shapes ------------------------------------------------------------------
// Mean milliseconds of `reps` launches of the batched K1 (which 0) or K2 (which 1) over the items
// `ids` (CUDA events on the handle's stream, one untimed launch first). Before every launch each
// item's state is set to a running step with a tiny non-zero deferred step, so that K1 stages
// and writes e as inside a solve; no solve state survives (the next solve starts afresh).
double time_batch_launch(ecmg_handle* h, const std::vector<int>& ids, int which, int ry, int reps)
{
    Batch& B = *h->batch;
    cudaStream_t s = h->user_stream;
    SolveState tmpl = {};
    tmpl.rho = 1.0;
    tmpl.beta = 0.5;
    tmpl.alpha = 1e-30;
    tmpl.alpha_prev = 1e-30;
    tmpl.max_iters = 1 << 30;
    tmpl.thresh2 = -1.0;
    tmpl.inner2 = -1.0;
    const size_t ni = B.items.size();
    const BLaunch k1 = make_launch_k1(B, ids, ry), flat = make_launch(B, ids, BG_SPAN),
                  fine = make_launch(B, ids, BG_SPAN_FINE);
    const CondHandles none{0, 0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double total = 0.0;
    try {
        ck(cudaEventCreate(&e0));
        ck(cudaEventCreate(&e1));
        for (int rep = 0; rep <= reps; ++rep) {
            ck(cudaStreamSynchronize(s));  // the pinned staging array is refilled below
            for (size_t i = 0; i < ni; ++i) B.host_states[i] = tmpl;
            ck(cudaMemcpyAsync(B.states, B.host_states, sizeof(SolveState) * ni, cudaMemcpyHostToDevice, s));
            ck(cudaEventRecord(e0, s));
            if (which == 0) blaunch_pq_tma(B.d_items, B.d_maps, k1, ry, B.robin, B.cube, 0, 1, s);
            else if (which == 11) blaunch_step_tma(B.d_items, B.d_maps, k1, ry, B.robin, B.cube, 0, 1, B.ctl, none, s);
            else if (which == 2) {
                // the FP64 residual of every item (its max |x| first), into r, reported only
                blaunch_absmax(B.d_items, fine, s);
                blaunch_res(B.d_items, make_launch(B, ids, BG_STENCIL), B.robin, B.cube, RES_REPORT, B.ctl, none, s);
            } else blaunch_update(B.d_items, flat, B.ctl, none, s);
            ck(cudaEventRecord(e1, s));
            ck(cudaEventSynchronize(e1));
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) total += ms;
        }
        ck(cudaGetLastError());
    } catch (CudaFail&) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return total / reps;
}

void upload_items(ecmg_handle* h)
{
    Batch& B = *h->batch;
    ck(cudaMemcpyAsync(B.d_items, B.items.data(), sizeof(BItem) * B.items.size(), cudaMemcpyHostToDevice,
                       h->user_stream));
    ck(cudaStreamSynchronize(h->user_stream));
}

// Autotuner of the batched K1: per stage, first one shape for every item (ry in {1, 2} x planes
// per block in {4, 8, 16, 32, 64}), timed as the stage's whole launch; then, with the others
// fixed, the planes per block of each size class (items whose z extent has the same power of
// two), again by the time of the whole launch.
void batch_autotune(ecmg_handle* h, int reps)
{
    Batch& B = *h->batch;
    const int kzs[5] = {4, 8, 16, 32, 64};
    for (int s = 0; s < B.Lmax; ++s) {
        const std::vector<int> ids = stage_items(B, s);
        if (ids.empty()) continue;
        auto set_kz = [&](const std::vector<int>& which, int kz) {
            for (int id : which) B.items[id].k1kz = kz;
        };
        int best_ry = B.stage_ry[s], best_kz = B.items[ids[0]].k1kz;
        double best = 1e300;
        for (int ry = 1; ry <= 2; ++ry)
            for (int kz : kzs) {
                set_kz(ids, kz);
                upload_items(h);
                const double ms = time_batch_launch(h, ids, B.sp ? 11 : 0, ry, reps);
                if (ms < best) {
                    best = ms;
                    best_ry = ry;
                    best_kz = kz;
                }
            }
        B.stage_ry[s] = best_ry;
        set_kz(ids, best_kz);
        std::vector<std::vector<int>> classes(32);
        for (int id : ids) {
            int c = 0;
            while ((1 << c) < B.items[id].g.nz + 1) ++c;
            classes[c].push_back(id);
        }
        int nclass = 0;
        for (const auto& c : classes) nclass += c.empty() ? 0 : 1;
        if (nclass > 1)
            for (const auto& c : classes) {
                if (c.empty()) continue;
                int ckz = best_kz;
                for (int kz : kzs) {
                    if (kz == best_kz) continue;
                    set_kz(c, kz);
                    upload_items(h);
                    const double ms = time_batch_launch(h, ids, B.sp ? 11 : 0, best_ry, reps);
                    if (ms < best) {
                        best = ms;
                        ckz = kz;
                    }
                }
                set_kz(c, ckz);
            }
        upload_items(h);
    }
    drop_graph(h);
}

// Tile shape of the FP32 stencil kernel (K1, or the single-pass step) per level: every candidate
// shape is set on all tuned levels at once (their kernels do not interact), the whole solve runs
// `reps` times, and each level keeps the shape of its shortest level time (device time stamps).
// Inside the solve a level's kernels meet the cache state the kernels before them leave (K1
// after K2 or after a replacement), which a kernel timed alone does not: alone, the 256^3 level
// of the cos_cube benchmark preferred 128 planes per block, inside the solve 16 (16.6 against
// 15.3 ms).
void autotune(ecmg_handle* h, int reps)
{
    if (h->batch) {
        batch_autotune(h, reps);
        return;
    }
    // the tuned levels: MIXED levels of at least AUTOTUNE_MIN_NODES nodes
    std::vector<int> lv;
    for (int l = 2; l < h->L; ++l) {
        const Level& v = h->lv[l];
        if (v.r32 && (int64_t)(v.g.nx + 1) * (v.g.ny + 1) * (v.g.nz + 1) >= AUTOTUNE_MIN_NODES) lv.push_back(l);
    }
    if (lv.empty()) return;
    const int nl = (int)lv.size();
    // level seconds of the fastest of `reps` whole solves with the shapes now set (device time
    // stamps) and the levels' iteration counts; false when a solve did not succeed
    std::vector<double> t(nl);
    std::vector<int> it(nl);
    auto measure = [&]() -> bool {
        drop_graph(h);
        std::fill(t.begin(), t.end(), INFINITY);
        for (int r = 0; r < reps; ++r) {
            ecmg_stats st;
            if (run_solve(h, 0, nullptr, &st) != ECMG_OK) return false;
            for (int i = 0; i < nl; ++i) {
                t[i] = std::min(t[i], st.seconds[lv[i]]);
                it[i] = st.iters[lv[i]];
            }
        }
        return true;
    };
    std::vector<K1Config> best(nl);
    std::vector<double> best_t(nl, INFINITY);
    std::vector<int> it0(nl, 0);
    for (int i = 0; i < nl; ++i) best[i] = h->lv[lv[i]].k1;
    if (measure()) {
        best_t = t;
        it0 = it;
    }
    K1Config cand[32];
    const int n = k1_candidates(h->lv[lv[0]].g, cand, 32);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < nl; ++i) h->lv[lv[i]].k1 = cand[c];
        if (!measure()) continue;
        for (int i = 0; i < nl; ++i) {
            // a shape sums p.q in another order, which can move a level's iteration count by a
            // step: compare per iteration, at the starting shape's count
            const double ti = (it[i] > 0 && it0[i] > 0) ? t[i] * it0[i] / it[i] : t[i];
            if (ti < best_t[i]) {
                best_t[i] = ti;
                best[i] = cand[c];
            }
        }
    }
    for (int i = 0; i < nl; ++i) h->lv[lv[i]].k1 = best[i];
    drop_graph(h);
    g_last_error.clear();
}

}  // namespace

extern "C" {

void ecmg_default_options(ecmg_options* o)
{
    if (!o) return;
    o->rtol = 1e-9;
    o->precision = ECMG_FP64;
    o->inner_rtol = 1e-3;
    o->max_iters = 100000;
    o->use_graph = 1;
    o->dsolve_rtol = 1e-14;
    o->exp_variant = ECMG_EXP_SERENDIPITY20;
    o->true_residual = 1;
    o->autotune = 0;
    o->preconditioner = ECMG_PREC_JACOBI;
    o->schedule = ECMG_SCHED_TOLERANCE;
    o->sched_mL = 4;
    o->sched_beta = 4.0;
    o->cg_form = ECMG_CG_AUTO;
    o->ring_slots = ECMG_RING_AUTO;
}

namespace {

// Bytes of a single-problem handle's workspace (the arithmetic of ecmg_create's allocations),
// with o.ring_slots already a slot count.
uint64_t workspace_of(const ecmg_problem* p, const ecmg_options& o)
{
    uint64_t b = 0;
    int maxb = 0;
    for (int l = 0; l < p->levels; ++l) {
        Grid g = make_grid(*p, l);
        b += level_bytes(g, o.precision == ECMG_MIXED, single_pass_level(o, g, l), ring_slots_level(*p, o, g, l));
        if (p->f_mode == ECMG_F_SEPARABLE) b += 8ull * (uint64_t)sep_factor_len(g, p->f_terms);
        if (p->gD_terms > 0 && l < p->levels - 1) b += 8ull * (uint64_t)sep_factor_len(g, p->gD_terms);
        maxb = std::max(maxb, std::max(max_stencil_blocks(g), max_stream_blocks()));
        if (o.precision == ECMG_MIXED) maxb = std::max(maxb, std::max(max_tma_blocks(g), res_cc_blocks(g)));
    }
    return b + (uint64_t)maxb * partials_per_block(o) * 8 + (uint64_t)max_stream_blocks() * 8 + 8 +
           sizeof(SolveState) * MAX_LEVELS + 1024 * 2 * 8;
}

// The slot count of ring_slots: ECMG_RING_AUTO takes 64 when the workspace with them stays
// within 3/4 of the current device's total memory, else the most slots (>= 8) that do, else 0
// (also when no device answers). A ring of R slots moves 4 + 8 / (R - 2) bytes per node and step
// for the correction (the directions read once, e read and written once per R - 2 steps) against
// 8 without a ring; 8 slots keep most of that gain.
int resolve_ring_slots(const ecmg_problem* p, const ecmg_options& o)
{
    if (o.ring_slots != ECMG_RING_AUTO) return o.ring_slots;
    ecmg_options z = o;
    z.ring_slots = 0;
    const uint64_t base = workspace_of(p, z);
    z.ring_slots = 1;
    const uint64_t per_slot = workspace_of(p, z) - base;
    if (per_slot == 0) return 0;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const uint64_t budget = (uint64_t)prop.totalGlobalMem / 4 * 3;
    if (budget <= base) return 0;
    const uint64_t r = std::min<uint64_t>(64, (budget - base) / per_slot);
    return r >= 8 ? (int)r : 0;
}

}  // namespace

ecmg_status ecmg_workspace_bytes(const ecmg_problem* p, const ecmg_options* o, uint64_t* bytes)
{
    ecmg_status s = validate(p, o);
    if (s != ECMG_OK) return s;
    if (!bytes) return fail(ECMG_ERR_INVALID_ARG, "bytes is null");
    ecmg_options r = *o;
    r.ring_slots = resolve_ring_slots(p, *o);
    *bytes = workspace_of(p, r);
    return ECMG_OK;
}

ecmg_status ecmg_create(const ecmg_problem* prob, const ecmg_options* opt, void* stream,
                        ecmg_handle** out)
{
    return ecmg_create_with_allocator(prob, opt, stream, nullptr, nullptr, nullptr, out);
}

ecmg_status ecmg_create_with_allocator(const ecmg_problem* prob, const ecmg_options* opt, void* stream,
                                       ecmg_alloc_fn alloc, ecmg_free_fn free_fn, void* ctx, ecmg_handle** out)
{
    if (!out) return fail(ECMG_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(ECMG_ERR_INVALID_ARG, "alloc and free go together");
    ecmg_status s = validate(prob, opt);
    if (s != ECMG_OK) return s;
    ecmg_problem pr = *prob;
    if (!resolve_inputs(&pr))
        return fail(ECMG_ERR_INVALID_ARG, "inputs must be device memory of the current device or page-locked host memory");
    ecmg_handle* h = new ecmg_handle();
    h->alloc_fn = alloc;
    h->free_fn = free_fn;
    h->alloc_ctx = ctx;
    h->prob = pr;
    h->opt = *opt;
    h->opt.ring_slots = resolve_ring_slots(&pr, *opt);
    h->user_stream = (cudaStream_t)stream;
    h->L = prob->levels;
    try {
        for (int i = 0; i < 3; ++i) ck(cudaStreamCreateWithFlags(&h->cap[i], cudaStreamNonBlocking));
        ck(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        ck(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        for (auto& e : h->ev_level) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&h->ev_out_fork, cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&h->ev_out_join, cudaEventDisableTiming));
        const bool mixed = opt->precision == ECMG_MIXED;
        if (mixed) {
            ck(k1_prepare());
            ck(res_cc_prepare());
        }
        int maxb = 0;
        for (int l = 0; l < h->L; ++l) {
            Level& v = h->lv[l];
            v.g = make_grid(*prob, l);
            v.op = make_op(v.g.h, prob->face_bc, prob->robin_alpha);
            const int64_t n = v.g.total;
            v.U = dalloc<double>(h, n);
            v.W = dalloc<double>(h, n);
            v.Ut = dalloc<double>(h, n);
            v.b = dalloc<double>(h, n);
            v.beta = dalloc<double>(h, n);
            v.dinv = dalloc<double>(h, n);
            v.f = dalloc<double>(h, n);
            v.gD = dalloc<double>(h, n);
            v.gR = dalloc<double>(h, n);
            v.r = dalloc<double>(h, n);
            v.pA = dalloc<double>(h, n);
            v.pB = dalloc<double>(h, n);
            v.q = dalloc<double>(h, n);
            if (prob->f_mode == ECMG_F_SEPARABLE) v.Hf = dalloc<double>(h, sep_factor_len(v.g, prob->f_terms));
            if (prob->gD_terms > 0 && l < h->L - 1) v.Hg = dalloc<double>(h, sep_factor_len(v.g, prob->gD_terms));
            if (mixed) {
                v.beta32 = dalloc<float>(h, n);
                v.dinv32 = dalloc<float>(h, n);
                v.r32 = dalloc<float>(h, n);
                v.pA32 = dalloc<float>(h, n);
                v.pB32 = dalloc<float>(h, n);
                v.q32 = dalloc<float>(h, n);
                v.e32 = dalloc<float>(h, n);
                if (!make_plane_maps(&v.maps, v.r32, v.pA32, v.pB32, v.dinv32, v.beta32, v.e32, v.g) ||
                    !make_res_maps(&v.rmaps, v.U, v.r, v.g))
                    throw CudaFail{cudaErrorNotSupported};
                if (single_pass_level(*opt, v.g, l)) {
                    v.r32B = dalloc<float>(h, n);
                    v.q32B = dalloc<float>(h, n);
                    if (!make_plane_maps_sp(&v.maps, v.r32B, v.q32, v.q32B, v.g)) throw CudaFail{cudaErrorNotSupported};
                }
                if (const int R = ring_slots_level(h->prob, h->opt, v.g, l)) {
                    v.R = R;
                    v.ring = dalloc<float>(h, ring_stride(n) * R);
                    v.ring_alpha = dalloc<double>(h, R);
                    if (!make_ring_maps(&v.maps, v.ring, R, v.g)) throw CudaFail{cudaErrorNotSupported};
                }
                v.k1 = k1_default(v.g, v.op);
                maxb = std::max(maxb, std::max(max_tma_blocks(v.g), res_cc_blocks(v.g)));
            }
            maxb = std::max(maxb, std::max(max_stencil_blocks(v.g), max_stream_blocks()));
        }
        h->part.buf = dalloc<double>(h, (int64_t)maxb * partials_per_block(*opt));
        h->part.max_blocks = maxb;
        h->part.fs = dalloc<FixedScale>(h, 1);
        h->part_side.buf = dalloc<double>(h, max_stream_blocks());  // ||f_h||: one partial per block
        h->part_side.max_blocks = max_stream_blocks();
        h->out_slot = dalloc<double*>(h, 1);
        h->states = dalloc<SolveState>(h, MAX_LEVELS);
        h->timers = dalloc<KTimer>(h, MAX_LEVELS);
        {
            KTimer idle[MAX_LEVELS];
            for (auto& t : idle) t = KTimer{~0ull, 0ull, 0ull};
            ck(cudaMemcpyAsync(h->timers, idle, sizeof(idle), cudaMemcpyHostToDevice, h->cap[0]));
        }
        int* flags = dalloc<int>(h, MAX_LEVELS);
        for (int l = 0; l < h->L; ++l) h->lv[l].uniform = flags + l;
        h->norm_part = dalloc<double>(h, 2048);
        ck(cudaMallocHost(&h->host_states, sizeof(SolveState) * MAX_LEVELS));
        ck(cudaMallocHost(&h->host_norms, sizeof(double) * 2048));
        h->stamps = dalloc<unsigned long long>(h, MAX_LEVELS + 2);
        ck(cudaMallocHost(&h->host_stamps, sizeof(unsigned long long) * (MAX_LEVELS + 2)));
        ck(cudaStreamSynchronize(h->cap[0]));
        if (mixed && opt->autotune) autotune(h, 3);
    } catch (CudaFail& f) {
        ecmg_destroy(h);
        if (f.e == cudaErrorMemoryAllocation) return fail(ECMG_ERR_OOM, "device allocation failed");
        return fail(ECMG_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(f.e));
    }
    *out = h;
    return ECMG_OK;
}

ecmg_status ecmg_solve(ecmg_handle* h, double* u_out, ecmg_stats* stats)
{
    if (!h) return fail(ECMG_ERR_INVALID_ARG, "null handle");
    if (h->batch) return fail(ECMG_ERR_INVALID_ARG, "batched handle: use ecmg_solve_batched");
    return run_solve(h, 0, u_out, stats);
}

ecmg_status ecmg_create_batched(const ecmg_problem* probs, int32_t n, const ecmg_options* opt, void* stream,
                                ecmg_handle** out)
{
    if (!out || !probs || !opt) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n < 1 || n > BATCH_MAX) return fail(ECMG_ERR_INVALID_ARG, "batch size must be 1..128");
    if (opt->precision != ECMG_MIXED) return fail(ECMG_ERR_INVALID_ARG, "batched solves run in MIXED precision");
    for (int p = 0; p < n; ++p) {
        ecmg_status s = validate(probs + p, opt);
        if (s != ECMG_OK) return s;
    }
    std::vector<ecmg_problem> resolved(probs, probs + n);
    for (auto& q : resolved)
        if (!resolve_inputs(&q))
            return fail(ECMG_ERR_INVALID_ARG, "inputs must be device memory of the current device or page-locked host memory");
    probs = resolved.data();
    ecmg_handle* h = new ecmg_handle();
    h->prob = probs[0];
    h->opt = *opt;
    h->user_stream = (cudaStream_t)stream;
    h->L = 0;  // no single-problem levels
    h->batch = new Batch();
    Batch& B = *h->batch;
    B.n = n;
    B.sp = opt->cg_form == ECMG_CG_SINGLE_PASS;
    B.probs.assign(probs, probs + n);
    B.Hf.assign(n, nullptr);
    try {
        for (int i = 0; i < 3; ++i) ck(cudaStreamCreateWithFlags(&h->cap[i], cudaStreamNonBlocking));
        int nitems = 0;
        for (int p = 0; p < n; ++p) {
            B.L.push_back(probs[p].levels);
            B.first.push_back(nitems);
            nitems += probs[p].levels;
            B.Lmax = std::max(B.Lmax, probs[p].levels);
        }
        B.items.resize(nitems);
        B.states = dalloc<SolveState>(h, nitems);
        B.ctl = dalloc<BCtl>(h, 1);
        ck(cudaMallocHost(&B.host_states, sizeof(SolveState) * nitems));
        // vectors, finest first so that every level can point at its finer neighbour
        for (int p = 0; p < n; ++p) {
            const ecmg_problem& pr = probs[p];
            for (int l = pr.levels - 1; l >= 0; --l) {
                BItem& it = B.items[B.item(p, l)];
                it = BItem{};
                it.g = make_grid(pr, l);
                it.op = make_op(it.g.h, pr.face_bc, pr.robin_alpha);
                it.level = l;
                it.problem = p;
                it.depth = pr.levels - 1 - l;
                // separable f: the finest load is assembled before the batched set-up, and the
                // coarse ones are its restrictions, as for a given load functional
                it.fmode = pr.f_mode == ECMG_F_SEPARABLE ? ECMG_F_LOAD : pr.f_mode;
                if (it.depth == 0) {
                    it.pre_beta = pr.beta ? 0 : 1;
                    it.pre_load = pr.f_mode == ECMG_F_SEPARABLE ? 1 : 0;
                    it.pre_gD = pr.gD_terms > 0 ? 1 : 0;
                    if (pr.f_mode == ECMG_F_SEPARABLE) B.Hf[p] = dalloc<double>(h, sep_factor_len(it.g, pr.f_terms));
                }
                it.kz = std::min(8, it.g.nz + 1);  // short columns: a replacement often runs on one item alone
                it.k1kz = 16;
                it.fixed = (opt->schedule == ECMG_SCHED_FIXED && l >= 2) ? 1 : 0;
                it.rtol = l < 2 ? opt->dsolve_rtol : (it.fixed ? 0.0 : opt->rtol);
                it.max_iters = it.fixed ? schedule_steps(pr.levels, l, opt->sched_mL, opt->sched_beta) : opt->max_iters;
                it.precond = opt->preconditioner == ECMG_PREC_JACOBI ? 1 : 0;
                const int64_t nv = it.g.total;
                it.U = dalloc<double>(h, nv);
                it.W = dalloc<double>(h, nv);
                it.Ut = dalloc<double>(h, nv);
                it.b = dalloc<double>(h, nv);
                it.beta = dalloc<double>(h, nv);
                it.f = dalloc<double>(h, nv);
                it.gD = dalloc<double>(h, nv);
                it.gR = dalloc<double>(h, nv);
                it.beta32 = dalloc<float>(h, nv);
                it.dinv32 = dalloc<float>(h, nv);
                it.r32 = dalloc<float>(h, nv);
                it.pA32 = dalloc<float>(h, nv);
                it.pB32 = dalloc<float>(h, nv);
                it.q32 = dalloc<float>(h, nv);
                it.e32 = dalloc<float>(h, nv);
                if (B.sp) {
                    it.r32B = dalloc<float>(h, nv);
                    it.q32B = dalloc<float>(h, nv);
                }
                it.st = B.states + B.item(p, l);
                // 7 sums per block in the single-pass step on the general path
                it.part = dalloc<double>(h, (B.sp ? 8 : 2) * (int64_t)bitem_partials(it));
                if (it.depth == 0) {
                    it.in_beta = pr.beta;
                    it.in_f = pr.f;
                    it.in_gD = pr.g_D;
                    it.in_gR = pr.g_R;
                } else {
                    const BItem& fi = B.items[B.item(p, l + 1)];
                    it.gf = fi.g;
                    it.fbeta = fi.beta;
                    it.ff = fi.f;
                    it.fgD = fi.gD;
                    it.fgR = fi.gR;
                    it.fb = fi.b;
                }
                B.robin |= op_robin(it.op);
                B.cube &= it.op.cube;
            }
            for (int l = 2; l < pr.levels; ++l) {
                BItem& it = B.items[B.item(p, l)];
                const BItem& i1 = B.items[B.item(p, l - 1)];
                const BItem& i0 = B.items[B.item(p, l - 2)];
                it.g1 = i1.g;
                it.U1 = i1.U;
                it.g0 = i0.g;
                it.U0 = i0.U;
            }
        }
        // tensor maps of every item's FP32 vectors for the TMA-staged K1
        std::vector<PlaneMaps> maps(nitems);
        for (int i = 0; i < nitems; ++i) {
            const BItem& it = B.items[i];
            if (!make_plane_maps(&maps[i], it.r32, it.pA32, it.pB32, it.dinv32, it.beta32, it.e32, it.g))
                throw CudaFail{cudaErrorInvalidValue};
            if (B.sp && !make_plane_maps_sp(&maps[i], it.r32B, it.q32, it.q32B, it.g))
                throw CudaFail{cudaErrorInvalidValue};
        }
        B.d_maps = dalloc<PlaneMaps>(h, nitems);
        ck(cudaMemcpyAsync(B.d_maps, maps.data(), sizeof(PlaneMaps) * nitems, cudaMemcpyHostToDevice, h->cap[0]));
        B.stage_ry.assign(B.Lmax, 1);
        ck(bk1_prepare());
        B.d_items = dalloc<BItem>(h, nitems);
        ck(cudaMemcpyAsync(B.d_items, B.items.data(), sizeof(BItem) * nitems, cudaMemcpyHostToDevice, h->cap[0]));
        ck(cudaStreamSynchronize(h->cap[0]));
        if (opt->autotune) batch_autotune(h, 3);
    } catch (CudaFail& f) {
        ecmg_destroy(h);
        if (f.e == cudaErrorMemoryAllocation) return fail(ECMG_ERR_OOM, "device allocation failed");
        return fail(ECMG_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(f.e));
    }
    *out = h;
    return ECMG_OK;
}

ecmg_status ecmg_solve_batched(ecmg_handle* h, double* const* u_out, ecmg_stats* stats)
{
    if (!h || !h->batch) return fail(ECMG_ERR_INVALID_ARG, "not a batched handle");
    return run_batched(h, u_out, stats);
}

ecmg_status ecmg_get_level_batched(ecmg_handle* h, int32_t problem, int32_t level, int32_t which, double* out)
{
    if (!h || !h->batch || !out) return fail(ECMG_ERR_INVALID_ARG, "null argument or not a batched handle");
    Batch& B = *h->batch;
    if (problem < 0 || problem >= B.n) return fail(ECMG_ERR_INVALID_ARG, "bad problem index");
    const int l = level < 0 ? B.L[problem] - 1 : level;
    if (l < 0 || l >= B.L[problem]) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    const BItem& it = B.items[B.item(problem, l)];
    const double* src = nullptr;
    switch (which) {
    case ECMG_VEC_U: src = it.U; break;
    case ECMG_VEC_W: src = it.W; break;
    case ECMG_VEC_UTILDE:
        if (l < 2) return fail(ECMG_ERR_INVALID_ARG, "U~ exists on levels >= 2 only");
        src = it.Ut;
        break;
    case ECMG_VEC_B: src = it.b; break;
    default: return fail(ECMG_ERR_INVALID_ARG, "bad vector selector (U, W, U~ or B)");
    }
    unpack_nodal(it.g, src, out, h->user_stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ECMG_ERR_CUDA, cudaGetErrorString(e));
    return ECMG_OK;
}

ecmg_status ecmg_solve_from(ecmg_handle* h, int32_t first, double* u_out, ecmg_stats* stats)
{
    if (!h) return fail(ECMG_ERR_INVALID_ARG, "null handle");
    if (first < 2 || first >= h->L) return fail(ECMG_ERR_INVALID_ARG, "first must be in 2..levels-1");
    return run_solve(h, first, u_out, stats);
}

ecmg_status ecmg_extrapolate(ecmg_handle* h, int32_t level, double* u_tilde_out)
{
    return ecmg_get_level(h, level, ECMG_VEC_UTILDE, u_tilde_out);
}

ecmg_status ecmg_get_level(ecmg_handle* h, int32_t level, int32_t which, double* out)
{
    if (!h || !out) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    if (!(out = resolve_array(out)))
        return fail(ECMG_ERR_INVALID_ARG, "out must be device memory of the current device or page-locked host memory");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    Level& v = h->lv[l];
    const double* src = nullptr;
    switch (which) {
    case ECMG_VEC_U: src = v.U; break;
    case ECMG_VEC_W: src = v.W; break;
    case ECMG_VEC_UTILDE:
        if (l < 2) return fail(ECMG_ERR_INVALID_ARG, "U~ exists on levels >= 2 only");
        src = v.Ut;
        break;
    case ECMG_VEC_B: src = v.b; break;
    case ECMG_VEC_BETA: src = v.beta; break;
    default: return fail(ECMG_ERR_INVALID_ARG, "bad vector selector");
    }
    if (which == ECMG_VEC_BETA) {
        // element (i,j,k) sits at the node offset of its lowest corner; copy row by row
        for (int k = 0; k < v.g.nz; ++k)
            for (int j = 0; j < v.g.ny; ++j) {
                cudaError_t e = cudaMemcpyAsync(out + (size_t)v.g.nx * (j + (size_t)v.g.ny * k),
                                                src + v.g.off(0, j, k), (size_t)v.g.nx * 8,
                                                cudaMemcpyDefault, h->user_stream);
                if (e != cudaSuccess) return fail(ECMG_ERR_CUDA, cudaGetErrorString(e));
            }
        return ECMG_OK;
    }
    unpack_nodal(v.g, src, out, h->user_stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ECMG_ERR_CUDA, cudaGetErrorString(e));
    return ECMG_OK;
}

ecmg_status ecmg_set_level(ecmg_handle* h, int32_t level, const double* in)
{
    if (!h || !in) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    if (!(in = resolve_array(in))) return fail(ECMG_ERR_INVALID_ARG, "arrays must be device memory of the current device or page-locked host memory");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    pack_nodal(h->lv[l].g, in, h->lv[l].U, h->user_stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ECMG_ERR_CUDA, cudaGetErrorString(e));
    return ECMG_OK;
}

ecmg_status ecmg_apply_operator(ecmg_handle* h, int32_t level, int32_t precision, const double* x,
                                double* y)
{
    if (!h || !x || !y) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    if (!(x = resolve_array(x)) || !(y = resolve_array(y))) return fail(ECMG_ERR_INVALID_ARG, "arrays must be device memory of the current device or page-locked host memory");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    Level& v = h->lv[l];
    cudaStream_t s = h->user_stream;
    // x -> padded (into r), y <- padded (from q)
    pack_nodal(v.g, x, v.r, s);
    if (precision == ECMG_MIXED) {
        if (!v.r32) return fail(ECMG_ERR_INVALID_ARG, "handle was created without MIXED precision");
        convert_f32(v.r, v.r32, v.g.total, s);
        launch_apply32(v.g, v.op, v.beta32, v.r32, v.q, s);
    } else if (precision == ECMG_FP64) {
        launch_apply64(v.g, v.op, v.beta, v.uniform, v.r, v.q, h->part, s);
    } else if (precision == ECMG_APPLY_K1) {
        if (!v.r32) return fail(ECMG_ERR_INVALID_ARG, "handle was created without MIXED precision");
        // p = D^-1 r + beta p_old with r = 0, beta = 1: p = x; q = A p; alpha_prev = 0: e untouched
        bool cc = false;
        try {
            cc = constant_coefficient(h, v);
        } catch (CudaFail& f) {
            return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
        }
        // a level that runs the ring runs K1's ring form: p_old from slot 0, p into slot 1
        const bool ring_on = v.ring && cc;
        SolveState* st = h->states + (MAX_LEVELS - 1);
        SolveState tmpl = {};
        tmpl.rho = 1.0;
        tmpl.beta = 1.0;
        tmpl.alpha = 1.0;
        tmpl.max_iters = 1 << 30;
        tmpl.thresh2 = -1.0;
        tmpl.inner2 = -1.0;
        if (ring_on) tmpl.pring = v.R;
        const size_t n4 = (size_t)v.g.total * 4;
        const CondHandles none{0, 0, 0};
        cudaError_t e = cudaMemcpyAsync(st, &tmpl, sizeof(tmpl), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(v.r32, 0, n4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(v.q32, 0, n4, s);
        if (e != cudaSuccess) return fail(ECMG_ERR_CUDA, cudaGetErrorString(e));
        convert_f32(v.r, ring_on ? v.ring : v.pA32, v.g.total, s);
        const RingArgs ring{v.ring, v.ring_alpha, v.R};
        launch_pq32_tma(v.maps, 0, v.k1, v.g, v.op, cc, v.uniform, v.beta32, v.dinv32, v.pB32, v.q32, v.e32, st, h->part,
                        1, none, nullptr, s, ring_on ? &ring : nullptr);
        convert_f64(v.q32, v.q, v.g.total, s);
    } else {
        return fail(ECMG_ERR_INVALID_ARG, "bad precision");
    }
    unpack_nodal(v.g, v.q, y, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ECMG_ERR_CUDA, cudaGetErrorString(e));
    return ECMG_OK;
}

ecmg_status ecmg_error_norms(ecmg_handle* h, int32_t level, const double* a, const double* b,
                             double* max_abs, double* rms)
{
    if (!h || !a || !max_abs || !rms) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    if (!(a = resolve_array(a)) || (b && !(b = resolve_array(b)))) return fail(ECMG_ERR_INVALID_ARG, "arrays must be device memory of the current device or page-locked host memory");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    Level& v = h->lv[l];
    cudaStream_t s = h->user_stream;
    try {
        pack_nodal(v.g, a, v.r, s);
        if (b) pack_nodal(v.g, b, v.q, s);
        launch_norms(v.g, v.r, b ? v.q : nullptr, h->norm_part, s);
        const int nb = norms_blocks(v.g);
        ck(cudaMemcpyAsync(h->host_norms, h->norm_part, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        double mx = 0.0, ss = 0.0;
        for (int i = 0; i < nb; ++i) {
            const double m = h->host_norms[2 * i];
            mx = (std::isnan(m) || std::isnan(mx)) ? m + mx : std::max(mx, m);  // keeps a NaN
            ss += h->host_norms[2 * i + 1];
        }
        *max_abs = mx;
        *rms = std::sqrt(ss / (double)((int64_t)(v.g.nx + 1) * (v.g.ny + 1) * (v.g.nz + 1)));
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
    }
    return ECMG_OK;
}

void ecmg_destroy(ecmg_handle* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->user_stream);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (auto& a : h->allocs) {
        if (h->free_fn) h->free_fn(a.first, a.second, (void*)h->user_stream, h->alloc_ctx);
        else cudaFree(a.first);
    }
    if (h->batch) {
        if (h->batch->host_states) cudaFreeHost(h->batch->host_states);
        delete h->batch;
    }
    if (h->host_states) cudaFreeHost(h->host_states);
    if (h->host_norms) cudaFreeHost(h->host_norms);
    if (h->host_stamps) cudaFreeHost(h->host_stamps);
    for (int i = 0; i < 3; ++i)
        if (h->cap[i]) cudaStreamDestroy(h->cap[i]);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_out_fork) cudaEventDestroy(h->ev_out_fork);
    if (h->ev_out_join) cudaEventDestroy(h->ev_out_join);
    for (auto e : h->ev_level)
        if (e) cudaEventDestroy(e);
    delete h;
}

const char* ecmg_status_string(ecmg_status s)
{
    switch (s) {
    case ECMG_OK: return "ok";
    case ECMG_ERR_INVALID_ARG: return "invalid argument";
    case ECMG_ERR_SINGULAR: return "singular problem (no Dirichlet face and all Robin alpha = 0)";
    case ECMG_ERR_NO_CONVERGENCE: return "iteration cap reached before the tolerance";
    case ECMG_ERR_BREAKDOWN: return "JCG breakdown (p.q <= 0 or non-finite value)";
    case ECMG_ERR_OOM: return "device allocation failed";
    case ECMG_ERR_CUDA: return "CUDA runtime error";
    }
    return "unknown status";
}

const char* ecmg_last_error(void) { return g_last_error.c_str(); }

ecmg_status ecmg_kernel_launches(uint64_t* out)
{
    if (!out) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    *out = launches_setup() + launches_jcg() + launches_exp() + launches_pq_tma() + launches_pq_sp() + launches_batch() + launches_batch_tma() +
           launches_separable() + launches_res_cc();
    return ECMG_OK;
}

ecmg_status ecmg_time_kernel(ecmg_handle* h, int32_t level, int32_t which, int32_t reps,
                             double* ms_out, double* bytes_out)
{
    if (!h || !ms_out || !bytes_out || reps < 1) return fail(ECMG_ERR_INVALID_ARG, "bad argument");
    if (h->batch) {
        // batched handle: `level` is a stage (-1 = the last), the kernel its K1 (0) or K2 (1)
        // launch over every item of the stage
        Batch& B = *h->batch;
        const int s = level < 0 ? B.Lmax - 1 : level;
        if (s < 0 || s >= B.Lmax) return fail(ECMG_ERR_INVALID_ARG, "bad stage");
        if (which != 0 && which != 1 && which != 2 && which != 11)
            return fail(ECMG_ERR_INVALID_ARG, "batched handles time kernels 0, 1, 2 and 11");
        if (which != 2 && (which == 11) != B.sp)
            return fail(ECMG_ERR_INVALID_ARG, "kernel 11 on single-pass batches, 0 and 1 on two-pass ones");
        const std::vector<int> ids = stage_items(B, s);
        double bytes = 0.0;
        for (int id : ids) {
            const BItem& it = B.items[id];
            const double N = (double)(it.g.nx + 1) * (it.g.ny + 1) * (it.g.nz + 1);
            const double E = (double)it.g.nx * it.g.ny * it.g.nz;
            // K1 28 N_f + 4 E; K2 16 N; the residual reads x, b, beta, D^-1 and writes r (24 N + 8 E,
            // its max |x| pass 8 N more); the single-pass step 36 N_f + 4 E
            bytes += which == 0    ? 28.0 * (double)bk1_nodes(it) + 4.0 * E
                     : which == 1  ? 16.0 * N
                     : which == 2  ? 32.0 * N + 8.0 * E
                                   : 36.0 * (double)bk1_nodes(it) + 4.0 * E;
        }
        *bytes_out = bytes;
        try {
            *ms_out = time_batch_launch(h, ids, which, B.stage_ry[s], reps);
        } catch (CudaFail& f) {
            return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
        }
        return ECMG_OK;
    }
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    if (which < 0 || which > 11) return fail(ECMG_ERR_INVALID_ARG, "bad kernel selector");
    Level& v = h->lv[l];
    if (which == 11 && !v.r32B) return fail(ECMG_ERR_INVALID_ARG, "level has no single-pass buffers");
    if ((which <= 2 || which == 9) && !v.r32) return fail(ECMG_ERR_INVALID_ARG, "handle has no FP32 vectors");
    if (which >= 6 && l < 2) return fail(ECMG_ERR_INVALID_ARG, "EXP kernels need level >= 2");
    const double N = (double)(v.g.nx + 1) * (v.g.ny + 1) * (v.g.nz + 1);
    const double E = (double)v.g.nx * v.g.ny * v.g.nz;
    // K1 visits only the nodes off the Dirichlet faces (p = q = 0 there stay untouched). With one
    // beta on the level and every face Dirichlet (constant coefficient), K1 and K2 read no beta
    // and no D^-1.
    const double N1 = (double)k1_nodes(v.g, v.op);
    bool cc = false;
    try {
        cc = constant_coefficient(h, v);
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
    }
    // the constant-coefficient residual (kernel 2) reads x and b / c and writes r: 20 bytes per
    // node; ||f_h|| (8) reads b (and on a MIXED one-beta cube writes b / c on the nodes off the
    // faces); the fold (9) updates x and e and reads p; max |x| (10) reads x;
    // the single-pass step (11) moves r, q, p and e in and out (and D^-1, beta in)
    // with a ring of search directions K1 moves no correction vector (8 bytes fewer per node) and
    // the fold reads ring_slots - 2 directions instead of e and p and writes no e
    const bool ring_on = v.ring && cc;
    const double e1 = ring_on ? 0.0 : 8.0;
    const double bytes[12] = {(cc ? 16 + e1 : 20 + e1) * N1 + (cc ? 0.0 : 4 * E), (cc ? 12 * N : 16 * N),
                              (cc && v.op.cube ? 20 * N : 24 * N + 8 * E), 56 * N + 8 * E, 32 * N, 32 * N + 8 * E,
                              16 * N + 8 * (N / 8 + N / 64), 17 * N, (v.r32 && cc && v.op.cube) ? 8 * N + 8 * N1 : 8 * N,
                              ring_on ? (16.0 + 4.0 * ring_cap(v.R)) * N : 28 * N, 8 * N,
                              (cc ? 32 * N1 : 36 * N1 + 4 * E)};
    *bytes_out = bytes[which];
    try {
        *ms_out = time_launches(h, l, which, reps);
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
    }
    return ECMG_OK;
}

ecmg_status ecmg_set_tiles(ecmg_handle* h, int32_t level, int32_t ry, int32_t kz)
{
    if (!h) return fail(ECMG_ERR_INVALID_ARG, "null handle");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    if (!h->lv[l].r32) return fail(ECMG_ERR_INVALID_ARG, "handle has no FP32 vectors");
    const K1Config c{ry, kz};
    if (!k1_valid(c)) return fail(ECMG_ERR_INVALID_ARG, "tile shape: ry must be 1 or 2 and kz in 4..1024");
    h->lv[l].k1 = c;
    drop_graph(h);
    return ECMG_OK;
}

ecmg_status ecmg_get_tiles(ecmg_handle* h, int32_t level, int32_t* ry, int32_t* kz)
{
    if (!h || !ry || !kz) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    if (!h->lv[l].r32) return fail(ECMG_ERR_INVALID_ARG, "handle has no FP32 vectors");
    *ry = h->lv[l].k1.ry;
    *kz = h->lv[l].k1.kz;
    return ECMG_OK;
}

ecmg_status ecmg_stencil_timer(ecmg_handle* h, int32_t level, int32_t reset, double* ms_total,
                               int64_t* launches)
{
    if (!h || !ms_total || !launches) return fail(ECMG_ERR_INVALID_ARG, "null argument");
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return fail(ECMG_ERR_INVALID_ARG, "bad level");
    KTimer t{};
    try {
        ck(cudaMemcpyAsync(&t, h->timers + l, sizeof(t), cudaMemcpyDeviceToHost, h->user_stream));
        ck(cudaStreamSynchronize(h->user_stream));
        if (reset) {
            const KTimer idle{~0ull, 0ull, 0ull};
            ck(cudaMemcpyAsync(h->timers + l, &idle, sizeof(idle), cudaMemcpyHostToDevice, h->user_stream));
            ck(cudaStreamSynchronize(h->user_stream));
        }
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
    }
    *ms_total = (double)t.ns * 1e-6;
    *launches = (int64_t)t.n;
    return ECMG_OK;
}

ecmg_status ecmg_autotune(ecmg_handle* h, int32_t reps)
{
    if (!h || reps < 1) return fail(ECMG_ERR_INVALID_ARG, "bad argument");
    try {
        autotune(h, reps);
    } catch (CudaFail& f) {
        return fail(ECMG_ERR_CUDA, cudaGetErrorString(f.e));
    }
    return ECMG_OK;
}

}  // extern "C"
