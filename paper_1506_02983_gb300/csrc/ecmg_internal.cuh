// ecmg_internal.cuh -- shared definitions of the CUDA implementation of ECMG_jcg.
//
// Device data layout (every vector of a level, nodal or element, FP64 or FP32):
//   node (i, j, k), i in -1..nx+1 (one ghost layer on each side), is stored at
//       off(i, j, k) = (k + 1) * plane + (j + 1) * pitch + (i + XL)
//   with XL = 4 (so node i = 0 starts a 16-byte aligned run for both FP64 and FP32) and
//   pitch = round_up(nx + 1 + XL + 2, 8) elements (rows start on 32-byte sectors; every
//   stride is a multiple of 16 bytes, as TMA requires). Element (ex, ey, ez) of the level is
//   stored at the offset of its lowest corner node, so elements -1..nx are addressable and
//   the ghost elements hold beta = 0. Ghost entries are zero and are never written; a kernel
//   may therefore read the 27 neighbours of any owned node, and the 8 elements around it,
//   without bounds checks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ecmg {

constexpr int XL = 4;            // left pad in elements (16 B for FP32, 32 B for FP64)
constexpr int MAX_LEVELS = 16;

struct Grid {
    int nx, ny, nz;              // elements per axis
    int pitch;                   // row pitch in elements
    int64_t plane;               // plane pitch in elements
    int64_t total;               // elements in one stored vector
    double h[3];                 // element sides
    __host__ __device__ int64_t off(int i, int j, int k) const {
        return plane_base(k) + in_plane(i, j);
    }
    // 64-bit offset of node plane k, and the 32-bit offset of (i, j) inside a plane. Kernels
    // that visit many nodes of one plane form the product once: wide integer multiplies are
    // not free on GB300.
    __host__ __device__ int64_t plane_base(int k) const { return (int64_t)(k + 1) * plane; }
    __host__ __device__ int in_plane(int i, int j) const { return (j + 1) * pitch + (i + XL); }
};

// Operator of one level (Sec. 2): per-element stiffness entries by neighbour class for
// beta = 1, and the Robin face terms.  For the element matrix
//   K = kx(x)my(x)mz + mx(x)ky(x)mz + mx(x)my(x)kz,  k(0) = 1/h, k(1) = -1/h, m(0) = h/3,
//   m(1) = h/6,
// the entry between two nodes of one element depends only on which axes differ:
//   w_c: all three differ; w_e[a]: the two axes other than a differ; w_f[a]: only axis a
//   differs; w_0: same node.
struct Op {
    double w0, wc, we[3], wf[3];
    int cube;                    // 1 when hx = hy = hz (face weights 0, edge weight = corner weight)
    float w032, wc32, we32[3], wf32[3];  // the same weights rounded to FP32 on the host
    // Robin: alpha on each face (0 when Dirichlet or Neumann) and the in-face 1D mass entries
    double alpha[6];
    int bc[6];                   // 0 Dirichlet, 1 Robin
    int robin;                   // 1 when some alpha != 0 (integer test: FP64 compares run at 1/64 rate)
    int robin_mask;              // bit f set when face f has alpha != 0
    // alpha_F h_a h_b / 36 per face (a, b its in-face axes): the Robin face-mass weight of the
    // level, times small integer multiplicities at each node (host-rounded to FP32 as well)
    double rw64[6];
    float rw32[6];
};

__host__ inline Op make_op(const double h[3], const int bc[6], const double alpha[6])
{
    Op o;
    auto k = [&](int a, int d) { return (d ? -1.0 : 1.0) / h[a]; };
    auto m = [&](int a, int d) { return h[a] * (d ? 1.0 : 2.0) / 6.0; };
    auto K = [&](int dx, int dy, int dz) {
        return k(0, dx) * m(1, dy) * m(2, dz) + m(0, dx) * k(1, dy) * m(2, dz) +
               m(0, dx) * m(1, dy) * k(2, dz);
    };
    o.w0 = K(0, 0, 0);
    o.wc = K(1, 1, 1);
    o.we[0] = K(0, 1, 1);
    o.we[1] = K(1, 0, 1);
    o.we[2] = K(1, 1, 0);
    o.wf[0] = K(1, 0, 0);
    o.wf[1] = K(0, 1, 0);
    o.wf[2] = K(0, 0, 1);
    o.cube = (h[0] == h[1] && h[1] == h[2]) ? 1 : 0;
    o.w032 = (float)o.w0;
    o.wc32 = (float)o.wc;
    for (int a = 0; a < 3; ++a) {
        o.we32[a] = (float)o.we[a];
        o.wf32[a] = (float)o.wf[a];
    }
    for (int f = 0; f < 6; ++f) {
        o.bc[f] = bc[f];
        o.alpha[f] = (bc[f] == 1) ? alpha[f] : 0.0;
    }
    o.robin = 0;
    o.robin_mask = 0;
    for (int f = 0; f < 6; ++f) {
        o.robin |= o.alpha[f] != 0.0;
        if (o.alpha[f] != 0.0) o.robin_mask |= 1 << f;
        const int an = f / 2, aa = an == 0 ? 1 : 0, ab = an == 2 ? 1 : 2;
        o.rw64[f] = o.alpha[f] * h[aa] * h[ab] / 36.0;
        o.rw32[f] = (float)o.rw64[f];
    }
    return o;
}

// Device-side state of one JCG / mixed solve on one level. Written by the last block of each
// reducing kernel, read by the next kernel. All scalars FP64.
struct SolveState {
    double rho;          // r . z of the current residual
    double pq;           // p . q of the current iteration
    double alpha;        // step of the current iteration
    double alpha_prev;   // step not yet applied to the iterate (deferred update)
    double beta;         // coefficient of the next search direction
    double rr;           // ||r||^2, recursive (or true right after a residual evaluation)
    double rr_ref;       // MIXED: ||r||^2 at the last FP64 residual replacement
    double thresh2;      // (rtol ||f_h||)^2
    double fh2;          // ||f_h||^2
    double inner2;       // MIXED: inner_rtol^2
    double rr_true;      // last true ||r||^2
    double rtol2;        // rtol^2
    int iters;           // JCG iterations done
    int updates;         // MIXED: FP64 residual replacements done
    int max_iters;
    int status;          // 0 running/ok, 3 no convergence, 4 breakdown, 5 a staged copy never arrived,
                         // 6 stale constant-coefficient stencil path (the level computed nothing)
    int done;            // 1 when the level has finished
    int need_update;     // MIXED: 1 when the next step is an FP64 residual replacement
    int stop_after_update; // MIXED: iteration cap reached, finish after the next replacement
    int p_latest;        // which of the two search-direction buffers holds the newest p
    unsigned int arrive; // block arrival counter of the last-block reductions
    unsigned long long bcbits;  // MIXED, constant coefficient: bits of max |b / c| over the free nodes
                                // (fixed-point scale; c = -beta h / 36)
    unsigned long long xbits;   // batched MIXED: bits of max |x| for the next exact residual (0 = not taken)
    int fixed;           // 1: exactly max_iters steps, no tolerance test (the schedule of Alg. 3)
    // MIXED two-pass levels with a ring of search directions: the FP32 correction of the iterate,
    // sum of alpha_k p_k since the last replacement, is formed from the stored directions (at a
    // replacement, or into the correction vector when the ring fills) instead of being
    // accumulated in a vector by every step
    int pj;              // ring slot of the newest search direction
    int pbase;           // ring slot of the oldest direction not yet added
    int pend;            // directions not yet added
    int pring;           // ring slots (0: no ring on this level)
    int espill;          // 1 when the correction vector holds directions added from a full ring
};
// When this many directions are pending in a ring of pring slots, K2 adds them to the
// correction vector (the next step must not overwrite a pending direction).
__host__ __device__ inline int ring_cap(int pring) { return pring - 2; }

// Elements from one slot of a ring of search directions to the next: the level's stored length
// rounded up to 64 (256 bytes), so that every slot, like a vector of its own, starts on a DRAM
// burst boundary (at 32-byte alignment the fold's reads of 62 slots fetched 13 % more than they used).
__host__ __device__ inline int64_t ring_stride(int64_t total) { return (total + 63) / 64 * 64; }

// The ring of search directions of a two-pass MIXED level: R FP32 level vectors back to back,
// the step alpha of the direction in each slot, and R. With a ring, K1 reads p_old from slot
// st->pj, writes p to the next slot and records its alpha there, and moves no correction
// vector; K2 adds a full ring to the correction vector e, and the fold of a replacement adds e
// (when it holds anything) and the pending alpha p.
struct RingArgs {
    float* base;
    double* alpha;
    int R;
};

// Fixed-point scale of an iterate: bit pattern of max |x| (nonnegative doubles order like their
// bit patterns) and the block arrival counter of the reduction that forms it.
struct FixedScale {
    unsigned long long bits;
    unsigned int arrive;
};

// Device-side duration of the launches of one kernel on one level, taken inside whatever runs
// it (a CUDA graph included): the earliest block start of a launch (atomicMin of the global
// timer) to the end of its last block; the last block adds the difference and rearms t0.
struct KTimer {
    unsigned long long t0;   // earliest block start of the running launch (~0 when idle)
    unsigned long long ns;   // summed launch durations
    unsigned long long n;    // launches summed
};
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Launch helper of one reducing kernel: where its per-block partial sums go.
struct Partials {
    double* buf;         // >= 3 * max_blocks doubles
    int max_blocks;
    FixedScale* fs;      // fixed-point scale of the exact residual (one per handle)
};

// ---- set-up kernels (setup.cu) -------------------------------------------------------
void pack_nodal(const Grid& g, const double* dense, double* dst, cudaStream_t s);
// pack_nodal on the Dirichlet nodes only (the only nodes where g_D is read)
void pack_dirichlet(const Grid& g, const Op& op, const double* dense, double* dst, cudaStream_t s);
void pack_elements(const Grid& g, const double* dense, double* dst, cudaStream_t s);
void unpack_nodal(const Grid& g, const double* src, double* dense, cudaStream_t s);
// unpack_nodal into the array whose address *slot holds on the device (null: no copy); set_out
// stores that address (a graph records the copy once and writes a new array at each launch).
void set_out(double** slot, double* out, cudaStream_t s);
void unpack_out(const Grid& g, const double* src, double* const* slot, cudaStream_t s);
void coarsen_beta(const Grid& gc, const double* bf, const Grid& gf, double* bc, cudaStream_t s);
// The finest beta from the caller's dense array in one pass: packed (beta), in FP32 (beta32, the
// elements only), the uniform flag (as beta32_uniform) and the beta of the level below (bc, as
// coarsen_beta).
void beta_finest(const Grid& g, const Grid& gc, const double* dense, double* beta, float* beta32, int* flag,
                 double* bc, cudaStream_t s);
void inject_nodal(const Grid& gc, const double* vf, const Grid& gf, double* vc, cudaStream_t s);
void restrict_load(const Grid& gc, const double* bf, const Grid& gf, double* bc, cudaStream_t s);
void nodal_load(const Grid& g, const Op& op, const double* f, const double* gR, double* b,
                cudaStream_t s);
// b = int f phi_i by the 3x3x3 Gauss rule per element from f at the rule's points (f27, the
// ECMG_F_GAUSS layout), plus M_F gR_I on Robin faces when gR is given.
void gauss_load(const Grid& g, const Op& op, const double* f27, const double* gR, double* b, cudaStream_t s);
// D^-1 in FP64 and/or FP32 (beta32 = beta rounded). uniform: the level's flag, with beta32
// already converted by beta32_uniform; a one-beta all-Dirichlet cube then keeps only the D^-1
// of node (1, 1, 1) in FP32. nullptr: beta32 converted here, D^-1 on every node.
void jacobi_diag(const Grid& g, const Op& op, const double* beta, double* dinv64, float* dinv32,
                 float* beta32, int precond, cudaStream_t s, const int* uniform = nullptr);
// x = g_D on the Dirichlet nodes (0 when gD is null) and 0 on the free nodes; shell: only the
// nodes within two steps of a Dirichlet face (enough for ||f_h|| before EXP_finite writes every
// free node of the level).
void dirichlet_extension(const Grid& g, const Op& op, const double* gD, double* x, cudaStream_t s,
                         bool shell = false);
void convert_f32(const double* src, float* dst, int64_t n, cudaStream_t s);
void convert_f64(const float* src, double* dst, int64_t n, cudaStream_t s);
// flag = 1 when every element of the level has the same beta, else 0.
void uniform_check(const Grid& g, const double* beta, int* flag, cudaStream_t s);
// beta32 = beta (every padded element) and the flag of uniform_check, in one pass.
void beta32_uniform(const Grid& g, const double* beta, float* beta32, int* flag, cudaStream_t s);

// One thread writes the GPU's global timer (ns) into *t (device).
void launch_stamp(unsigned long long* t, cudaStream_t s);

// Kernel executions counted on the device, per source file (for the benchmark's launch count).
unsigned long long launches_setup();
unsigned long long launches_jcg();
unsigned long long launches_exp();

}  // namespace ecmg
