/*
 * ecmg.h -- C ABI of the GB300 ECMG_jcg library (libecmg.so).
 *
 * The library solves the model problem of Pan, He and Hu (arXiv 1506.02983), Sec. 1,
 * eq. (bvp):
 *
 *     -div(beta grad u) = f      in a box Omega,
 *     u = g_D                    on the Dirichlet faces,
 *     alpha u + beta du/dn = g_R on the Robin faces (alpha = 0 is Neumann),
 *
 * discretised by trilinear (Q1) finite elements on nested uniform hexahedral grids (Sec. 2),
 * with the extrapolation cascadic multigrid method ECMG_jcg of Alg. 4: a direct solve on the
 * two coarsest grids, then on every finer grid an extrapolated initial guess (EXP_finite,
 * Sec. 4.2-4.3), Jacobi-preconditioned CG until ||A u - f||_2 <= rtol ||f||_2, and a fourth
 * order Richardson-extrapolated solution (EXP_true, Sec. 4.2.1 and 4.3).
 *
 * Memory and ownership
 *   - Every pointer argument documented as "device" is read or written by the library's
 *     kernels: device memory of the current device, managed memory, or page-locked host memory
 *     (cudaHostAlloc, cudaHostRegister; a GB300 reaches it over its coherent chip-to-chip link,
 *     so a solve can take its inputs from, and write its solution to, pinned host buffers with
 *     no separate copy). Any other pointer is refused with ECMG_ERR_INVALID_ARG before a kernel
 *     touches it. "host" pointers are ordinary host memory. Inputs are read, never written.
 *   - The caller owns every array it passes. ecmg_create records the problem description and
 *     the input pointers; the input arrays must stay valid and unchanged until the last
 *     ecmg_solve on the handle has completed (ecmg_solve reads them on the device).
 *   - The handle owns the device workspace it allocates in ecmg_create (all levels, all
 *     vectors) and frees it in ecmg_destroy.
 *   - All work is ordered on the CUDA stream passed to ecmg_create (NULL = legacy default
 *     stream). Functions that return values on the host synchronise that stream.
 *
 * Layout of caller arrays (the "dense" layout)
 *   - Nodal arrays of a level with n = (nx, ny, nz) elements hold (nx+1)(ny+1)(nz+1) doubles,
 *     index i + (nx+1) (j + (ny+1) k), x fastest.
 *   - Element arrays hold nx ny nz doubles, index i + nx (j + ny k).
 *
 * Errors
 *   Every function returns an ecmg_status. Nothing aborts and no kernel traps: a failure on
 *   the device (breakdown, iteration cap) is recorded in a status word that the host reads
 *   back; the best iterate stays in place. ECMG_ERR_CUDA reports a CUDA runtime error; the
 *   message of the last error is available from ecmg_last_error().
 */
#ifndef ECMG_H
#define ECMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ECMG_OK = 0,
    ECMG_ERR_INVALID_ARG = 1,    /* bad size, pointer, option or level                      */
    ECMG_ERR_SINGULAR = 2,       /* no Dirichlet face and every Robin alpha is zero          */
    ECMG_ERR_NO_CONVERGENCE = 3, /* a level hit options.max_iters                            */
    ECMG_ERR_BREAKDOWN = 4,      /* p.q <= 0 or a non-finite value in JCG                    */
    ECMG_ERR_OOM = 5,            /* device allocation failed                                 */
    ECMG_ERR_CUDA = 6            /* any other CUDA runtime error                             */
} ecmg_status;

enum { ECMG_BC_DIRICHLET = 0, ECMG_BC_ROBIN = 1 };
/* f is nodal values of f (load b = M f_I + sum_F M_F g_R,I per level), or the finest
 * assembled load functional b_i = f(phi_i) of Sec. 2 (coarse loads b_{l-1} = P^T b_l), or f as
 * separable terms (ECMG_F_SEPARABLE, below), or f at the points of the 3x3x3 Gauss rule of every
 * finest element (ECMG_F_GAUSS, below). */
enum { ECMG_F_NODAL = 0, ECMG_F_LOAD = 1, ECMG_F_SEPARABLE = 2, ECMG_F_GAUSS = 3 };
enum { ECMG_FP64 = 0, ECMG_MIXED = 1 };
/* ecmg_apply_operator only: the FP32 stencil kernel of the MIXED iteration itself (K1). */
enum { ECMG_APPLY_K1 = 2 };
/* EXP_finite variant: the 20-node Serendipity interpolation of Sec. 4.3, or the 27-node
 * tri-quadratic Lagrange variant of the Remark that follows it. */
enum { ECMG_EXP_SERENDIPITY20 = 0, ECMG_EXP_LAGRANGE27 = 1 };
/* Smoother of Alg. 4 line 8 (Sec. 3): JCG (ECMG_jcg) or plain CG (ECMG_cg). */
enum { ECMG_PREC_JACOBI = 0, ECMG_PREC_NONE = 1 };
/* Steps per level: the relative residual test of Alg. 4 line 7, or the fixed counts
 * m_j = ceil(m_L beta^(L-j)) of Alg. 3, eq. (ee), with j = 1 .. L the levels above the two
 * direct ones. */
enum { ECMG_SCHED_TOLERANCE = 0, ECMG_SCHED_FIXED = 1 };
/* Form of one FP32 step of the MIXED iteration (the recurrence of Alg. 4 line 8 is the same):
 * TWO_PASS runs the search-direction/stencil kernel (p, q = A p, p.q) and then the residual
 * kernel (r -= alpha q, r.z, r.r); SINGLE_PASS does both in one kernel per step: the residual
 * update of the previous step is applied while its tiles are staged, and the next r.z and r.r
 * are obtained from the dots of the same pass by expanding (r - alpha q).D^-1(r - alpha q) and
 * (r - alpha q).(r - alpha q). Equal to TWO_PASS in exact arithmetic; the FP64 residual
 * replacements bound the difference in floating point. Needs two more FP32 vectors per level. */
enum { ECMG_CG_TWO_PASS = 0, ECMG_CG_SINGLE_PASS = 1, ECMG_CG_AUTO = 2 };
/* ECMG_CG_AUTO: SINGLE_PASS on the levels of fewer than ECMG_AUTO_SINGLE_PASS_NODES nodes, where
 * a step's time is mostly launch and reduction latency and one kernel per step saves a launch,
 * TWO_PASS on the larger ones, where both forms stream at their bandwidth and take the same
 * time per step. */
#define ECMG_AUTO_SINGLE_PASS_NODES (1 << 22)

/* ecmg_options.ring_slots: slots chosen by ecmg_create from the workspace and the device memory:
 * 64, 8..63 or 0. */
#define ECMG_RING_AUTO (-1)
/* ecmg_get_level: which vector */
enum { ECMG_VEC_U = 0, ECMG_VEC_W = 1, ECMG_VEC_UTILDE = 2, ECMG_VEC_B = 3, ECMG_VEC_BETA = 4 };

/* Problem statement of eq. (bvp) (Sec. 1) on the finest grid. */
typedef struct {
    int32_t n0[3];          /* coarsest grid elements per axis, >= 1                        */
    int32_t levels;         /* total nested levels, 3..12; level l has n0 * 2^l elements  */
    double lo[3], hi[3];    /* box corners, hi > lo                                          */
    int32_t face_bc[6];     /* faces x-,x+,y-,y+,z-,z+: ECMG_BC_DIRICHLET or ECMG_BC_ROBIN  */
    double robin_alpha[6];  /* alpha on each Robin face (>= 0); ignored on Dirichlet faces  */
    const double* beta;     /* device, finest elements, > 0 (dense element layout)          */
    const double* f;        /* device: f values or load functional at the finest nodes, or
                               the compact forms below (f_mode)                             */
    const double* g_D;      /* device, finest nodes, read on Dirichlet nodes; NULL = 0      */
    const double* g_R;      /* device, finest nodes, read on Robin faces (ECMG_F_NODAL and
                               ECMG_F_GAUSS only); NULL = 0                                   */
    int32_t f_mode;         /* ECMG_F_NODAL, ECMG_F_LOAD, ECMG_F_SEPARABLE or ECMG_F_GAUSS   */
    /* Compact inputs (single-problem and batched handles):
     * ECMG_F_SEPARABLE: f = sum over f_terms terms of fx(x) fy(y) fz(z); the device array f
     *   holds every factor at the 3-point Gauss-Legendre nodes of every finest element interval
     *   [x_e, x_e + h], in the order x_e + h (1 - sqrt(3/5))/2, x_e + h/2, x_e + h (1 + sqrt(3/5))/2:
     *   f_terms x 3 (nx + ny + nz) doubles, term-major, then x, y, z, interval-major. The library
     *   assembles the load functional int f phi_i of Sec. 2 from them (the rule is exact for
     *   factors of degree <= 4) and its exact coarse restrictions P^T b; g_R must be NULL.
     * ECMG_F_GAUSS: the device array f holds f at the 27 points of the 3-point Gauss-Legendre rule
     *   of every finest element: 27 nx ny nz doubles, elements x fastest (index ex + nx (ey + ny ez)),
     *   then the points qx fastest, qy, qz, each axis in the order above (x_e + h (1 - sqrt(3/5))/2,
     *   x_e + h/2, x_e + h (1 + sqrt(3/5))/2). The library assembles the load functional int f phi_i
     *   of Sec. 2 with that rule on every element (plus the face mass of the nodal g_R on Robin faces)
     *   and its coarse restrictions P^T b; f may be any function (singular ones included, since no
     *   point lies on an element's boundary).
     * gD_terms > 0: g_D = sum over gD_terms terms of gx(x) gy(y) gz(z); the device array g_D holds
     *   the factors at the finest nodes: gD_terms x ((nx+1) + (ny+1) + (nz+1)) doubles,
     *   term-major, then x, y, z.
     * beta == NULL: one beta everywhere, beta_const (> 0). */
    int32_t f_terms;        /* ECMG_F_SEPARABLE: terms of f, 1..64                           */
    int32_t gD_terms;       /* 0: g_D nodal (or NULL); 1..64: g_D separable                  */
    double beta_const;      /* the beta of every element when beta is NULL                  */
} ecmg_problem;

/* Solver options. ecmg_default_options fills the defaults given in brackets. */
typedef struct {
    double rtol;            /* relative residual tolerance epsilon of Alg. 4 line 7 [1e-9]  */
    int32_t precision;      /* ECMG_FP64 or ECMG_MIXED                        [ECMG_FP64]   */
    double inner_rtol;      /* MIXED: FP32 inner reduction between FP64 residual
                               replacements                                  [1e-3]        */
    int32_t max_iters;      /* per-level JCG iteration cap                   [100000]      */
    int32_t use_graph;      /* 1: one CUDA graph per solve with device-side loop control;
                               0: host-driven loop (debugging)               [1]           */
    double dsolve_rtol;     /* relative residual of the direct solve on levels 0, 1 [1e-14]*/
    int32_t exp_variant;    /* ECMG_EXP_SERENDIPITY20 / ECMG_EXP_LAGRANGE27  [SERENDIPITY20]*/
    int32_t true_residual;  /* 1: report the true FP64 residual of every level [1]         */
    int32_t autotune;       /* MIXED: 1 = ecmg_create times the tile shapes of the FP32
                               stencil kernel on every level of >= 2^18 nodes and keeps the
                               fastest (ecmg_autotune); 0 = built-in shape       [0]       */
    int32_t preconditioner; /* ECMG_PREC_JACOBI (ECMG_jcg) or ECMG_PREC_NONE (ECMG_cg), on
                               every level                                   [JACOBI]      */
    int32_t schedule;       /* ECMG_SCHED_TOLERANCE or ECMG_SCHED_FIXED; with FIXED every
                               level >= 2 runs exactly m_j steps (rtol and max_iters unused
                               there)                                        [TOLERANCE]   */
    int32_t sched_mL;       /* FIXED: m_L, the steps on the finest level, >= 1  [4]         */
    double sched_beta;      /* FIXED: beta of eq. (ee), 1..64                   [4.0]       */
    int32_t cg_form;        /* MIXED: ECMG_CG_TWO_PASS, ECMG_CG_SINGLE_PASS or ECMG_CG_AUTO (batched
                               handles run TWO_PASS for AUTO)                   [AUTO]     */
    int32_t ring_slots;     /* MIXED two-pass levels of single-problem handles: ECMG_RING_AUTO, 0, or
                               4..64 slots of a ring of FP32 search directions. Without a ring every
                               FP32 step adds alpha_k p_k to a correction vector e (4 bytes read
                               and 4 written per node); with one, the step only stores p_k, and
                               e += alpha_k p_k runs over all pending directions at once when
                               ring_slots - 2 are pending, and at a residual replacement, as the
                               same FP32 fused multiply-adds in the same order: the solve is
                               bit-identical to the one without a ring. Costs 4 ring_slots bytes
                               per stored node of each such level. 0: no ring. ECMG_RING_AUTO: 64
                               slots when the handle's workspace with them stays within 3/4 of the
                               current device's memory, else the most slots (at least 8) that do,
                               else 0; the choice depends only on the problem's sizes, the options
                               and the device's total memory                     [AUTO]      */
} ecmg_options;

/* Per-solve statistics, one entry per level (coarsest first). */
typedef struct {
    int32_t levels;
    int32_t iters[16];      /* JCG iterations (FP32 inner iterations in MIXED mode)         */
    int32_t updates[16];    /* MIXED: FP64 residual replacements; FP64: 0                   */
    double rel_res[16];     /* ||b - A u||_2 / ||f_h||_2 on exit (true residual if enabled, */
                            /* else the recursive one)                                      */
    double rhs_norm[16];    /* ||f_h||_2, the free-node right-hand side with g_D moved over */
    int32_t status;         /* ecmg_status of the solve                                     */
    double seconds[16];     /* single-problem solves: device time of each level (its DSOLVE or
                               EXP_finite, JCG and EXP_true), from the GPU's global timer at
                               the level's first and the next level's first kernel; 0 for
                               levels a solve did not run and for batched solves             */
    double setup_seconds;   /* device time of the level set-up of all levels (0 when a solve
                               starts above level 0, or batched)                             */
} ecmg_stats;

typedef struct ecmg_handle ecmg_handle;

/* Fill *opt with the defaults listed in ecmg_options. */
void ecmg_default_options(ecmg_options* opt);

/* Validate the problem, allocate the device workspace of every level and record the problem
 * (Alg. 4 inputs). stream: a cudaStream_t (NULL = default stream). *out receives the handle.
 * Returns ECMG_ERR_INVALID_ARG for bad sizes or options, ECMG_ERR_SINGULAR when no face is
 * Dirichlet and every Robin alpha is 0, ECMG_ERR_OOM when allocation fails. */
ecmg_status ecmg_create(const ecmg_problem* prob, const ecmg_options* opt, void* stream,
                        ecmg_handle** out);

/* Device memory from the caller: alloc returns `bytes` of device memory usable on `stream`
 * (NULL when it cannot), free gives back a block alloc returned, with the same size. `ctx`
 * is passed through unchanged. A framework that owns device memory (a caching allocator)
 * supplies both, so that the workspace counts against its pools. */
typedef void* (*ecmg_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ecmg_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* As ecmg_create, with every device allocation of the handle's workspace made through
 * alloc and released through free (in ecmg_destroy, after the stream has synchronised; also
 * when creation fails part way). alloc and free must both be given; ECMG_ERR_INVALID_ARG
 * otherwise. A NULL from alloc fails creation with ECMG_ERR_OOM. Pinned host buffers of the
 * handle still come from the CUDA runtime. */
ecmg_status ecmg_create_with_allocator(const ecmg_problem* prob, const ecmg_options* opt, void* stream,
                                       ecmg_alloc_fn alloc, ecmg_free_fn free, void* ctx, ecmg_handle** out);

/* Run Alg. 4: level set-up from the current input arrays (beta averaging, loads, Jacobi
 * diagonals), DSOLVE on levels 0 and 1, then for each finer level EXP_finite, JCG and
 * EXP_true. u_out: device, finest nodes (dense layout), may be NULL. stats: host, may be
 * NULL. Synchronises the stream. Returns the worst status over the levels. */
ecmg_status ecmg_solve(ecmg_handle* h, double* u_out, ecmg_stats* stats);

/* Copy the fourth-order extrapolated solution U~ (EXP_true) of level `level` (-1 = finest,
 * 2..levels-1 otherwise) into u_tilde_out (device, dense nodal layout of that level). Valid
 * after ecmg_solve. Ordered on the handle's stream; does not synchronise. */
ecmg_status ecmg_extrapolate(ecmg_handle* h, int32_t level, double* u_tilde_out);

/* Copy one stored vector of a level (ECMG_VEC_U solution, ECMG_VEC_W initial guess,
 * ECMG_VEC_UTILDE extrapolated solution, ECMG_VEC_B assembled load, ECMG_VEC_BETA element
 * coefficients) into out (device, dense layout of that level). level -1 = finest. */
ecmg_status ecmg_get_level(ecmg_handle* h, int32_t level, int32_t which, double* out);

/* Overwrite the stored solution U of a level (device, dense layout). With ecmg_solve_from this
 * resumes Alg. 4 at any level >= 2 from the two stored coarser solutions. */
ecmg_status ecmg_set_level(ecmg_handle* h, int32_t level, const double* in);

/* Run Alg. 4 from level `first` (>= 2) upwards, using the stored U of levels first-1 and
 * first-2 (after a previous ecmg_solve or ecmg_set_level). Same outputs as ecmg_solve. */
ecmg_status ecmg_solve_from(ecmg_handle* h, int32_t first, double* u_out, ecmg_stats* stats);

/* y = A_l x for level `level` (-1 = finest) with the level's matrix of Sec. 2 (Robin terms
 * included, no boundary elimination): x, y device, dense nodal layout. Valid after the
 * level set-up of an ecmg_solve. precision ECMG_FP64 or ECMG_MIXED (FP32 arithmetic on FP32
 * rounded x). ECMG_APPLY_K1 (MIXED handles) runs the search-direction kernel of the FP32
 * iteration (line 8 of Alg. 4 fused with q = A p) with r = 0, p_old = x and beta = 1, so it
 * forms p = x and q = A p with the level's current tile shape and kernel path; y is q on the
 * nodes off Dirichlet faces and 0 on them. It overwrites the level's FP32 iteration vectors.
 * Ordered on the handle's stream. */
ecmg_status ecmg_apply_operator(ecmg_handle* h, int32_t level, int32_t precision,
                                const double* x, double* y);

/* Error norms between two device vectors of one level (dense nodal layout): max |a - b| and
 * root-mean-square over all nodes (the max and "L2" norms of the tables of Sec. 5).
 * b may be NULL (norms of a). A NaN anywhere in a - b makes both results NaN (an error norm
 * never hides one). Results on the host; synchronises the stream. */
ecmg_status ecmg_error_norms(ecmg_handle* h, int32_t level, const double* a, const double* b,
                             double* max_abs, double* rms);

void ecmg_destroy(ecmg_handle* h);
const char* ecmg_status_string(ecmg_status s);
const char* ecmg_last_error(void);

/* ---- batched solves (no counterpart in the paper) ----------------------------------------
 *
 * Many independent problems of any sizes, boundary conditions and coefficients solved by
 * Alg. 4 side by side: every step of the method (level set-up, EXP_finite, the FP64 residual,
 * each FP32 JCG iteration, the residual replacement, EXP_true) is one kernel launch over all
 * problems, and the whole solve is one CUDA graph whose loops run while any problem runs.
 * Levels are aligned at the finest: a problem with fewer levels starts later and every problem
 * finishes its finest level in the last stage. Precision is MIXED only; the direct solves of
 * levels 0 and 1 are the same FP32 JCG with FP64 residual replacement, run to dsolve_rtol. */

/* probs: n problems (1..128), each validated as by ecmg_create; their device arrays must stay
 * valid and unchanged while a solve reads them. opt: shared options (precision must be
 * ECMG_MIXED). stream: a cudaStream_t. Returns a handle for ecmg_solve_batched,
 * ecmg_get_level_batched and ecmg_destroy; single-problem calls reject it. */
ecmg_status ecmg_create_batched(const ecmg_problem* probs, int32_t n, const ecmg_options* opt, void* stream,
                                ecmg_handle** out);
/* Solve every problem. u_out: NULL, or n device pointers (each NULL or the finest nodal
 * solution of that problem, dense layout). stats: NULL or n entries (host). Synchronises the
 * stream. Returns the worst status over all problems and levels. */
ecmg_status ecmg_solve_batched(ecmg_handle* h, double* const* u_out, ecmg_stats* stats);
/* As ecmg_get_level for one problem of a batch (which: U, W, U~ or B). */
ecmg_status ecmg_get_level_batched(ecmg_handle* h, int32_t problem, int32_t level, int32_t which, double* out);

/* ---- measurement helpers (no counterpart in the paper) --------------------------------- */

/* Total kernel executions of this library in the process so far (counted on the device by
 * every kernel; a kernel that finds its level already finished still counts). out: host. */
ecmg_status ecmg_kernel_launches(uint64_t* out);

/* Time one kernel of the solve alone on level `level` (-1 = finest): `reps` launches, each
 * bracketed by CUDA events on the handle's stream, after one untimed launch. which:
 * 0 K1 FP32 (search direction + operator), 1 K2 FP32 (residual update), 2 FP64 residual with
 * FP32 output, 3 K1 FP64, 4 K2 FP64, 5 FP64 residual, 6 EXP_finite, 7 EXP_true, 8 ||f_h|| (on a
 * MIXED level with one beta, every face Dirichlet and cubic elements also b / c for the exact
 * residual, as the solve runs it),
 * 9 MIXED fold of the FP32 correction into the FP64 iterate (applied to U~; on a level with a
 * ring of search directions the fold of ring_slots - 2 pending directions), 10 max |U|,
 * 11 the single-pass FP32 step (handles created with ECMG_CG_SINGLE_PASS).
 * ms_out: mean duration of one launch (host). bytes_out: the algorithmic bytes one launch
 * must move (each owned input read once, each output written once; host); for kernel 0 the
 * nodes counted are those off the Dirichlet faces, the only ones it visits, and on a level
 * with one beta and every face Dirichlet kernels 0 and 1 count no beta and no D^-1 (they read
 * none). Valid after
 * ecmg_solve; it overwrites the level's work vectors and U~ (kernel 3 uses U~ as its
 * iterate); U and W are never changed. Synchronises the stream.
 * Batched handles: `level` is a stage of the batched solve (-1 = the last, where every problem
 * works on its finest level) and which is 0 (the batched K1 over every item of the stage), 1 (the
 * batched K2), 2 (the batched FP64 residual with its max |x| pass) or 11 (the batched single-pass
 * step, on batches created with ECMG_CG_SINGLE_PASS); bytes_out sums the items' algorithmic
 * bytes. The launches overwrite the
 * items' work vectors and states, which the next ecmg_solve_batched sets up afresh. */
ecmg_status ecmg_time_kernel(ecmg_handle* h, int32_t level, int32_t which, int32_t reps,
                             double* ms_out, double* bytes_out);

/* Device-side timer of the MIXED FP32 stencil kernel (K1) of one level (-1 = finest): the
 * summed durations of its launches inside ecmg_solve (graph or eager), each from the earliest
 * block start (global timer) to the end of its last block, and the number of launches summed.
 * Launches that find their level finished are not counted. reset != 0 zeroes both after
 * reading. ms_total, launches: host. Synchronises the stream. */
ecmg_status ecmg_stencil_timer(ecmg_handle* h, int32_t level, int32_t reset, double* ms_total,
                               int64_t* launches);

/* ---- tile shapes of the FP32 stencil kernel (no counterpart in the paper) --------------
 *
 * In MIXED mode the stencil kernel of every level runs on tiles of 32 x (8 ry) nodes, each
 * thread computing ry vertically adjacent nodes, with each block marching kz node planes.
 * Shapes change only the launch geometry and the order of the partial sums of p.q. */

/* Force the shape of one level (-1 = finest): ry in {1, 2}, kz in 4..1024. Invalid shapes
 * return ECMG_ERR_INVALID_ARG; FP64 handles have no such kernel (ECMG_ERR_INVALID_ARG). */
ecmg_status ecmg_set_tiles(ecmg_handle* h, int32_t level, int32_t ry, int32_t kz);
/* Read the shape of one level into *ry, *kz (host). */
ecmg_status ecmg_get_tiles(ecmg_handle* h, int32_t level, int32_t* ry, int32_t* kz);
/* Autotuner: on every MIXED level of at least 2^18 nodes, try each candidate shape (ry in
 * {1, 2} x kz in {4, 6, 8, 10, 12, 14, 16, 20, 24, 32, 48, 64, 128}) and the current one: each
 * shape is set on all those levels at once and the whole solve runs `reps` times (level times from
 * device time stamps, so each level is timed as the solve runs it); every level keeps its fastest
 * shape. Costs 27 x reps solves. Overwrites every level's vectors (the solution included); call it
 * before a solve or between solves. Synchronises the stream.
 * Batched handles (also run at ecmg_create_batched when options.autotune = 1): for every stage,
 * the stage's whole K1 launch is timed for ry in {1, 2} x kz in {4, 8, 16, 32, 64} applied to all
 * of its items, then the kz of each size class of items (the same power of two of z nodes) is
 * varied with the others fixed; the fastest shapes are kept. */
ecmg_status ecmg_autotune(ecmg_handle* h, int32_t reps);

/* ---- error norms without device allocation (no counterpart in the paper) ---------------
 *
 * The same two norms as ecmg_error_norms -- max |a - b| and sqrt(sum (a - b)^2 / n) -- for
 * callers that may not allocate device memory where they need them. cudaMalloc and cudaFree
 * can synchronise the whole device, so code inside a latency-critical loop or a host
 * callback, or code under a framework that owns every device allocation, must avoid them.
 * This entry point allocates nothing and needs no handle: its scratch (one partial pair per
 * block of 16384 elements, plus the final pair) is a fixed array of 512 KiB inside the
 * library, which every device that loads the library holds until the process exits.
 *
 * a, b: device arrays of n doubles (any layout; b may be NULL for the norms of a). n must be
 * 1..ECMG_NOALLOC_MAX_ELEMS; a larger n is rejected with ECMG_ERR_INVALID_ARG before any
 * device work. stream: a cudaStream_t (NULL = default stream), synchronised before return.
 * max_abs, rms: host outputs.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that first call before any
 * stream capture, and do not reset the device (cudaDeviceReset) after it. a and b are checked
 * with cudaPointerGetAttributes first: device memory of the current device, managed memory or
 * page-locked host memory; anything else returns ECMG_ERR_INVALID_ARG and leaves the outputs
 * unwritten. A NaN anywhere in a - b makes both outputs NaN. Every call overwrites
 * the whole part of the array it reads, so nothing has to start at zero, but all calls share
 * the one array: calls that overlap on the GPU (different streams, or different host threads
 * on one device) race and may return wrong norms. */
#define ECMG_NOALLOC_MAX_ELEMS 536870912LL
ecmg_status ecmg_error_norms_noalloc(const double* a, const double* b, int64_t n, void* stream,
                                     double* max_abs, double* rms);

/* Bytes of device workspace ecmg_create allocates for this problem and options. */
ecmg_status ecmg_workspace_bytes(const ecmg_problem* prob, const ecmg_options* opt,
                                 uint64_t* bytes);

#ifdef __cplusplus
}
#endif
#endif
