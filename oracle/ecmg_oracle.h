/*
 * ecmg_oracle.h -- plain FP64 CPU oracle for the ECMG_jcg method of Pan, He and Hu,
 * "A new extrapolation cascadic multigrid method for 3D elliptic boundary value
 * problems on rectangular domains" (arXiv 1506.02983).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark load this code. The CUDA library never includes, links or calls it, and
 * the two share no header, table or helper.
 *
 * Conventions (shared by every function below):
 *   - A level grid has n[0] x n[1] x n[2] hexahedral elements on the box [lo, hi]; the
 *     element sides are h[a] = (hi[a]-lo[a]) / n[a].
 *   - Nodes are numbered lexicographically with x fastest:
 *         node(i,j,k) = i + (n[0]+1) * (j + (n[1]+1) * k).
 *   - Elements likewise: elem(i,j,k) = i + n[0] * (j + n[1] * k).
 *   - Faces are numbered 0:x=lo 1:x=hi 2:y=lo 3:y=hi 4:z=lo 5:z=hi.
 *     face_bc[f] = OR_DIRICHLET or OR_ROBIN; a Robin face with alpha = 0 is Neumann
 *     (Sec. 1, eq. (bvp)).
 *   - A node lying on any Dirichlet face is a Dirichlet node; every other node is free.
 *
 * The header comment of ecmg_oracle.c lists the pins that check each function.
 */
#ifndef ECMG_ORACLE_H
#define ECMG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_DIRICHLET = 0, OR_ROBIN = 1 };
enum { OR_F_NODAL = 0, OR_F_LOAD = 1 };
enum { OR_EXP_SERENDIPITY20 = 0, OR_EXP_LAGRANGE27 = 1 };

/* Problem statement of eq. (bvp): finest-level data, host memory, FP64. */
typedef struct {
    int32_t n0[3];        /* coarsest elements per axis                               */
    int32_t levels;       /* total number of nested levels (>= 3)                      */
    double lo[3], hi[3];  /* the box                                                   */
    int32_t face_bc[6];   /* OR_DIRICHLET / OR_ROBIN per face                          */
    double alpha[6];      /* Robin coefficient per face                                */
    const double* beta;   /* finest level, one value per element                       */
    const double* f;      /* finest level nodal f (OR_F_NODAL) or load vector (OR_F_LOAD) */
    const double* gD;     /* finest level nodal Dirichlet data, or NULL for zero       */
    const double* gR;     /* finest level nodal Robin data, or NULL for zero           */
    int32_t f_mode;
} or_problem;

/* ---- discretisation (Sec. 2) ---------------------------------------------------- */
void or_element_matrix(double hx, double hy, double hz, double K[64]);
void or_face_mass(double ha, double hb, double M[16]);
void or_element_mass(double hx, double hy, double hz, double M[64]);
void or_dirichlet_mask(const int32_t n[3], const int32_t face_bc[6], uint8_t* mask);
int64_t or_assemble_csr(const int32_t n[3], const double h[3], const double* beta,
                        const int32_t face_bc[6], const double alpha[6],
                        int64_t* rowptr, int64_t* col, double* val);
void or_load_nodal(const int32_t n[3], const double h[3], const double* f,
                   const int32_t face_bc[6], const double* gR, double* b);
void or_csr_matvec(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                   const double* x, double* y);
/* (A x) at one node (i, j, k) from the element and Robin face matrices (the full matrix of
 * Sec. 2, no Dirichlet elimination): row (i, j, k) of or_assemble_csr times x. */
double or_apply_at(const int32_t n[3], const double h[3], const double* beta, const int32_t face_bc[6],
                   const double alpha[6], const double* x, int64_t i, int64_t j, int64_t k);

/* ---- level transfer --------------------------------------------------------------- */
void or_coarsen_beta(const int32_t nc[3], const double* beta_fine, double* beta_coarse);
void or_inject(const int32_t nc[3], const double* v_fine, double* v_coarse);
void or_restrict_load(const int32_t nc[3], const double* b_fine, double* b_coarse);

/* ---- solvers (Alg. 4) --------------------------------------------------------------- */
int or_jcg(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
           const uint8_t* mask, const double* b, const double* gext, double* x,
           double rtol, int32_t max_iters, int32_t* iters, double* rel_res_true,
           double* rhs_norm);
/* CG or Jacobi-preconditioned CG: precond 1 = Jacobi, 0 = none; fixed 1 = exactly max_iters steps
 * without the tolerance test (Alg. 3). Same outputs as or_jcg. */
int or_pcg(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
           const uint8_t* mask, const double* b, const double* gext, double* x,
           double rtol, int32_t max_iters, int32_t precond, int32_t fixed, int32_t* iters, double* rel_res_true,
           double* rhs_norm);
/* JCG (or CG, precond = 0) in the single-pass arrangement: the same iterates as or_pcg in exact
 * arithmetic, the next r.z and ||r|| by expansion of r - alpha q. Same outputs as or_jcg. */
int or_pcg_single_pass(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                       const uint8_t* mask, const double* b, const double* gext, double* x, double rtol,
                       int32_t max_iters, int32_t precond, int32_t* iters, double* rel_res_true,
                       double* rhs_norm);
int or_dsolve_banded(const int32_t n[3], int64_t N, const int64_t* rowptr,
                     const int64_t* col, const double* val, const uint8_t* mask,
                     const double* b, double* x);

/* ---- extrapolation operators (Sec. 4.2-4.3) --------------------------------------- */
void or_serendipity(double xi, double eta, double zeta, double N[20]);
void or_serendipity_nodes(int32_t abc[60]);
void or_exp_finite(const int32_t n[3], const double* U1, const double* U0, double* W);
/* EXP_finite at one level-l node (I, J, K): the value or_exp_finite leaves there. */
double or_exp_finite_at(const int32_t n[3], const double* U1, const double* U0, int64_t I, int64_t J, int64_t K);
void or_exp_finite27(const int32_t n[3], const double* U1, const double* U0, double* W);
void or_exp_true(const int32_t n[3], const double* U1, const double* U0, double* Ut);
/* EXP_true at one level-l node (I, J, K). */
double or_exp_true_at(const int32_t n[3], const double* U1, const double* U0, int64_t I, int64_t J, int64_t K);

/* ---- the whole method (Alg. 4) ------------------------------------------------------ */
typedef struct {
    int32_t iters[16];     /* JCG iterations per level (0 on the two DSOLVE levels)       */
    double rel_res[16];    /* true ||b - A u|| / ||f_h|| on exit, per level               */
    double rhs_norm[16];   /* ||f_h|| (lifted free-node load) per level                   */
    int32_t status;        /* 0 ok, 1 invalid input, 2 singular, 3 no convergence         */
    double seconds_assembly; /* wall time of the set-up: level data, CSR assembly, loads   */
    double seconds_solve;    /* wall time of DSOLVE, EXP_finite, JCG and EXP_true          */
} or_stats;

/* Threads for the loops that may run in parallel (CSR matrix-vector products and the
 * element-wise vector updates of JCG; every row and element is computed exactly as with one
 * thread, and the dot products stay sequential, so the results do not depend on the thread
 * count). Returns the threads that will be used: 1 unless built with OpenMP. */
int32_t or_set_threads(int32_t n);

int or_ecmg(const or_problem* p, double rtol, int32_t max_iters, int32_t exp_variant,
            double* U_all, double* W_all, double* Ut_all, or_stats* st);
/* or_ecmg with the variants of Sec. 3: precond 1 = JCG (ECMG_jcg), 0 = CG (ECMG_cg); schedule 1 =
 * the fixed step counts m_j = ceil(m_L beta^(L-j)) of Alg. 3, eq. (ee), instead of the tolerance. */
int or_ecmg_ex(const or_problem* p, double rtol, int32_t max_iters, int32_t exp_variant, int32_t precond,
               int32_t schedule, int32_t mL, double sched_beta, double* U_all, double* W_all, double* Ut_all,
               or_stats* st);
/* Steps of level l (>= 2) of an L-level hierarchy in that schedule. */
int32_t or_schedule_steps(int32_t L, int32_t l, int32_t mL, double beta);

/* ---- norms (Sec. 5: max norm and root-mean-square "L2" norm) ------------------------- */
void or_norms(int64_t N, const double* a, const double* b, double* max_abs, double* rms);

#ifdef __cplusplus
}
#endif
#endif
