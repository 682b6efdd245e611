// exp.cuh -- launch interface of the extrapolation and norm kernels (exp.cu).
#pragma once

#include "ecmg_internal.cuh"

namespace ecmg {

// EXP_finite: level-l grid g from U1 (level l-1, grid g1) and U0 (level l-2, grid g0).
// Writes W on every node (Dirichlet nodes copy x, which holds g_D there) and x on free nodes.
void launch_exp_finite(int variant, const Grid& g, const Op& op, const Grid& g1, const double* U1,
                       const Grid& g0, const double* U0, double* x, double* W, cudaStream_t s);
// EXP_true: Ut on level-l grid g from U1 (level l) and U0 (level l-1, grid gc). D: scratch of
// gc.total doubles that then holds d = U1 - U0 at the level-(l-1) nodes, formed once per node
// instead of once per element that shares it (same Ut bit for bit); null: no scratch.
void launch_exp_true(const Grid& g, const double* U1, const Grid& gc, const double* U0, double* Ut,
                     cudaStream_t s, double* D = nullptr);
// Per-block (max |a-b|, sum (a-b)^2) into part[2 * block]; returns via norms_blocks the count.
int norms_blocks(const Grid& g);
void launch_norms(const Grid& g, const double* a, const double* b, double* part, cudaStream_t s);

}  // namespace ecmg
