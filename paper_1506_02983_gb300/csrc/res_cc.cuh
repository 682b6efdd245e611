// res_cc.cuh -- residual of the MIXED iteration on a constant-coefficient level (res_cc.cu).
#pragma once

#include <cuda.h>

#include "jcg.cuh"

namespace ecmg {

// Tensor maps of a level's FP64 iterate U and of b / c (the level's FP64 r vector after
// launch_fh2 on a MIXED level).
struct ResMaps {
    CUtensorMap x, bc;
};
bool make_res_maps(ResMaps* m, const double* x, const double* bc, const Grid& g);
// Set the shared-memory limit of the kernel on the current device.
cudaError_t res_cc_prepare();
// Blocks of one launch on this level (the partials buffer must hold as many).
int res_cc_blocks(const Grid& g);

// r = b - A x on the free nodes of a level with one beta, every face Dirichlet and cubic
// elements (r on the Dirichlet nodes is not written and stays 0), exactly in fixed point and
// rounded once to FP32; ||r||^2 and r.z reduced, the last block acts by `mode` (RES_INIT,
// RES_REPLACE or RES_REPORT). Needs the level's max |x| in pr.fs (launch_absmax, same
// stream) and max |b / c| in st->bcbits (launch_fh2). If the level's uniform flag is
// clear when the kernel runs, it records status 6 and finishes the level without computing.
// r_b: with the single-pass buffer pair taken from the level state, the other r of the pair; the
// residual then goes to r_b when st->p_latest is 1 (the buffer the next step reads).
void launch_res32_cc(const ResMaps& m, const Grid& g, const int* uniform, const double* beta, const float* dinv32,
                     float* r, SolveState* st, Partials pr, ResMode mode, CondHandles ch, cudaStream_t s,
                     float* r_b = nullptr);

unsigned long long launches_res_cc();

}  // namespace ecmg
