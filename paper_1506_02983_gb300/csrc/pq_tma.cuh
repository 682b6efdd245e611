// pq_tma.cuh -- TMA-staged K1 of the FP32 JCG iteration (pq_tma.cu).
#pragma once

#include <cuda.h>

#include "jcg.cuh"

namespace ecmg {

// Tensor maps of one level's FP32 vectors for plane boxes of 40 x 10 x 1 elements.
struct PlaneMaps {
    CUtensorMap r, pA, pB, dinv, beta;
};

// Encode a 3D tensor map over one padded FP32 level vector. False if the driver entry point
// is unavailable or the encoding is rejected.
bool make_plane_map(CUtensorMap* map, const float* base, const Grid& g);

int max_tma_blocks(const Grid& g);

// p = D^-1 r + beta p_old (p_old = pA or pB), q = A p, e += alpha_prev p_old, p.q.
void launch_pq32_tma(const PlaneMaps& m, int pold_is_b, const Grid& g, const Op& op, float* pnew, float* q,
                     float* e, SolveState* st, Partials pr, int pidx, CondHandles ch, cudaStream_t s);

unsigned long long launches_pq_tma();

}  // namespace ecmg
