// pq_tma.cuh -- TMA-staged K1 of the FP32 JCG iteration (pq_tma.cu).
#pragma once

#include <cuda.h>

#include "jcg.cuh"

namespace ecmg {

// Node rows a thread of K1 computes (the tile is 32 x 8*ry nodes), one tensor-map set each.
constexpr int K1_NRY = 2;
constexpr int K1_RY[K1_NRY] = {1, 2};

// Tensor maps of one level's FP32 vectors; set v stages boxes of 40 x (8*K1_RY[v]+2) x 1
// (e: 36 x 8*K1_RY[v] x 1, the tile's own rows). r is the first residual buffer; rB, qA and qB
// (the second residual buffer and the two q buffers) are encoded for single-pass levels only.
struct PlaneMaps {
    CUtensorMap r[K1_NRY], pA[K1_NRY], pB[K1_NRY], dinv[K1_NRY], beta[K1_NRY], e[K1_NRY];
    CUtensorMap rB[K1_NRY], qA[K1_NRY], qB[K1_NRY];
    CUtensorMap ring[K1_NRY];  // 4D: the ring of search directions (two-pass MIXED levels)
};


// Tile shape of K1 on one level: ry node rows per thread, kz planes marched per block.
struct K1Config {
    int ry;
    int kz;
};

// Encode the tensor maps of one level. False if the driver entry point is unavailable or an
// encoding is rejected.
bool make_plane_maps(PlaneMaps* m, const float* r, const float* pA, const float* pB, const float* dinv,
                     const float* beta, const float* e, const Grid& g);

// The single-pass buffers of a level: second residual buffer and the two q buffers.
bool make_plane_maps_sp(PlaneMaps* m, const float* rB, const float* qA, const float* qB, const Grid& g);
// The 4D maps of a level's ring of R search directions.
bool make_ring_maps(PlaneMaps* m, const float* ring, int R, const Grid& g);

// Set the shared-memory limit of every K1 instantiation (both forms) on the current device.
cudaError_t k1_prepare();
// Heuristic tile shape, the candidate shapes an autotuner may try, and validity.
K1Config k1_default(const Grid& g, const Op& op);
int k1_candidates(const Grid& g, K1Config* out, int cap);
bool k1_valid(const K1Config& c);
// Nodes K1 computes on this level: every node off the Dirichlet faces.
int64_t k1_nodes(const Grid& g, const Op& op);
// Most blocks any valid shape launches on this grid (size of the partials buffer).
int max_tma_blocks(const Grid& g);

// p = D^-1 r + beta p_old (p_old = pA or pB), q = A p, e += alpha_prev p_old, p.q.
// cc: the constant-coefficient kernel (the caller has seen every face Dirichlet and the level's
// device flag `uniform` set: one beta everywhere); beta and D^-1 are then constants read once
// from beta32 and dinv32 instead of streamed. If the flag is clear when the kernel runs, it
// records status 6 (stale path) in st and finishes the level without computing.
// tm: device timer that accumulates the durations of these launches, or nullptr.
// ring: the level's ring of search directions, or nullptr (pold_is_b, pnew and e are then used);
// the constant-coefficient kernel only (cc true): the general kernel takes no ring, and a caller
// passes one only with cc.
void launch_pq32_tma(const PlaneMaps& m, int pold_is_b, const K1Config& c, const Grid& g, const Op& op, bool cc,
                     const int* uniform, const float* beta32, const float* dinv32, float* pnew, float* q, float* e,
                     SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm, cudaStream_t s,
                     const RingArgs* ring = nullptr);

// Single-pass step (ECMG_CG_SINGLE_PASS): with (r_in, q_in, p_old) the buffers A (in_b = 0) or
// B (in_b = 1) and the outputs the other three: r = r_in - alpha_prev q_in, e += alpha_prev p_old,
// p = D^-1 r + beta p_old, q = A p; stores r, p, q; the last block sets alpha, the expanded
// next r.z and r.r, the test of update_epilogue and the loop's conditions (loop, update).
// cc as for launch_pq32_tma.
// sets: with a one-beta, all-Dirichlet level (cc) the buffer sets may instead be taken from the
// level state: the step reads set st->p_latest and writes the other (in_b, pnew, qnew, rnew and
// pidx are then unused), and a step that finds a replacement requested returns at once, so that
// several steps can share one replacement check.
struct SpSets {
    float *p[2], *q[2], *r[2];
};
void launch_step32(const PlaneMaps& m, int in_b, const K1Config& c, const Grid& g, const Op& op, bool cc,
                   const int* uniform, const float* beta32, const float* dinv32, float* pnew, float* qnew,
                   float* rnew, float* e, SolveState* st, Partials pr, int pidx, CondHandles ch, KTimer* tm,
                   cudaStream_t s, const SpSets* sets = nullptr);
cudaError_t k1_sp_prepare();

unsigned long long launches_pq_tma();
unsigned long long launches_pq_sp();

}  // namespace ecmg
