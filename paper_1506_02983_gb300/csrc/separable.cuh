// separable.cuh -- on-device assembly from separable data (separable.cu).
#pragma once

#include "ecmg_internal.cuh"

namespace ecmg {

// Doubles of the 1D factor arrays of one level: terms x ((nx+1) + (ny+1) + (nz+1)), term-major,
// x then y then z.
int64_t sep_factor_len(const Grid& g, int terms);
// Finest level: H = 1D hat integrals of the Gauss samples (terms x 3 (nx + ny + nz), term-major,
// x then y then z, three points per interval), then b = sum_t Hx_t Hy_t Hz_t on every node.
void sep_load_finest(const Grid& g, int terms, const double* samples, double* H, double* b, cudaStream_t s);
// Coarse level gc from the finer level gf: Fc = restriction (restrict_, the load functional) or
// injection (nodal data) of each 1D factor, then out = sum_t Fx_t Fy_t Fz_t.
void sep_coarsen(const Grid& gc, const Grid& gf, int terms, const double* Ff, double* Fc, bool restrict_,
                 double* out, cudaStream_t s);
// out = sum_t Fx_t Fy_t Fz_t on every node of level g (nodal factors F of that level).
void sep_nodal(const Grid& g, int terms, const double* F, double* out, cudaStream_t s);
// beta = value on every element of level g.
void fill_beta(const Grid& g, double value, double* beta, cudaStream_t s);

unsigned long long launches_separable();

}  // namespace ecmg
