// stencil_core.cuh -- the matrix-free Q1 operator of Sec. 2 at one node, shared by every
// stencil kernel (jcg.cu, pq_tma.cu).
//
// With S_d(i) the sum of beta over the elements containing node i and node i+d, and K(d) the
// beta = 1 element-matrix entry of the offset class of d (Op), every element matrix has zero
// row sums, so
//     (A v)_i = sum_{d != 0} K(d) S_d(i) (v_{i+d} - v_i)  +  Robin face terms.
// The difference form keeps FP32 evaluation accurate: the differences of neighbouring values
// are exact, and no O(1) terms cancel.
//
// V(dx, dy, dz) returns the operand at node i + (dx, dy, dz); every call below uses
// compile-time offsets, so a caller may keep its operand window in registers.
#pragma once

#include "ecmg_internal.cuh"

namespace ecmg {

__device__ __forceinline__ bool on_dirichlet(const Grid& g, const Op& op, int i, int j, int k)
{
    return (i == 0 && op.bc[0] == 0) || (i == g.nx && op.bc[1] == 0) ||
           (j == 0 && op.bc[2] == 0) || (j == g.ny && op.bc[3] == 0) ||
           (k == 0 && op.bc[4] == 0) || (k == g.nz && op.bc[5] == 0);
}

// Offset-class weights of Op in the arithmetic type. A conversion from FP64 runs on the FP64
// pipe, which on GB300 is 1/64 of the FP32 rate.
template <typename VT>
struct Weights;
template <>
struct Weights<double> {
    double wf0, wf1, wf2, we0, we1, we2, wc;
    __device__ __forceinline__ explicit Weights(const Op& op)
        : wf0(op.wf[0]), wf1(op.wf[1]), wf2(op.wf[2]), we0(op.we[0]), we1(op.we[1]), we2(op.we[2]), wc(op.wc)
    {
    }
};
// FP32 weights come rounded from the host, so the kernel holds no conversion the compiler
// could re-issue inside a loop.
template <>
struct Weights<float> {
    float wf0, wf1, wf2, we0, we1, we2, wc;
    __device__ __forceinline__ explicit Weights(const Op& op)
        : wf0(op.wf32[0]), wf1(op.wf32[1]), wf2(op.wf32[2]), we0(op.we32[0]), we1(op.we32[1]),
          we2(op.we32[2]), wc(op.wc32)
    {
    }
};

// b<ex><ey><ez>: beta of the element (i-1+ex, j-1+ey, k-1+ez). CUBE: cubic elements, where
// the face-neighbour weights vanish and edge and corner weights coincide (both -h/12), so the
// sum needs one weight and no face terms.
template <bool CUBE, typename VT, typename VF>
__device__ __forceinline__ VT q1_interior(VF V, VT b000, VT b100, VT b010, VT b110, VT b001, VT b101,
                                         VT b011, VT b111, const Weights<VT>& w)
{
    const VT xc = V(0, 0, 0);
    // pair sums over the axis an offset does not cross
    const VT sx00 = b000 + b100, sx01 = b010 + b110, sx10 = b001 + b101, sx11 = b011 + b111;  // [ez][ey]
    const VT sy00 = b000 + b010, sy01 = b100 + b110, sy10 = b001 + b011, sy11 = b101 + b111;  // [ez][ex]
    const VT sz00 = b000 + b001, sz01 = b100 + b101, sz10 = b010 + b011, sz11 = b110 + b111;  // [ey][ex]
    const VT ex = sx00 * (V(0, -1, -1) - xc) + sx01 * (V(0, 1, -1) - xc) + sx10 * (V(0, -1, 1) - xc) +
                  sx11 * (V(0, 1, 1) - xc);
    const VT ey = sy00 * (V(-1, 0, -1) - xc) + sy01 * (V(1, 0, -1) - xc) + sy10 * (V(-1, 0, 1) - xc) +
                  sy11 * (V(1, 0, 1) - xc);
    const VT ez = sz00 * (V(-1, -1, 0) - xc) + sz01 * (V(1, -1, 0) - xc) + sz10 * (V(-1, 1, 0) - xc) +
                  sz11 * (V(1, 1, 0) - xc);
    const VT cc = b000 * (V(-1, -1, -1) - xc) + b100 * (V(1, -1, -1) - xc) + b010 * (V(-1, 1, -1) - xc) +
                  b110 * (V(1, 1, -1) - xc) + b001 * (V(-1, -1, 1) - xc) + b101 * (V(1, -1, 1) - xc) +
                  b011 * (V(-1, 1, 1) - xc) + b111 * (V(1, 1, 1) - xc);
    if (CUBE) return w.wc * ((ex + ey) + (ez + cc));
    const VT fx = (sz01 + sz11) * (V(1, 0, 0) - xc) + (sz00 + sz10) * (V(-1, 0, 0) - xc);
    const VT fy = (sx01 + sx11) * (V(0, 1, 0) - xc) + (sx00 + sx10) * (V(0, -1, 0) - xc);
    const VT fz = (sx10 + sx11) * (V(0, 0, 1) - xc) + (sx00 + sx01) * (V(0, 0, -1) - xc);
    return w.wf0 * fx + w.wf1 * fy + w.wf2 * fz + w.we0 * ex + w.we1 * ey + w.we2 * ez + w.wc * cc;
}

// Element count along one axis between node index a and a + d (d in -1..1), grid size n.
__device__ __forceinline__ int elems_between(int a, int n, int d)
{
    return d < 0 ? (a >= 1) : d > 0 ? (a < n) : (a >= 1) + (a < n);
}

// Robin face-mass weight alpha_F h_a h_b / 36 of face f in the arithmetic type (rounded on the
// host: no FP64 instruction in an FP32 kernel, and no FP64 divide anywhere).
template <typename VT>
__device__ __forceinline__ VT robin_weight(const Op& op, int f);
template <>
__device__ __forceinline__ double robin_weight<double>(const Op& op, int f) { return op.rw64[f]; }
template <>
__device__ __forceinline__ float robin_weight<float>(const Op& op, int f) { return op.rw32[f]; }

// alpha_F times the face mass matrix, summed over every Robin face through the node (the
// Gamma_R part of the bilinear form of Sec. 2): the face mass entry between the node and its
// in-face neighbour (da, db) is alpha_F h_a h_b / 36 times the number of face quads they share
// times 2 per axis with da = 0 (resp. db = 0). Fully unrolled: offsets are compile-time.
template <typename VT, typename VF>
__device__ __forceinline__ VT q1_robin(VF V, int i, int j, int k, const Grid& g, const Op& op)
{
    VT acc = VT(0);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int an = f / 2;
        const int ia = an == 0 ? i : an == 1 ? j : k;
        const int na = an == 0 ? g.nx : an == 1 ? g.ny : g.nz;
        if (!((op.robin_mask >> f) & 1) || ia != ((f & 1) ? na : 0)) continue;
        // in-face axes a < b
        const int aa = an == 0 ? 1 : 0, ab = an == 2 ? 1 : 2;
        const int ja = aa == 0 ? i : j, jb = ab == 1 ? j : k;
        const int nA = aa == 0 ? g.nx : g.ny, nB = ab == 1 ? g.ny : g.nz;
        const VT rw = robin_weight<VT>(op, f);
#pragma unroll
        for (int db = -1; db <= 1; ++db)
#pragma unroll
            for (int da = -1; da <= 1; ++da) {
                const int c = elems_between(ja, nA, da) * elems_between(jb, nB, db);
                if (!c) continue;
                const VT w = rw * (VT)(c * (da ? 1 : 2) * (db ? 1 : 2));
                const int dx = aa == 0 ? da : 0;
                const int dy = aa == 1 ? da : (ab == 1 ? db : 0);
                const int dz = ab == 2 ? db : 0;
                acc += w * V(dx, dy, dz);
            }
    }
    return acc;
}

// The same sum with rolled loops, for operands addressable with run-time offsets (shared
// memory): much smaller code than the unrolled form.
template <typename VT, typename VF>
__device__ __forceinline__ VT q1_robin_rolled(VF V, int i, int j, int k, const Grid& g, const Op& op)
{
    VT acc = VT(0);
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
        const int an = f / 2;
        const int ia = an == 0 ? i : an == 1 ? j : k;
        const int na = an == 0 ? g.nx : an == 1 ? g.ny : g.nz;
        if (!((op.robin_mask >> f) & 1) || ia != ((f & 1) ? na : 0)) continue;
        const int aa = an == 0 ? 1 : 0, ab = an == 2 ? 1 : 2;
        const int ja = aa == 0 ? i : j, jb = ab == 1 ? j : k;
        const int nA = aa == 0 ? g.nx : g.ny, nB = ab == 1 ? g.ny : g.nz;
        const VT rw = robin_weight<VT>(op, f);
#pragma unroll 1
        for (int db = -1; db <= 1; ++db)
#pragma unroll 1
            for (int da = -1; da <= 1; ++da) {
                const int c = elems_between(ja, nA, da) * elems_between(jb, nB, db);
                if (!c) continue;
                const VT w = rw * (VT)(c * (da ? 1 : 2) * (db ? 1 : 2));
                const int dx = aa == 0 ? da : 0;
                const int dy = aa == 1 ? da : (ab == 1 ? db : 0);
                const int dz = ab == 2 ? db : 0;
                acc += w * V(dx, dy, dz);
            }
    }
    return acc;
}

// ROLLED = true when V accepts run-time offsets (operand in shared memory); false when the
// operand lives in registers and every offset must be a compile-time constant. ROBIN = false
// compiles the Robin terms out (no Robin face with alpha != 0): the kernel then carries no
// FP64 arithmetic at all, which matters on GB300 even for predicated-off instructions.
template <bool ROLLED, bool ROBIN, bool CUBE, typename VT, typename VF>
__device__ __forceinline__ VT q1_apply(VF V, VT b000, VT b100, VT b010, VT b110, VT b001, VT b101, VT b011,
                                      VT b111, int i, int j, int k, const Grid& g, const Op& op,
                                      const Weights<VT>& w)
{
    VT Av = q1_interior<CUBE, VT>(V, b000, b100, b010, b110, b001, b101, b011, b111, w);
    if (ROBIN) {
        if (i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz) {
            if (ROLLED) Av += q1_robin_rolled<VT>(V, i, j, k, g, op);
            else Av += q1_robin<VT>(V, i, j, k, g, op);
        }
    }
    return Av;
}

// f_h at the free node (i, j, k) at offset o: b minus A x, where x holds g_D on the Dirichlet
// nodes and 0 elsewhere, so only nodes next to a Dirichlet face see the lift. Operands come
// straight from global memory (the lift touches one layer of nodes per Dirichlet face).
template <bool ROBIN, bool CUBE>
__device__ __forceinline__ double fh_at(const Grid& g, const Op& op, const Weights<double>& wts,
                                        const double* __restrict__ beta, const double* __restrict__ x,
                                        const double* __restrict__ b, int64_t o, int i, int j, int k)
{
    double f = b[o];
    const bool near = (op.bc[0] == 0 && i <= 1) || (op.bc[1] == 0 && i >= g.nx - 1) ||
                      (op.bc[2] == 0 && j <= 1) || (op.bc[3] == 0 && j >= g.ny - 1) ||
                      (op.bc[4] == 0 && k <= 1) || (op.bc[5] == 0 && k >= g.nz - 1);
    if (near) {
        auto V = [&](int ddx, int ddy, int ddz) -> double {
            return x[o + (int64_t)ddz * g.plane + (int64_t)ddy * g.pitch + ddx];
        };
        auto be = [&](int ex, int ey, int ez) { return beta[g.off(i - 1 + ex, j - 1 + ey, k - 1 + ez)]; };
        f -= q1_apply<true, ROBIN, CUBE, double>(V, be(0, 0, 0), be(1, 0, 0), be(0, 1, 0), be(1, 1, 0), be(0, 0, 1),
                                                 be(1, 0, 1), be(0, 1, 1), be(1, 1, 1), i, j, k, g, op, wts);
    }
    return f;
}

__device__ __forceinline__ bool op_has_robin(const Op& op) { return op.robin != 0; }

}  // namespace ecmg
