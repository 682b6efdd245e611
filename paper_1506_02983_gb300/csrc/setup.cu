// setup.cu -- per-level set-up of Alg. 4: packing of the caller's finest arrays into the
// ghost-padded device layout, beta averaging, injection, load vectors (Sec. 2) and the
// Jacobi diagonal of JCG. All of it runs once per level per solve; FP64 throughout.
#include "ecmg_internal.cuh"
#include "setup_core.cuh"

namespace ecmg {

namespace {

__device__ unsigned long long g_launches = 0;  // kernel executions of this file
#define COUNT_LAUNCH()                                                                   \
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y | threadIdx.z) == 0) \
        atomicAdd(&g_launches, 1ull)

// The GPU's global timer (ns) into *t: the time stamps of the per-level solve times.
__global__ void k_stamp(unsigned long long* t)
{
    COUNT_LAUNCH();
    *t = global_ns();
}

constexpr int TPB = 256;
constexpr int TX = 32, TY = 8;  // node-parallel kernels: 32 x 8 nodes of a plane per block

inline int blocks_for(int64_t n) { return (int)((n + TPB - 1) / TPB); }
// one thread per point of an (mx+1) x (my+1) x (mz+1) box: x, y tiles and one block row per plane
inline dim3 grid3(int mx, int my, int mz) { return dim3((mx + TX) / TX, (my + TY) / TY, mz + 1); }
#define POINT_IJK(MX, MY)                                                            \
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y; \
    const int k = blockIdx.z;                                                       \
    if (i > (MX) || j > (MY)) return
// Kernels that may find nothing to do on most nodes (a one-beta cube keeps a single FP32 D^-1;
// the Dirichlet shell is a thin layer), and the whole-array copies between the caller's dense
// layout and the padded one, walk ZT planes per block, so that the grid does not cost a block
// launch per node row and plane (the copies: 0.50 ms at 513^3 with one plane per block).
constexpr int ZT = 16;
inline dim3 grid3z(int mx, int my, int mz) { return dim3((mx + TX) / TX, (my + TY) / TY, (mz + ZT) / ZT); }

// Copy of a nodal array between the dense layout (UNPACK false: dense -> padded) and the padded
// one (true: padded -> dense): node column (i, j) over the block's ZT planes, the loads of four
// planes issued before their stores.
template <bool UNPACK>
__global__ void k_copy_nodal(Grid g, const double* __restrict__ src, double* __restrict__ dst)
{
    COUNT_LAUNCH();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const int k0 = blockIdx.z * ZT, k1 = min(k0 + ZT, g.nz + 1);
    const int64_t plane = (int64_t)(g.nx + 1) * (g.ny + 1);
    const int64_t t0 = i + (int64_t)(g.nx + 1) * j;  // dense index of (i, j, 0)
    for (int k = k0; k < k1; k += 4) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k + u < k1) v[u] = UNPACK ? src[g.off(i, j, k + u)] : src[t0 + plane * (k + u)];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k + u < k1) {
                if (UNPACK) dst[t0 + plane * (k + u)] = v[u];
                else dst[g.off(i, j, k + u)] = v[u];
            }
    }
}

__global__ void k_pack_elements(Grid g, const double* __restrict__ dense, double* __restrict__ dst)
{
    COUNT_LAUNCH();
    POINT_IJK(g.nx - 1, g.ny - 1);
    const int64_t t = i + (int64_t)g.nx * (j + (int64_t)g.ny * k);  // dense index
    dst[g.off(i, j, k)] = dense[t];
}

// The finest level's beta in one pass over the caller's dense array, one thread per element of
// the level below: its eight fine elements are packed into the padded FP64 layout and into FP32,
// compared with element (0, 0, 0) for the uniform flag (bit patterns), and averaged for the
// coarse beta in the order of coarse_beta_at. Fine rows are even in length, so every access is
// an aligned pair.
__global__ void k_beta_finest(Grid g, Grid gc, const double* __restrict__ dense, double* __restrict__ beta,
                              float* __restrict__ beta32, int* flag, double* __restrict__ bc)
{
    COUNT_LAUNCH();
    POINT_IJK(gc.nx - 1, gc.ny - 1);
    const long long ref = __double_as_longlong(dense[0]);
    double2 v[4];  // rows (b, c) = (0, 0), (1, 0), (0, 1), (1, 1): elements 2i and 2i + 1
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int fj = 2 * j + (r & 1), fk = 2 * k + (r >> 1);
        const int64_t t = 2 * i + (int64_t)g.nx * (fj + (int64_t)g.ny * fk);  // dense index, even
        v[r] = *reinterpret_cast<const double2*>(dense + t);
    }
    bool same = true;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t o = g.off(2 * i, 2 * j + (r & 1), 2 * k + (r >> 1));  // even: a 16-byte pair
        *reinterpret_cast<double2*>(beta + o) = v[r];
        *reinterpret_cast<float2*>(beta32 + o) = make_float2((float)v[r].x, (float)v[r].y);
        same = same && __double_as_longlong(v[r].x) == ref && __double_as_longlong(v[r].y) == ref;
    }
    double sum = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) sum += (c & 1) ? v[c >> 1].y : v[c >> 1].x;
    bc[gc.off(i, j, k)] = sum / 8.0;
    if (!same) *flag = 0;
}

__global__ void k_coarsen_beta(Grid gc, const double* __restrict__ bf, Grid gf, double* __restrict__ bc)
{
    COUNT_LAUNCH();
    POINT_IJK(gc.nx - 1, gc.ny - 1);
    bc[gc.off(i, j, k)] = coarse_beta_at(bf, gf, i, j, k);
}

__global__ void k_inject(Grid gc, const double* __restrict__ vf, Grid gf, double* __restrict__ vc)
{
    COUNT_LAUNCH();
    POINT_IJK(gc.nx, gc.ny);
    vc[gc.off(i, j, k)] = vf[gf.off(2 * i, 2 * j, 2 * k)];
}

// P^T b with the weights (1/2, 1, 1/2) of the trilinear prolongation per axis, summed axis by
// axis: per fine plane a block stages the 65 x 17 fine values under its 32 x 8 coarse nodes,
// sums them along x and then y in shared memory, and forms each coarse value from the sums of
// three consecutive fine planes. 14.5 FP64 operations per coarse node instead of the 27 of the
// full weighted sum (restrict_at); the same weights, summed in another order.
constexpr int RKZ = 8;  // coarse planes per block
__global__ void __launch_bounds__(TX * TY) k_restrict(Grid gc, const double* __restrict__ bf, Grid gf,
                                                      double* __restrict__ bc)
{
    COUNT_LAUNCH();
    constexpr int SR = 2 * TY + 1, SCOL = 2 * TX + 1;  // staged fine rows and columns
    __shared__ double S[SR][SCOL];
    __shared__ double T[SR][TX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
    const int I0 = blockIdx.x * TX, J0 = blockIdx.y * TY, K0 = blockIdx.z * RKZ;
    const int K1 = min(K0 + RKZ, gc.nz + 1);  // coarse planes [K0, K1)
    const int I = I0 + tx, J = J0 + ty;
    const bool own = I <= gc.nx && J <= gc.ny;
    double t2m = 0.0, t2c = 0.0;  // the y, x sums of fine planes kf - 2 and kf - 1
    for (int kf = 2 * K0 - 1; kf <= 2 * K1 - 1; ++kf) {
        const int64_t pb = gf.plane_base(kf);
        for (int c = tid; c < SR * SCOL; c += TX * TY) {
            const int r = c / SCOL, col = c % SCOL;
            const int jf = 2 * J0 - 1 + r, ifn = 2 * I0 - 1 + col;
            S[r][col] = (jf <= gf.ny + 1 && ifn <= gf.nx + 1) ? bf[pb + gf.in_plane(ifn, jf)] : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < SR; r += TY) T[r][tx] = S[r][2 * tx + 1] + 0.5 * (S[r][2 * tx] + S[r][2 * tx + 2]);
        __syncthreads();
        const double t2 = T[2 * ty + 1][tx] + 0.5 * (T[2 * ty][tx] + T[2 * ty + 2][tx]);
        // fine plane 2K + 1 closes coarse plane K
        if (kf > 2 * K0 && (kf & 1) && own) bc[gc.off(I, J, (kf - 1) / 2)] = t2c + 0.5 * (t2m + t2);
        t2m = t2c;
        t2c = t2;
    }
}

__global__ void k_nodal_load(Grid g, Op op, const double* __restrict__ f,
                             const double* __restrict__ gR, double* __restrict__ b)
{
    COUNT_LAUNCH();
    POINT_IJK(g.nx, g.ny);
    b[g.off(i, j, k)] = nodal_load_at(g, op, f, gR, i, j, k);
}

__global__ void k_gauss_load(Grid g, Op op, const double* __restrict__ f27, const double* __restrict__ gR,
                             double* __restrict__ b)
{
    COUNT_LAUNCH();
    POINT_IJK(g.nx, g.ny);
    b[g.off(i, j, k)] = gauss_load_at(g, op, f27, gR, i, j, k);
}

// Jacobi diagonal: diag = w0 * (sum of the 8 element betas) + Robin face mass diagonal.
// Dirichlet nodes get dinv = 0, which also masks them in every JCG kernel.
__global__ void k_jacobi64(Grid g, Op op, const double* __restrict__ beta, double* __restrict__ dinv64, int precond)
{
    COUNT_LAUNCH();
    POINT_IJK(g.nx, g.ny);
    if (!precond) {  // plain CG (ECMG_cg): the identity on free nodes
        dinv64[g.off(i, j, k)] = on_dirichlet(g, op, i, j, k) ? 0.0 : 1.0;
        return;
    }
    double B = 0.0;
    for (int c = 0; c < 8; ++c)
        B += beta[g.off(i - 1 + (c & 1), j - 1 + ((c >> 1) & 1), k - 1 + (c >> 2))];
    double d = op.w0 * B;
    const int idx[3] = {i, j, k};
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int fc = 0; fc < 6; ++fc) {
        if (!((op.robin_mask >> fc) & 1)) continue;
        int an = fc / 2;
        if (idx[an] != ((fc & 1) ? nn[an] : 0)) continue;
        int aa = (an == 0) ? 1 : 0, ab = (an == 2) ? 1 : 2;
        // alpha h_a h_b / 9 per shared face quad pair: the diagonal of the face mass matrix
        d += op.rw64[fc] * (double)(4 * cnt1(idx[aa], nn[aa], 0) * cnt1(idx[ab], nn[ab], 0));
    }
    dinv64[g.off(i, j, k)] = on_dirichlet(g, op, i, j, k) ? 0.0 : 1.0 / d;
}

// The same diagonal in FP32 arithmetic from the FP32 betas, for the FP32 iteration of MIXED
// mode: no FP64 division or conversion per node (FP64 runs at 1/64 of the FP32 rate on GB300).
// Robin terms (boundary nodes only) are formed in FP64 and rounded.
// uniform: the level's flag, already set by the set-up. On a level with one beta, every face
// Dirichlet and cubic elements the FP32 iteration reads D^-1 at node (1, 1, 1) only (it is the
// same on every free node), so the other nodes are skipped.

// g_D on the Dirichlet nodes only: a block walks ZT planes of its node columns; a column off
// the Dirichlet x and y faces holds Dirichlet nodes only on the z faces.
__global__ void k_pack_dirichlet(Grid g, Op op, const double* __restrict__ dense, double* __restrict__ dst)
{
    COUNT_LAUNCH();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const bool column = (i == 0 && op.bc[0] == 0) || (i == g.nx && op.bc[1] == 0) || (j == 0 && op.bc[2] == 0) ||
                        (j == g.ny && op.bc[3] == 0);
    const int k1 = min((int)(blockIdx.z + 1) * ZT, g.nz + 1);
    for (int k = blockIdx.z * ZT; k < k1; ++k) {
        if (!column && !((k == 0 && op.bc[4] == 0) || (k == g.nz && op.bc[5] == 0))) continue;
        const int64_t t = i + (int64_t)(g.nx + 1) * (j + (int64_t)(g.ny + 1) * k);  // dense index
        dst[g.off(i, j, k)] = dense[t];
    }
}

__global__ void k_jacobi32(Grid g, Op op, const float* __restrict__ beta32, float* __restrict__ dinv32, int precond,
                           const int* __restrict__ uniform)
{
    COUNT_LAUNCH();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const bool diri = (op.bc[0] | op.bc[1] | op.bc[2] | op.bc[3] | op.bc[4] | op.bc[5]) == 0;
    const bool one = uniform && diri && op.cube && *uniform;  // only node (1, 1, 1) is read
    if (one && !(i == 1 && j == 1)) return;
    const int k1 = min((int)(blockIdx.z + 1) * ZT, g.nz + 1);
    for (int k = blockIdx.z * ZT; k < k1; ++k) {
        if (one && k != 1) continue;
        dinv32[g.off(i, j, k)] = jacobi32_at(g, op, beta32, i, j, k, precond);
    }
}

// x = g_D on Dirichlet nodes, 0 on free nodes (gD == nullptr: zero everywhere).
__global__ void k_dirichlet_ext(Grid g, Op op, const double* __restrict__ gD, double* __restrict__ x, int shell)
{
    COUNT_LAUNCH();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    // shell: only nodes within two steps of a Dirichlet face
    auto near = [](int a, int n, int lo, int hi) { return (lo == 0 && a <= 2) || (hi == 0 && a >= n - 2); };
    const bool column = !shell || near(i, g.nx, op.bc[0], op.bc[1]) || near(j, g.ny, op.bc[2], op.bc[3]);
    const int k1 = min((int)(blockIdx.z + 1) * ZT, g.nz + 1);
    for (int k = blockIdx.z * ZT; k < k1; ++k) {
        if (!column && !near(k, g.nz, op.bc[4], op.bc[5])) continue;
        const int64_t o = g.off(i, j, k);
        x[o] = (gD && on_dirichlet(g, op, i, j, k)) ? gD[o] : 0.0;
    }
}

__global__ void k_uniform(Grid g, const double* __restrict__ beta, int* flag)
{
    COUNT_LAUNCH();
    POINT_IJK(g.nx - 1, g.ny - 1);
    // bit patterns compared as integers (an FP64 compare runs at 1/64 of the FP32 rate); every
    // writer stores the same value
    const long long* bb = reinterpret_cast<const long long*>(beta);
    if (bb[g.off(i, j, k)] != bb[g.off(0, 0, 0)]) *flag = 0;
}

__global__ void k_set_flag(int* flag)
{
    COUNT_LAUNCH();
    *flag = 1;
}

__global__ void k_convert_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n)
{
    COUNT_LAUNCH();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

// beta32 = beta over the whole padded level (ghost elements included) and, in the same pass,
// flag = 0 when a real element's beta differs from element (0, 0, 0)'s (bit patterns compared
// as integers). Row jj, plane kk of the padded layout per thread row.
__global__ void k_beta32_uniform(Grid g, const double* __restrict__ beta, float* __restrict__ beta32, int* flag)
{
    COUNT_LAUNCH();
    const int ii = blockIdx.x * TX + threadIdx.x, jj = blockIdx.y * TY + threadIdx.y, kk = blockIdx.z;
    if (ii >= g.pitch || jj >= g.ny + 3) return;
    const int64_t t = (int64_t)kk * g.plane + (int64_t)jj * g.pitch + ii;
    const double v = beta[t];
    beta32[t] = (float)v;
    const int i = ii - XL, j = jj - 1, k = kk - 1;  // element (i, j, k) sits at its lowest corner node
    if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz &&
        __double_as_longlong(v) != __double_as_longlong(beta[g.off(0, 0, 0)]))
        *flag = 0;
}

__global__ void k_convert_f64(const float* __restrict__ src, double* __restrict__ dst, int64_t n)
{
    COUNT_LAUNCH();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (double)src[t];
}

}  // namespace

void beta32_uniform(const Grid& g, const double* beta, float* beta32, int* flag, cudaStream_t s)
{
    k_set_flag<<<1, 1, 0, s>>>(flag);
    k_beta32_uniform<<<dim3((g.pitch + TX - 1) / TX, (g.ny + 3 + TY - 1) / TY, g.nz + 3), dim3(TX, TY), 0, s>>>(
        g, beta, beta32, flag);
}

void uniform_check(const Grid& g, const double* beta, int* flag, cudaStream_t s)
{
    k_set_flag<<<1, 1, 0, s>>>(flag);
    k_uniform<<<grid3(g.nx - 1, g.ny - 1, g.nz - 1), dim3(TX, TY), 0, s>>>(g, beta, flag);
}

void convert_f32(const double* src, float* dst, int64_t n, cudaStream_t s)
{
    int b = blocks_for(n);
    k_convert_f32<<<b < 4096 ? b : 4096, TPB, 0, s>>>(src, dst, n);
}

void convert_f64(const float* src, double* dst, int64_t n, cudaStream_t s)
{
    int b = blocks_for(n);
    k_convert_f64<<<b < 4096 ? b : 4096, TPB, 0, s>>>(src, dst, n);
}

void pack_nodal(const Grid& g, const double* dense, double* dst, cudaStream_t s)
{
    k_copy_nodal<false><<<grid3z(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, dense, dst);
}
void pack_dirichlet(const Grid& g, const Op& op, const double* dense, double* dst, cudaStream_t s)
{
    k_pack_dirichlet<<<grid3z(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, op, dense, dst);
}
// The caller's output array as a device-side pointer (null: nothing to write), so that a recorded
// graph can write a different array at every launch: k_set_out stores it, k_unpack_out copies.
__global__ void k_set_out(double** slot, double* out)
{
    COUNT_LAUNCH();
    *slot = out;
}
__global__ void k_unpack_out(Grid g, const double* __restrict__ src, double* const* slot)
{
    COUNT_LAUNCH();
    double* dst = *slot;
    if (!dst) return;
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const int k0 = blockIdx.z * ZT, k1 = min(k0 + ZT, g.nz + 1);
    const int64_t plane = (int64_t)(g.nx + 1) * (g.ny + 1);
    const int64_t t0 = i + (int64_t)(g.nx + 1) * j;
    for (int k = k0; k < k1; k += 4) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k + u < k1) v[u] = src[g.off(i, j, k + u)];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k + u < k1) dst[t0 + plane * (k + u)] = v[u];
    }
}
void set_out(double** slot, double* out, cudaStream_t s) { k_set_out<<<1, 1, 0, s>>>(slot, out); }
void unpack_out(const Grid& g, const double* src, double* const* slot, cudaStream_t s)
{
    k_unpack_out<<<grid3z(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, src, slot);
}
void unpack_nodal(const Grid& g, const double* src, double* dense, cudaStream_t s)
{
    k_copy_nodal<true><<<grid3z(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, src, dense);
}
void pack_elements(const Grid& g, const double* dense, double* dst, cudaStream_t s)
{
    k_pack_elements<<<grid3(g.nx - 1, g.ny - 1, g.nz - 1), dim3(TX, TY), 0, s>>>(g, dense, dst);
}
void beta_finest(const Grid& g, const Grid& gc, const double* dense, double* beta, float* beta32, int* flag,
                 double* bc, cudaStream_t s)
{
    k_set_flag<<<1, 1, 0, s>>>(flag);
    k_beta_finest<<<grid3(gc.nx - 1, gc.ny - 1, gc.nz - 1), dim3(TX, TY), 0, s>>>(g, gc, dense, beta, beta32, flag, bc);
}
void coarsen_beta(const Grid& gc, const double* bf, const Grid& gf, double* bc, cudaStream_t s)
{
    k_coarsen_beta<<<grid3(gc.nx - 1, gc.ny - 1, gc.nz - 1), dim3(TX, TY), 0, s>>>(gc, bf, gf, bc);
}
void inject_nodal(const Grid& gc, const double* vf, const Grid& gf, double* vc, cudaStream_t s)
{
    k_inject<<<grid3(gc.nx, gc.ny, gc.nz), dim3(TX, TY), 0, s>>>(gc, vf, gf, vc);
}
void restrict_load(const Grid& gc, const double* bf, const Grid& gf, double* bc, cudaStream_t s)
{
    const dim3 grid((gc.nx + TX) / TX, (gc.ny + TY) / TY, (gc.nz + RKZ) / RKZ);
    k_restrict<<<grid, dim3(TX, TY), 0, s>>>(gc, bf, gf, bc);
}
void nodal_load(const Grid& g, const Op& op, const double* f, const double* gR, double* b,
                cudaStream_t s)
{
    k_nodal_load<<<grid3(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, op, f, gR, b);
}
void gauss_load(const Grid& g, const Op& op, const double* f27, const double* gR, double* b, cudaStream_t s)
{
    k_gauss_load<<<grid3(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, op, f27, gR, b);
}
void jacobi_diag(const Grid& g, const Op& op, const double* beta, double* dinv64, float* dinv32,
                 float* beta32, int precond, cudaStream_t s, const int* uniform)
{
    if (dinv64) k_jacobi64<<<grid3(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, op, beta, dinv64, precond);
    if (beta32) {
        if (!uniform) convert_f32(beta, beta32, g.total, s);  // else beta32_uniform has run
        if (dinv32)
            k_jacobi32<<<grid3z(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, op, beta32, dinv32, precond, uniform);
    }
}
void dirichlet_extension(const Grid& g, const Op& op, const double* gD, double* x, cudaStream_t s, bool shell)
{
    k_dirichlet_ext<<<grid3z(g.nx, g.ny, g.nz), dim3(TX, TY), 0, s>>>(g, op, gD, x, shell ? 1 : 0);
}

void launch_stamp(unsigned long long* t, cudaStream_t s) { k_stamp<<<1, 1, 0, s>>>(t); }

unsigned long long launches_setup()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_launches, sizeof(v));
    return v;
}

}  // namespace ecmg
