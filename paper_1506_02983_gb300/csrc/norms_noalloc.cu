// norms_noalloc.cu -- max-norm and root-mean-square norm of a - b without allocating device
// memory (ecmg_error_norms_noalloc in include/ecmg.h).
//
// Who needs this: callers that must not allocate at the point where they want the norm.
// cudaMalloc and cudaFree can synchronise the whole device, so a caller inside a latency-
// critical loop, inside a host callback, or working under a framework that owns every device
// allocation (a caching allocator or a fixed memory budget) cannot call them. Such a caller
// passes its own input vectors and gets the two norms back; the scratch the reduction needs
// (one partial pair per block and the final pair) lives in the fixed array below, which
// every device that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ecmg.h"

namespace {

constexpr int NA_TPB = 256;                                   // threads per block
constexpr int NA_ITEMS = 64;                                  // elements per thread
constexpr int64_t NA_PER_BLOCK = (int64_t)NA_TPB * NA_ITEMS;  // 16384 elements per block
constexpr int NA_MAX_BLOCKS = (int)(ECMG_NOALLOC_MAX_ELEMS / NA_PER_BLOCK);  // 32768
constexpr int NA_RESULT = 2 * NA_MAX_BLOCKS;                  // index of the final pair
static_assert((int64_t)NA_MAX_BLOCKS * NA_PER_BLOCK == ECMG_NOALLOC_MAX_ELEMS, "limit/scratch mismatch");

// Scratch: [2b] = max |a-b| and [2b+1] = sum (a-b)^2 of block b; then the final pair.
// 2 * 32768 + 2 doubles = 512 KiB + 16 B per device.
static __device__ __align__(256) double g_noalloc_scratch[2 * NA_MAX_BLOCKS + 2];

// Device address of g_noalloc_scratch per device, looked up once per device. The address
// belongs to the device's primary context: after cudaDeviceReset (which destroys that context
// and unloads the module) it would be stale, so resetting a device after the first call on it
// is not supported.
std::mutex g_lookup_mutex;
double* g_scratch_ptr[256] = {};

// The max is taken over the bit patterns of |a-b| as unsigned integers: for non-negative
// doubles that order is the numeric one and every NaN (sign cleared) sorts above +inf, so a NaN
// anywhere in a - b makes max_abs NaN instead of dropping out as it would with fmax.
__device__ __forceinline__ void block_max_sum(unsigned long long& mx, double& ss)
{
    __shared__ unsigned long long smx[32];
    __shared__ double sss[32];
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        smx[warp] = mx;
        sss[warp] = ss;
    }
    __syncthreads();
    if (warp == 0) {
        mx = lane < nw ? smx[lane] : 0ull;
        ss = lane < nw ? sss[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
            ss += __shfl_down_sync(0xffffffffu, ss, o);
        }
    }
}

__device__ __forceinline__ unsigned long long abs_bits(double d)
{
    return (unsigned long long)__double_as_longlong(fabs(d));
}

// One partial pair per block of NA_PER_BLOCK consecutive elements.
__global__ void __launch_bounds__(NA_TPB) k_noalloc_partials(const double* __restrict__ a, const double* __restrict__ b,
                                                            int64_t n, double* __restrict__ scratch)
{
    const int64_t base = (int64_t)blockIdx.x * NA_PER_BLOCK + threadIdx.x;
    unsigned long long mx = 0ull;
    double ss = 0.0;
    for (int it = 0; it < NA_ITEMS; ++it) {
        const int64_t t = base + (int64_t)it * NA_TPB;
        if (t < n) {
            const double d = a[t] - (b ? b[t] : 0.0);
            mx = max(mx, abs_bits(d));
            ss = fma(d, d, ss);
        }
    }
    block_max_sum(mx, ss);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = __longlong_as_double((long long)mx);
        scratch[2 * blockIdx.x + 1] = ss;
    }
}

// Fixed-order reduction of the nb partial pairs into the final pair (deterministic).
__global__ void __launch_bounds__(1024) k_noalloc_final(int nb, double* __restrict__ scratch)
{
    unsigned long long mx = 0ull;
    double ss = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        mx = max(mx, abs_bits(scratch[2 * b]));
        ss += scratch[2 * b + 1];
    }
    block_max_sum(mx, ss);
    if (threadIdx.x == 0) {
        scratch[NA_RESULT] = __longlong_as_double((long long)mx);
        scratch[NA_RESULT + 1] = ss;
    }
}

// The kernels read a and b through the pointers they are given, so those must be reachable
// from the current device: its own device memory, managed memory, or page-locked host memory
// (then the mapped device address is used). Pageable host memory or another device's memory
// would make the kernel fault, so such pointers are refused before any launch. The check is
// cudaPointerGetAttributes, which allocates nothing.
bool device_readable(const double* p, int dev, const double** out)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) error an unknown pointer leaves behind
        return false;
    }
    switch (at.type) {
    case cudaMemoryTypeDevice:
        if (at.device != dev) return false;
        *out = p;
        return true;
    case cudaMemoryTypeManaged:
        *out = p;
        return true;
    case cudaMemoryTypeHost:
        if (!at.devicePointer) return false;
        *out = static_cast<const double*>(at.devicePointer);
        return true;
    default:
        return false;
    }
}

// Set-up, once per device, with that device current: the host-side symbol is only a stand-in,
// so the kernels get the array's device address from cudaGetSymbolAddress.
ecmg_status scratch_address(int dev, double** out)
{
    if (dev < 0 || dev >= 256) return ECMG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_lookup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ECMG_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ECMG_OK;
}

}  // namespace

extern "C" ecmg_status ecmg_error_norms_noalloc(const double* a, const double* b, int64_t n, void* stream,
                                                double* max_abs, double* rms)
{
    if (!a || !max_abs || !rms || n < 1) return ECMG_ERR_INVALID_ARG;
    if (n > ECMG_NOALLOC_MAX_ELEMS) return ECMG_ERR_INVALID_ARG;  // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ECMG_ERR_CUDA;
    if (!device_readable(a, dev, &a) || (b && !device_readable(b, dev, &b))) return ECMG_ERR_INVALID_ARG;
    double* scratch = nullptr;
    const ecmg_status st = scratch_address(dev, &scratch);
    if (st != ECMG_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    k_noalloc_partials<<<nb, NA_TPB, 0, s>>>(a, b, n, scratch);
    k_noalloc_final<<<1, 1024, 0, s>>>(nb, scratch);
    if (cudaGetLastError() != cudaSuccess) return ECMG_ERR_CUDA;
    double res[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(res, scratch + NA_RESULT, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return ECMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ECMG_ERR_CUDA;
    *max_abs = res[0];
    *rms = std::sqrt(res[1] / (double)n);
    return ECMG_OK;
}
