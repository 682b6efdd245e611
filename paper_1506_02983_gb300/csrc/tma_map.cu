// tma_map.cu -- tensor maps (TMA descriptors) of level vectors in the padded layout.
#include <cuda.h>
#include <cuda_runtime.h>

#include "ecmg_internal.cuh"
#include "tma.cuh"

namespace ecmg {
namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's encoder, fetched once through the runtime (no link against libcuda).
EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace

bool encode_level_map(CUtensorMap* map, bool fp64, const void* base, const Grid& g, int sx, int sy)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t es = fp64 ? 8 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 3), (cuuint64_t)(g.nz + 3)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)sx, (cuuint32_t)sy, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
               const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_ring_map(CUtensorMap* map, const float* base, const Grid& g, int nvec, int sx, int sy)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t es = 4;
    const cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 3), (cuuint64_t)(g.nz + 3), (cuuint64_t)nvec};
    const cuuint64_t strides[3] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.plane * es,
                                   (cuuint64_t)ring_stride(g.total) * es};
    const cuuint32_t box[4] = {(cuuint32_t)sx, (cuuint32_t)sy, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace ecmg
