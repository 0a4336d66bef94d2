// fsp_tma_host.cu -- host side of the TMA-staged passes: tensor maps.
//
// cuTensorMapEncodeTiled is a driver-API function; it is looked up once
// through the runtime (cudaGetDriverEntryPointByVersion), so the library links
// the runtime only.  Encoding is pure host work (no GPU call), cheap enough to
// do for every solve: the maps hold the addresses of that solve's buffers and
// travel to the kernels as __grid_constant__ parameters.
#include "fsp_internal.h"

#include <cuda.h>
#include <mutex>

namespace fsp {

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
    });
    return fn;
}
} // namespace

int encode_tensor_map(void *map, const void *base, int rank, int elem_bytes, const unsigned long long *dims,
                      const unsigned long long *strides, const unsigned *box)
{
    EncodeTiled fn = encoder();
    if (!fn) return (int)CUDA_ERROR_NOT_FOUND;
    if (rank < 1 || rank > 5 || (elem_bytes != 4 && elem_bytes != 8)) return (int)CUDA_ERROR_INVALID_VALUE;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) st[i] = strides[i];
    }
    const CUtensorMapDataType ty = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return (int)fn(reinterpret_cast<CUtensorMap *>(map), ty, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

} // namespace fsp
