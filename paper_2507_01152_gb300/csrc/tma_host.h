// Host side of the tensor-memory-accelerator copies: encoding of tiled
// tensor maps for BF16 operands.  The driver's encoder is reached through
// the runtime's driver entry-point query, so the library does not link
// the driver library directly.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ussim {
namespace tma {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encoder() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// BF16 tensor of `rank` dimensions (innermost first): extents `dims`,
// byte strides of dimensions 1.. in `strides`, copy box `box`, traversal
// steps `steps` (1 = dense).  The shared-memory image of a box has rows of
// box[0] elements; `swizzle_bytes` (128, 64 or 0) names the swizzle of
// those rows, which must then be exactly that long.  Elements outside the
// tensor read as zero.  Returns false when the driver rejects the
// description.
inline bool encode_bf16(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                        const uint32_t* box, const uint32_t* steps, int swizzle_bytes = 128) {
  const EncodeTiledFn f = encoder();
  if (!f || (swizzle_bytes && (uint64_t)box[0] * 2 != (uint64_t)swizzle_bytes)) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = steps[i];
    if (i + 1 < rank) st[i] = strides[i];
  }
  return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), d, st, b, e,
           CU_TENSOR_MAP_INTERLEAVE_NONE,
           swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : (swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE),
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma
}  // namespace ussim
