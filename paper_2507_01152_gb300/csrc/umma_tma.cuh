// Operand loaders of the tcgen05 tile GEMM that stage each K step with
// tiled tensor copies (TMA) instead of per-thread cp.async: the tensor
// maps are encoded on the host for every call and passed in the kernel's
// parameter space.
#pragma once
#include <cuda_bf16.h>

#include "tma_host.h"
#include "umma_gemm.cuh"

namespace ussim {
namespace umma {

// A [M][K] and B [N][K] as rows with their own pitch (plain GEMM, the
// transposed convolution's forward pass); rows and K past the end read 0
struct RowsTmaLoader {
  static constexpr bool kTma = true;
  CUtensorMap ta, tb;
  __device__ void issue_a(uint32_t as, int m0, int kt, uint32_t bar) const { tma_load_2d(as, &ta, kt * kBK, m0, bar); }
  __device__ void issue_b(uint32_t bs, int n0, int kt, uint32_t bar) const { tma_load_2d(bs, &tb, kt * kBK, n0, bar); }
};

// a [rows][K] BF16 matrix with row pitch `pitch` elements, copied in
// boxes of 64 K-elements x box_rows rows
inline bool rows_map(CUtensorMap* m, const __nv_bfloat16* p, long long pitch, int rows, int K, int box_rows) {
  const uint64_t d[2] = {(uint64_t)K, (uint64_t)rows}, st[1] = {(uint64_t)pitch * 2};
  const uint32_t bx[2] = {(uint32_t)kBK, (uint32_t)box_rows}, e[2] = {1, 1};
  return tma::encode_bf16(m, p, 2, d, st, bx, e);
}

}  // namespace umma
}  // namespace ussim
