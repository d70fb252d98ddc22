// Plain BF16 GEMM on the tcgen05 tile kernel (C = A B^T, FP32 out): the
// building block of the surrogate's implicit-GEMM convolutions, exposed
// as its own op so it can be checked in isolation.  Operands are staged
// with tensor copies (rows and K past the end read as zero).
#include <cuda_bf16.h>

#include "ussim_surrogate.h"
#include "umma_tma.cuh"

namespace ussim {
namespace {

using namespace umma;

struct F32Store {
  float* C;
  int N;
  __device__ void store(int m, int n0, const float* v, bool valid) const {
    if (!valid) return;
    float4* dst = reinterpret_cast<float4*>(C + (size_t)m * N + n0);
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  }
};


}  // namespace
}  // namespace ussim

using namespace ussim;

extern "C" us_status us_gemm_bf16_nt(const uint16_t* A, const uint16_t* B, float* C, int32_t M, int32_t N, int32_t K,
                                     uint32_t* err, void* stream) {
  if (!A || !B || !C || !err || M < 1 || N < 32 || K < 8 || (N % 32) || (K % 8)) return US_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15u)
    return US_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const auto* a = reinterpret_cast<const __nv_bfloat16*>(A);
  const auto* b = reinterpret_cast<const __nv_bfloat16*>(B);
  cudaError_t e;
  const int bn = (N % 256 == 0) ? 256 : (N % 128 == 0) ? 128 : (N % 64 == 0) ? 64 : 32;
  umma::RowsTmaLoader ld;
  if (!umma::rows_map(&ld.ta, a, K, M, K, umma::kBM) || !umma::rows_map(&ld.tb, b, K, N, K, bn)) return US_ERR_CUDA;
  F32Store ep{C, N};
  switch (bn) {
    case 256: e = umma::launch_umma_gemm<256, 1>(ld, ep, M, N, K, err, st); break;
    case 128: e = umma::launch_umma_gemm<128, 2>(ld, ep, M, N, K, err, st); break;
    case 64: e = umma::launch_umma_gemm<64, 4>(ld, ep, M, N, K, err, st); break;
    default: e = umma::launch_umma_gemm<32, 4>(ld, ep, M, N, K, err, st); break;
  }
  return e == cudaSuccess ? US_OK : US_ERR_CUDA;
}
