// Plain BF16 GEMM on the tcgen05 tile kernel (C = A B^T, FP32 out): the
// building block of the surrogate's implicit-GEMM convolutions, exposed
// as its own op so it can be checked in isolation.
#include <cuda_bf16.h>

#include "ussim_surrogate.h"
#include "umma_gemm.cuh"

namespace ussim {
namespace {

using namespace umma;

struct RowMajorLoader {
  static constexpr bool kAsync = true;
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int M, N, K, bn;
  struct State {};
  __device__ void prepare(State&, int, int, int) const {}
  __device__ void load(const State&, uint8_t* as, uint8_t* bs, int m0, int n0, int kt, int tid) const {
    for (int c = tid; c < kBM * 8; c += kProducers) {
      const int r = (c & 7) + ((c >> 6) << 3), kc = (c >> 3) & 7;
      const int m = m0 + r, k = kt * kBK + kc * 8;
      const bool v = m < M && k < K;
      cp_async16(as + tile_off(r, kc, kBK), v ? (const void*)(A + (size_t)m * K + k) : (const void*)A, v ? 16u : 0u);
    }
    for (int c = tid; c < bn * 8; c += kProducers) {
      const int r = (c & 7) + ((c >> 6) << 3), kc = (c >> 3) & 7;
      const int n = n0 + r, k = kt * kBK + kc * 8;
      const bool v = n < N && k < K;
      cp_async16(bs + tile_off(r, kc, kBK), v ? (const void*)(B + (size_t)n * K + k) : (const void*)B, v ? 16u : 0u);
    }
  }
};

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
  RowMajorLoader ld{a, b, M, N, K, bn};
  F32Store ep{C, N};
  switch (bn) {
    case 256: e = umma::launch_umma_gemm<256>(ld, ep, M, N, K, err, st); break;
    case 128: e = umma::launch_umma_gemm<128>(ld, ep, M, N, K, err, st); break;
    case 64: e = umma::launch_umma_gemm<64>(ld, ep, M, N, K, err, st); break;
    default: e = umma::launch_umma_gemm<32>(ld, ep, M, N, K, err, st); break;
  }
  return e == cudaSuccess ? US_OK : US_ERR_CUDA;
}
