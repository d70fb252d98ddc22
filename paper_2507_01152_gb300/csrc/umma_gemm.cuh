// Tile GEMM on the 5th-generation tensor cores:
//   D[m][n] = sum_k A[m][k] * B[n][k]      (BF16 in, FP32 accumulate in TMEM)
// One CTA of 128 threads computes a 128 x BN tile.  K advances in 64-wide
// steps through two shared-memory stages: while the tensor core works on
// stage s (four 128 x BN x 16 MMAs issued by one thread and committed to
// the stage's mbarrier), all threads stage the next K step into the other
// stage with cp.async.  Operands are gathered by a Loader functor, so the
// same kernel serves plain GEMMs and implicit-GEMM convolutions; the
// accumulator is read back with tcgen05.ld and handed to an Epilogue
// functor row by row (thread i of warp w owns tile row 32 w + i).
#pragma once
#include "umma.cuh"

namespace ussim {
namespace umma {

constexpr int kBM = 128, kBK = 64;
constexpr int kThreads = 128;
constexpr uint32_t kTileA = kBM * kBK * 2;          // bytes of one A stage
constexpr uint32_t kSbo = kBK * 16;                 // 8-row group stride in a stage
constexpr uint32_t kLbo = 128;                      // K-adjacent core matrices

template <int BN>
constexpr uint32_t stage_bytes() {
  return kTileA + (uint32_t)BN * kBK * 2;
}
template <int BN>
constexpr uint32_t gemm_smem_bytes() {
  return 2 * stage_bytes<BN>();
}
template <int BN>
constexpr uint32_t tmem_cols() {
  return BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));   // TMEM allocations: powers of 2, >= 32
}

// Loader:   void load(uint8_t* a_stage, uint8_t* b_stage, int m0, int n0, int kt, int tid)
//           stages the 128 x 64 A tile rows m0.., and the BN x 64 B tile rows
//           n0.., K step kt, into the K-major no-swizzle layout (use
//           tile_off(r, kc, kBK) for 16-byte chunk kc of row r), with cp.async
//           or plain shared stores; steps past the end of K must load zeros.
//           With split K (grid.z > 1), CTA z covers steps z*k_tiles .. +k_tiles.
// Epilogue: void store(int m, int n0, const float* v16, bool valid)
template <int BN, class Loader, class Epilogue>
__global__ void __launch_bounds__(kThreads) umma_gemm_kernel(Loader ld, Epilogue ep, int M, int k_tiles,
                                                              unsigned* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t NCOL = tmem_cols<BN>();
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, BN);
  uint8_t* stage[2] = {smem, smem + stage_bytes<BN>()};

  if (warp == 0) {
    tmem_alloc(&tmem_base, NCOL);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kt0 = blockIdx.z * k_tiles;

  ld.load(stage[0], stage[0] + kTileA, m0, n0, kt0, tid);
  cp_async_commit();
  bool ok = true;
  int t = 0;
  for (; t < k_tiles; ++t) {
    const int s = t & 1;
    if (t + 1 < k_tiles) {
      // the other stage was read by the MMAs of step t-1: wait for their commit
      if (t >= 1) ok = ok && mbar_wait(&bar[s ^ 1], ((t - 1) >> 1) & 1);
      if (ok) ld.load(stage[s ^ 1], stage[s ^ 1] + kTileA, m0, n0, kt0 + t + 1, tid);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    fence_proxy_async();
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a = smem_u32(stage[s]), b = smem_u32(stage[s] + kTileA);
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j)
        mma_bf16(tmem, smem_desc_kmajor(a + 256 * j, kLbo, kSbo), smem_desc_kmajor(b + 256 * j, kLbo, kSbo), IDESC,
                 (t > 0 || j > 0) ? 1u : 0u);
      mma_commit(&bar[s]);
    }
  }
  cp_async_wait<0>();
  const int last = (ok ? k_tiles : t) - 1;
  bool fin = last < 0 || mbar_wait(&bar[last & 1], (last >> 1) & 1);
  fin = __syncthreads_and(fin && ok);
  tc_fence_after();
  if (fin) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      ep.store(row, n0 + c, v, row < M);
    }
  } else if (tid == 0) {
    atomicOr(err, kErrWaitTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOL);
}

// splits > 1: split K into `splits` contiguous ranges (grid.z); the
// epilogue then receives partial sums and must reduce them itself
template <int BN, class Loader, class Epilogue>
cudaError_t launch_umma_gemm(const Loader& ld, const Epilogue& ep, int M, int N, int K, unsigned* err,
                             cudaStream_t st, int splits = 1) {
  auto kern = umma_gemm_kernel<BN, Loader, Epilogue>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes<BN>());
  if (e != cudaSuccess) return e;
  const int k_total = (K + kBK - 1) / kBK;
  splits = splits < 1 ? 1 : (splits > k_total ? k_total : splits);
  const int k_tiles = (k_total + splits - 1) / splits;
  splits = (k_total + k_tiles - 1) / k_tiles;
  const dim3 grid((M + kBM - 1) / kBM, N / BN, splits);
  kern<<<grid, kThreads, gemm_smem_bytes<BN>(), st>>>(ld, ep, M, k_tiles, err);
  return cudaGetLastError();
}

}  // namespace umma
}  // namespace ussim
