// Tile GEMM on the 5th-generation tensor cores:
//   D[m][n] = sum_k A[m][k] * B[n][k]      (BF16 in, FP32 accumulate in TMEM)
//
// Persistent and warp-specialised.  A CTA owns a sequence of tile groups;
// a group is X tiles of 128 x BN that share their B columns (X consecutive
// M tiles).  Roles run concurrently:
//   warps 0-7        producers: stage the operands of each 64-wide K step of
//                    a group into one of the shared-memory stages, up to
//                    `stages` steps ahead of the tensor cores.  Loaders that
//                    gather with cp.async (or plain stores) use all 256
//                    threads (X = 1); loaders that describe their operands
//                    as tensor maps have one thread issue tiled tensor copies
//                    (TMA): X A tiles and one shared B tile per stage;
//   warps 8..8+X-1   one thread each issues the four 128 x BN x 16 MMAs of
//                    its own tile of a stage and commits them to the stage's
//                    "empty" barrier.  A single thread can issue an MMA only
//                    every ~100 cycles, which is slower than the tensor core
//                    finishes a 128 x 64 x 16 step, so narrow tiles need
//                    several issuing warps to keep it busy;
//   last 4 warps     epilogue: read a finished accumulator with tcgen05.ld and
//                    hand it to the Epilogue functor, while the MMAs of the
//                    next group accumulate into the other half of each
//                    issuer's double-buffered TMEM allocation.
// Hand-offs use mbarriers: full[s] (producers -> MMA), empty[s] (the X MMA
// commits -> producers), tfull[w][a] (MMA commit -> epilogue), tempty[w][a]
// (epilogue -> MMA).  Every wait is bounded; a wait that runs out raises a
// shared abort flag that all roles check, so the CTA still drains its
// copies, waits for its MMAs and frees its TMEM.
#pragma once
#include <type_traits>

#include "umma.cuh"

namespace ussim {
namespace umma {

constexpr int kBM = 128, kBK = 64;
constexpr int kProducers = 256;                     // warps 0-7
constexpr int kMmaWarp = kProducers / 32;           // first issuing warp: 8
constexpr int kEpilogue = 128;                      // one epilogue group: 4 warps
constexpr int kEpiGroups = 2;                       // groups after the issuers; group e drains TMEM buffer e
template <int X>
constexpr int gemm_threads() {
  return kProducers + 32 * X + kEpiGroups * kEpilogue;
}
constexpr uint32_t kTileA = kBM * kBK * 2;          // bytes of one A tile of a stage
template <int BN, int X = 1>
constexpr uint32_t stage_bytes() {
  return X * kTileA + (uint32_t)BN * kBK * 2;
}
// stages: as many as fit in ~225 KB of shared memory, at most 8
template <int BN, int X = 1>
constexpr int gemm_stages() {
  constexpr int s = (int)((230400u - 1024u) / stage_bytes<BN, X>());
  return s > 8 ? 8 : s;
}
template <int BN, int X = 1>
constexpr uint32_t gemm_smem_bytes() {   // + slack to align the stages to 1024 B (swizzle atoms)
  return gemm_stages<BN, X>() * stage_bytes<BN, X>() + 1024;
}
template <int BN>
constexpr uint32_t tmem_cols() {   // one accumulator; TMEM allocations are powers of 2 >= 32
  return BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// arrive on `bar` once every cp.async this thread issued so far has landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// loaders that stage a K step with tensor copies declare kTma = true and
// provide issue_a(a_smem, m0, kt, bar) (one 128-row A tile) and
// issue_b(b_smem, n0, kt, bar) (the BN-row B tile)
template <class L, class = void>
struct is_tma_loader : std::false_type {};
template <class L>
struct is_tma_loader<L, std::void_t<decltype(L::kTma)>> : std::integral_constant<bool, L::kTma> {};

// layout of a stage's A tile, declared by the loader as kALayout:
//   0  one 128-byte-swizzled tile, rows of 64 K-elements (default);
//   1  two 64-byte-swizzled sub-tiles of 128 rows x 32 K-elements (8 KB);
//   2  eight unswizzled sub-tiles of 128 rows x 8 K-elements (2 KB),
//      8-row core matrices 128 B apart.
template <class L, class = void>
struct a_layout_of : std::integral_constant<int, 0> {};
template <class L>
struct a_layout_of<L, std::void_t<decltype(L::kALayout)>> : std::integral_constant<int, L::kALayout> {};

//   3  MN-major: two 128-byte-swizzled boxes of 64 K-rows x 64 M-elements
//      (8 KB each, the second M half 8 KB on)
//   4  MN-major: four 64-byte-swizzled boxes of 64 K-rows x 32 M-elements
//      (4 KB each)
// descriptor of the 16-wide K slice k (0..3) of a stage's A tile
template <int LAYOUT>
__device__ __forceinline__ uint64_t a_desc(uint32_t sa, int k) {
  if constexpr (LAYOUT == 1)
    return smem_desc_sw64(sa + (uint32_t)(k >> 1) * 8192u + (uint32_t)(k & 1) * 32u);
  else if constexpr (LAYOUT == 2)
    return smem_desc_kmajor(sa + (uint32_t)k * 4096u, 2048u, 128u);
  else if constexpr (LAYOUT == 3)
    return smem_desc_mn(sa + (uint32_t)k * 2048u, 128u, 8192u);
  else if constexpr (LAYOUT == 4)
    return smem_desc_mn(sa + (uint32_t)k * 1024u, 64u, 4096u);
  else
    return smem_desc_sw128(sa + 32u * (uint32_t)k);
}

// B tile layout, declared by the loader as kBMajorMN: false = K-major
// 128-byte swizzle (default); true = MN-major, BN / min(BN, 64) boxes of
// 64 K-rows x min(BN, 64) N-elements, rows of 2 min(BN, 64) bytes (BN >= 32:
// 128- or 64-byte swizzle)
template <class L, class = void>
struct b_mn_of : std::false_type {};
template <class L>
struct b_mn_of<L, std::void_t<decltype(L::kBMajorMN)>> : std::integral_constant<bool, L::kBMajorMN> {};

template <bool MN, int BN>
__device__ __forceinline__ uint64_t b_desc(uint32_t sb, int k) {
  if constexpr (MN) {
    constexpr uint32_t row = BN >= 64 ? 128u : (uint32_t)BN * 2u;
    return smem_desc_mn(sb + (uint32_t)k * 16u * row, row, 64u * row);
  } else {
    return smem_desc_sw128(sb + 32u * (uint32_t)k);
  }
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              unsigned* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicOr(err, kErrWaitTimeout);
      return false;
    }
  }
  return true;
}

// Loader:   static constexpr bool kAsync (stages with cp.async, else with
//           shared stores); struct State; prepare(State&, m0, n0, tid) once per tile, then
//           load(const State&, a_stage, b_stage, m0, n0, kt, tid) per K step:
//           stage the 128 x 64 A tile rows m0.., and the BN x 64 B tile rows
//           n0.., K step kt (global index), into the K-major 128-byte-swizzled
//           layout (tile_off(r, kc, kBK) for 16-byte chunk kc of row r); steps past
//           the end of K must load zeros.  Called by the kProducers producer threads
//           (X = 1 only).
//           TMA loaders (kTma) instead: issue_a / issue_b, called by one thread,
//           copying exactly X kTileA + BN x 128 bytes per stage into the same
//           layout (zero fill outside the tensor, including tiles past M).
// Epilogue: store(int m, int n0, const float* v16, bool valid).
// Groups: mg x nt x splits, M fastest; group g covers M tiles g*X .. g*X+X-1;
// split z covers K steps z*k_tiles ...
template <int BN, int X, class Loader, class Epilogue>
__global__ void __launch_bounds__(gemm_threads<X>(), 1)
    umma_gemm_kernel(const __grid_constant__ Loader ld, Epilogue ep, int M, int mt, int nt, int n_groups,
                     int k_tiles, unsigned* err) {
  constexpr int S = gemm_stages<BN, X>();
  constexpr uint32_t SB = stage_bytes<BN, X>();
  constexpr uint32_t NCOL = tmem_cols<BN>();
  constexpr bool A_MN = a_layout_of<Loader>::value >= 3, B_MN = b_mn_of<Loader>::value;
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, BN, A_MN, B_MN);
  constexpr bool TMA = is_tma_loader<Loader>::value;
  constexpr int kEpiWarp = kMmaWarp + X;
  static_assert(TMA || X == 1, "gather loaders stage one A tile per stage");
  static_assert(2 * X * NCOL <= 512, "accumulators exceed TMEM");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t full[S], empty[S], tfull[X][2], tempty[X][2], done[X];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mg = (mt + X - 1) / X;

  if (warp == 0) {
    tmem_alloc(&tmem_base, 2 * X * NCOL);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], TMA ? 1 : kProducers);
      mbar_init(&empty[s], X);
    }
    for (int w = 0; w < X; ++w) {
      for (int a = 0; a < 2; ++a) {
        mbar_init(&tfull[w][a], 1);
        mbar_init(&tempty[w][a], kEpilogue);
      }
      mbar_init(&done[w], 1);
    }
    abort_flag = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp < kMmaWarp) {
    // ---------------------------------------------------------- producers
    if constexpr (TMA) {
      if (tid == 0) {
        long long g = 0;
        for (int grp = blockIdx.x; grp < n_groups && !abort_flag; grp += gridDim.x) {
          const int z = grp / (mg * nt), rem = grp - z * mg * nt, ni = rem / mg, gi = rem - ni * mg;
          const int m0 = gi * X * kBM, n0 = ni * BN, kt0 = z * k_tiles;
          bool ok = true;
          for (int t = 0; t < k_tiles; ++t, ++g) {
            const int s = (int)(g % S);
            if (g >= S && !wait_or_abort(&empty[s], (uint32_t)((g / S - 1) & 1), &abort_flag, err)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&full[s], SB);
            const uint32_t sa = smem_u32(smem + s * SB), bar = smem_u32(&full[s]);
#pragma unroll
            for (int w = 0; w < X; ++w) ld.issue_a(sa + w * kTileA, m0 + w * kBM, kt0 + t, bar);
            ld.issue_b(sa + X * kTileA, n0, kt0 + t, bar);
          }
          if (!ok) break;
        }
        // every issued copy must have landed before the CTA may exit (on an
        // abort the MMA threads may not have consumed them)
        for (long long q = g > S ? g - S : 0; q < g; ++q)
          if (!mbar_wait(&full[q % S], (uint32_t)((q / S) & 1))) atomicOr(err, kErrWaitTimeout);
      }
    } else {
      long long g = 0;   // global K-step counter over this CTA's tiles
      for (int grp = blockIdx.x; grp < n_groups && !abort_flag; grp += gridDim.x) {
        const int z = grp / (mg * nt), rem = grp - z * mg * nt, ni = rem / mg, mi = rem - ni * mg;
        const int m0 = mi * kBM, n0 = ni * BN, kt0 = z * k_tiles;
        typename Loader::State st;
        ld.prepare(st, m0, n0, tid);
        bool ok = true;
        for (int t = 0; t < k_tiles; ++t, ++g) {
          const int s = (int)(g % S);
          if (g >= S && !wait_or_abort(&empty[s], (uint32_t)((g / S - 1) & 1), &abort_flag, err)) {
            ok = false;
            break;
          }
          ld.load(st, smem + s * SB, smem + s * SB + kTileA, m0, n0, kt0 + t, tid);
          // cp.async loaders: the barrier completes when the copies land; loaders
          // that store from registers release their stores with a plain arrive
          if (Loader::kAsync)
            cp_async_arrive(&full[s]);
          else
            mbar_arrive(&full[s]);
        }
        if (!ok) break;
      }
      cp_async_wait<0>();
    }
  } else if (warp < kEpiWarp) {
    // ---------------------------------------------------------- MMA issue
    const int w = warp - kMmaWarp;
    if (lane == 0) {
      long long g = 0;
      int j = 0;   // local group index
      for (int grp = blockIdx.x; grp < n_groups && !abort_flag; grp += gridDim.x, ++j) {
        const int a = j & 1;
        if (j >= 2 && !wait_or_abort(&tempty[w][a], (uint32_t)((j / 2 - 1) & 1), &abort_flag, err)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(w * 2 + a) * NCOL;
        bool ok = true;
        for (int t = 0; t < k_tiles; ++t, ++g) {
          const int s = (int)(g % S);
          if (!wait_or_abort(&full[s], (uint32_t)((g / S) & 1), &abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (!TMA) fence_proxy_async();   // stage written through the generic proxy; the MMA reads it async
          const uint32_t sa = smem_u32(smem + s * SB) + (uint32_t)w * kTileA, sb = smem_u32(smem + s * SB) + X * kTileA;
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            mma_bf16(acc, a_desc<a_layout_of<Loader>::value>(sa, k), b_desc<B_MN, BN>(sb, k), IDESC,
                     (t > 0 || k > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[w][a]);
      }
      mma_commit(&done[w]);   // tracks every MMA this thread issued
      if (!mbar_wait(&done[w], 0)) atomicOr(err, kErrWaitTimeout);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;   // TMEM lane quarter this warp may read
    // two groups of four warps: group e takes this CTA's tile groups j with
    // j mod 2 = e, whose accumulators sit in TMEM buffer e
    const int eg = (warp - kEpiWarp) >> 2;
    int j = eg;
    bool ok = true;
    for (int grp = blockIdx.x + eg * (int)gridDim.x; grp < n_groups && ok; grp += kEpiGroups * (int)gridDim.x,
             j += kEpiGroups) {
      const int a = j & 1;
      const int rem = grp % (mg * nt), ni = rem / mg, gi = rem - ni * mg;
      for (int w = 0; w < X; ++w) {
        if (!wait_or_abort(&tfull[w][a], (uint32_t)((j / 2) & 1), &abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int row = (gi * X + w) * kBM + q * 32 + lane;
        const uint32_t acc = tmem + (uint32_t)(w * 2 + a) * NCOL + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
          float v[16];
          tmem_ld16(acc + (uint32_t)c, v);
          ep.store(row, ni * BN + c, v, row < M);
        }
        tc_fence_before();
        mbar_arrive(&tempty[w][a]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * X * NCOL);
}

// splits > 1: split K into `splits` contiguous ranges; the epilogue then
// receives partial sums and must reduce them itself.  X = number of
// issuing warps (tiles per group); X > 1 needs a TMA loader.
template <int BN, int X = 1, class Loader, class Epilogue>
cudaError_t launch_umma_gemm(const Loader& ld, const Epilogue& ep, int M, int N, int K, unsigned* err,
                             cudaStream_t st, int splits = 1) {
  auto kern = umma_gemm_kernel<BN, X, Loader, Epilogue>;
  constexpr uint32_t smem = gemm_smem_bytes<BN, X>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int k_total = (K + kBK - 1) / kBK;
  splits = splits < 1 ? 1 : (splits > k_total ? k_total : splits);
  const int k_tiles = (k_total + splits - 1) / splits;
  splits = (k_total + k_tiles - 1) / k_tiles;
  const int mt = (M + kBM - 1) / kBM, nt = N / BN, mg = (mt + X - 1) / X;
  const long long n_groups = (long long)mg * nt * splits;
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, gemm_threads<X>(), smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long grid = n_groups < (long long)sms * per_sm ? n_groups : (long long)sms * per_sm;
  kern<<<(unsigned)grid, gemm_threads<X>(), smem, st>>>(ld, ep, M, mt, nt, (int)n_groups, k_tiles, err);
  return cudaGetLastError();
}

}  // namespace umma
}  // namespace ussim
