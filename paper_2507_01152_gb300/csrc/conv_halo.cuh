// Stride-1 3x3 convolution forward for the surrogate's narrow layers, with
// each tile's input staged once as a haloed box:
//
//   y[b,y,x,co] = act(bias[co] + sum_(ky,kx,ci) x[b, y+ky-1, x+kx-1, ci] w[co][ky][kx][ci])
//
// An output tile is 16 rows x 8 columns of one image (the 128 rows M of a
// tcgen05 MMA).  Its input box, 18 x 10 pixels with the one-pixel halo, is
// copied by tensor copies (TMA) once, as CIN / 8 planes of 16-byte pixels
// (the copies' zero fill is the padding); the nine taps are then nine
// shifted windows of that box, read by the MMAs through unswizzled K-major
// descriptors: 8-row core matrices are the 8 pixels of one box row
// (16 bytes apart), consecutive output rows one box row (160 bytes) apart,
// channel planes one plane (2944 bytes, 128-byte aligned) apart.  The
// tap-by-tap forms stage the box nine times over; this one moves it once,
// so the narrow layers (32 or 64 output channels on the full- and
// half-resolution grids) are no longer bound by the L2 -> shared-memory
// traffic of the re-reads.
//
// The weights [9 taps][CIN / 8 planes][COUT rows][16 B] stay resident in
// shared memory for the whole persistent CTA.  Roles: warp 0 (one thread)
// issues the box copies of up to S tiles ahead; X issuing warps each own
// every X-th tile of the CTA (one elected thread issues its 9 CIN / 16 MMAs
// of 128 x COUT x 16 into one half of its double-buffered TMEM
// accumulator); four groups of four epilogue warps, tile g to group g mod 4,
// add the bias, apply the ReLU and store BF16 pixels.  Every wait is bounded; a wait that runs out raises the
// shared abort flag, the CTA drains its copies and MMAs, frees its TMEM and
// reports kErrWaitTimeout.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "umma_gemm.cuh"

namespace ussim {
namespace umma {

template <int CIN, int COUT>
struct HaloCfg {
  static constexpr int TY = 16, TX = 8;                        // output tile: 16 rows x 8 columns
  static constexpr int BY = TY + 2, BX = TX + 2;               // staged box with the halo
  static constexpr int NCH = CIN / 8;                          // 16-byte channel planes
  // 8 input channels: one MMA of K = 16 takes two taps of 8 channels (the
  // tap pair's pixel offset is the descriptor's K stride); a tenth, zero
  // tap completes the last pair
  static constexpr bool PAIRED = CIN == 8;
  static constexpr int NTAPW = PAIRED ? 10 : 9;                // taps in the weight layout
  static constexpr uint32_t BOX = (uint32_t)BY * BX * 16;      // bytes of one plane's copy: 2880
  static constexpr uint32_t PLANE = (BOX + 127u) / 128u * 128u;   // plane stride, 128-byte aligned copies
  static constexpr uint32_t STAGE = NCH * PLANE;
  static constexpr uint32_t WBYTES = (uint32_t)NTAPW * NCH * COUT * 16;
  static constexpr int X = COUT <= 32 ? 8 : 4;                 // issuing warps: 2 X COUT TMEM columns = 512
  // stages: a multiple of X, so that stage s always serves issuer s mod X
  // and each issuer sees every phase of its stages' barriers in order
  static constexpr int S0 = (int)((225u * 1024u - WBYTES) / STAGE);
  static constexpr int S = (S0 > 8 ? 8 : S0) / X * X;
  // epilogue groups of 4 warps; group g mod kEpiGroups takes tile g.  With
  // kEpiGroups dividing X, every tile of one issuer goes to one group, which
  // therefore sees each of that issuer's accumulator phases in order
  static constexpr int kEpiGroups = 4;
  static constexpr int THREADS = 32 * (1 + X + 4 * kEpiGroups);
  static constexpr uint32_t SMEM = WBYTES + S * STAGE + 4 * COUT + 128;   // + bias, alignment slack
  static_assert((CIN == 8 || CIN % 16 == 0) && (COUT == 32 || COUT == 64), "halo conv shapes");
  static_assert(S >= X, "stages do not fit");
  static_assert(2 * X * COUT <= 512, "accumulators exceed TMEM");
  static_assert(X % kEpiGroups == 0, "an issuer's tiles must all go to one epilogue group");
};

struct HaloArgs {
  const __nv_bfloat16* w;   // [COUT][3][3][CIN]
  const float* bias;        // [COUT]
  __nv_bfloat16* y;         // output view: pixel p at y + p * y_cs + y_co (null: not stored)
  int y_cs, y_co, relu;
  int B, H, W, tiles_y, tiles_x, n_tiles;
  // optional fused 1 x 1 head (COUT = 32): head_out[p] = sigmoid(head_b[0] +
  // sum_c y[p][c] head_w[c]) over the BF16 outputs; each group of 8
  // channels summed in channel order, then head_b and the group sums in
  // group order
  const float* head_w = nullptr;
  const float* head_b = nullptr;
  float* head_out = nullptr;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(HaloCfg<CIN, COUT>::THREADS, 1)
    conv3x3_halo_kernel(const __grid_constant__ CUtensorMap tx, const HaloArgs a, unsigned* err) {
  using C = HaloCfg<CIN, COUT>;
  constexpr int X = C::X, S = C::S, NCH = C::NCH;
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, COUT);
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint8_t* wsm = smem;                          // resident weights
  uint8_t* box = smem + C::WBYTES;              // S staged boxes
  __shared__ uint64_t full[S], empty[S], tfull[X][2], tempty[X][2], done[X];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int w = 0; w < X; ++w) {
      for (int q = 0; q < 2; ++q) {
        mbar_init(&tfull[w][q], 1);
        mbar_init(&tempty[w][q], 128);   // the four warps of the epilogue group that takes the tile
      }
      mbar_init(&done[w], 1);
    }
    abort_flag = 0;
    mbar_init_fence();
  }
  // weights: w[co][tap][ci] -> plane-major [tap][ci / 8][co][16 B] (the
  // paired layout's tenth tap zero)
  for (int i = tid; i < C::NTAPW * NCH * COUT; i += blockDim.x) {
    const int co = i % COUT, r = i / COUT, ch = r % NCH, tap = r / NCH;
    const uint4 v = tap < 9 ? __ldg(reinterpret_cast<const uint4*>(a.w + ((size_t)co * 9 + tap) * CIN + ch * 8))
                            : make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(wsm + ((size_t)(tap * NCH + ch) * COUT + co) * 16) = v;
  }
  // the pad after each plane's copy reads as zero (the paired layout's last
  // pair reaches one pixel into it, against zero weights)
  constexpr int PADV = (int)(C::PLANE - C::BOX) / 16;
  for (int i = tid; i < S * NCH * PADV; i += blockDim.x) {
    const int pl = i / PADV, k = i - pl * PADV;
    *reinterpret_cast<uint4*>(box + (size_t)pl * C::PLANE + C::BOX + (size_t)k * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_proxy_async();   // generic-proxy stores, read by the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int n_local = a.n_tiles > (int)blockIdx.x ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto tile_of = [&](int g, int& b, int& y0, int& x0) {
    const int t = (int)blockIdx.x + g * (int)gridDim.x;
    const int per = a.tiles_y * a.tiles_x;
    b = t / per;
    const int r = t - b * per, ty = r / a.tiles_x;
    y0 = ty * C::TY;
    x0 = (r - ty * a.tiles_x) * C::TX;
  };

  if (warp == 0) {
    // ----------------------------------------------------------- producer
    if (lane == 0) {
      int g = 0;
      for (; g < n_local && !abort_flag; ++g) {
        const int s = g % S;
        if (g >= S && !wait_or_abort(&empty[s], (uint32_t)((g / S - 1) & 1), &abort_flag, err)) break;
        int b, y0, x0;
        tile_of(g, b, y0, x0);
        mbar_arrive_expect_tx(&full[s], NCH * C::BOX);
        const uint32_t dst = smem_u32(box + (size_t)s * C::STAGE), bar = smem_u32(&full[s]);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) tma_load_4d(dst + ch * C::PLANE, &tx, ch * 8, x0 - 1, y0 - 1, b, bar);
      }
      // every issued copy must land before the CTA may exit
      for (int q = g > S ? g - S : 0; q < g; ++q)
        if (!mbar_wait(&full[q % S], (uint32_t)((q / S) & 1))) atomicOr(err, kErrWaitTimeout);
    }
    __syncwarp();
  } else if (warp <= X) {
    // ---------------------------------------------------------- MMA issue
    const int w = warp - 1;
    if (lane == 0) {
      const uint32_t wbase = smem_u32(wsm);
      for (int g = w, j = 0; g < n_local && !abort_flag; g += X, ++j) {
        const int s = g % S, q = j & 1;
        if (j >= 2 && !wait_or_abort(&tempty[w][q], (uint32_t)((j / 2 - 1) & 1), &abort_flag, err)) break;
        if (!wait_or_abort(&full[s], (uint32_t)((g / S) & 1), &abort_flag, err)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(w * 2 + q) * COUT;
        const uint32_t sbox = smem_u32(box + (size_t)s * C::STAGE);
        if constexpr (C::PAIRED) {
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            const int t0 = 2 * j, t1 = 2 * j + 1;
            const int o0 = (t0 / 3) * C::BX + t0 % 3, o1 = t1 < 9 ? (t1 / 3) * C::BX + t1 % 3 : o0 + 1;
            const uint64_t ad = smem_desc_kmajor(sbox + (uint32_t)o0 * 16u, (uint32_t)(o1 - o0) * 16u,
                                                 (uint32_t)C::BX * 16u);
            const uint64_t bd = smem_desc_kmajor(wbase + (uint32_t)(t0 * COUT) * 16u, (uint32_t)COUT * 16u, 128u);
            mma_bf16(acc, ad, bd, IDESC, j > 0 ? 1u : 0u);
          }
        }
#pragma unroll
        for (int tap = 0; tap < (C::PAIRED ? 0 : 9); ++tap) {
          const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
          for (int kk = 0; kk < NCH / 2; ++kk) {
            const uint64_t ad = smem_desc_kmajor(sbox + (uint32_t)(2 * kk) * C::PLANE + (uint32_t)(ky * C::BX + kx) * 16u,
                                                 C::PLANE, (uint32_t)C::BX * 16u);
            const uint64_t bd = smem_desc_kmajor(wbase + (uint32_t)((tap * NCH + 2 * kk) * COUT) * 16u,
                                                 (uint32_t)COUT * 16u, 128u);
            mma_bf16(acc, ad, bd, IDESC, (tap > 0 || kk > 0) ? 1u : 0u);
          }
        }
        mma_commit(&empty[s]);
        mma_commit(&tfull[w][q]);
      }
      mma_commit(&done[w]);
      if (!mbar_wait(&done[w], 0)) atomicOr(err, kErrWaitTimeout);
    }
    __syncwarp();
  } else {
    // ----------------------------------------------------------- epilogue
    // groups of four warps take tiles g with g mod kEpiGroups = group; within a group, warp
    // (index mod 4) reads its TMEM lane quarter, all of a tile's columns in
    // flight before one wait
    const int grp = (warp - 1 - X) >> 2;
    const int qd = warp & 3;               // TMEM lane quarter this warp may read
    const int m = qd * 32 + lane;          // tile row: pixel (m / 8, m % 8)
    // the bias, staged once in shared memory (after the boxes) by the
    // epilogue warps and read as broadcasts; named barrier 1 joins only them
    float* sbias = reinterpret_cast<float*>(box + (size_t)S * C::STAGE);
    for (int i = (warp - 1 - X) * 32 + lane; i < COUT; i += 32 * 4 * C::kEpiGroups) sbias[i] = __ldg(&a.bias[i]);
    asm volatile("bar.sync 1, %0;" ::"r"(32 * 4 * C::kEpiGroups));
    for (int g = grp; g < n_local; g += C::kEpiGroups) {
      const int w = g % X, j = g / X, q = j & 1;
      if (!wait_or_abort(&tfull[w][q], (uint32_t)((j / 2) & 1), &abort_flag, err)) break;
      tc_fence_after();
      int b, y0, x0;
      tile_of(g, b, y0, x0);
      const int yy = y0 + (m >> 3), xx = x0 + (m & 7);
      const bool valid = yy < a.H && xx < a.W;
      const size_t pix = (size_t)((size_t)b * a.H + yy) * a.W + xx;
      __nv_bfloat16* dst = a.y ? a.y + pix * a.y_cs + a.y_co : nullptr;
      float zg[COUT / 8];   // the fused head's group sums
      const uint32_t acc = tmem + (uint32_t)(w * 2 + q) * COUT + ((uint32_t)(qd * 32) << 16);
      // 32 columns in flight per wait
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 32) {
        uint32_t r[32];
        tmem_ld16_nowait(acc + (uint32_t)c0, r);
        tmem_ld16_nowait(acc + (uint32_t)c0 + 16u, r + 16);
        tmem_wait_ld();
        if (c0 + 32 >= COUT) {
          tc_fence_before();
          mbar_arrive(&tempty[w][q]);      // the accumulator is free once it is in registers
        }
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
          __align__(16) __nv_bfloat16 o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float t = __uint_as_float(r[c + i]) + sbias[c0 + c + i];
            o[i] = __float2bfloat16_rn(a.relu ? fmaxf(t, 0.f) : t);
          }
          if (valid && dst) *reinterpret_cast<uint4*>(dst + c0 + c) = *reinterpret_cast<const uint4*>(o);
          if constexpr (COUT == 32) {
            if (a.head_out) {
              float t = 0.f;
#pragma unroll
              for (int i = 0; i < 8; ++i) t = fmaf(__bfloat162float(o[i]), __ldg(&a.head_w[c + i]), t);
              zg[c >> 3] = t;
            }
          }
        }
      }
      if constexpr (COUT == 32) {
        if (a.head_out && valid) {
          float z = __ldg(a.head_b);
#pragma unroll
          for (int k = 0; k < COUT / 8; ++k) z += zg[k];
          a.head_out[pix] = 1.f / (1.f + expf(-z));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// The same haloed-box forward for inputs too wide for resident weights
// (CIN a multiple of 64; COUT = 64, 128 or 256).  A CTA takes its tiles in
// pairs (local tiles 2p and 2p + 1; a missing second tile of the last pair
// reads zeros and stores nothing), and the pair's two MMA issuers share
// every weight chunk.  The weights stream through a ring of R chunks, each
// the COUT x 64 block of one tap and one 64-channel block of the input,
// copied by a 2-D tensor copy with the 128-byte swizzle (no repacking: a
// chunk is a box of the [COUT][3][3][CIN] array) and read through swizzled
// K-major descriptors; a slot is free again once both issuers' MMAs on it
// are done.  Each tile's box is staged in its 64-channel blocks through two
// block slots per issuer (block k of pair p is use u = p NKC + k, in slot
// u mod 2), and the chunks run block-major (the 9 taps of block 0, then of
// block 1, ...), so a block loads while the issuer works on the one before.
// Roles: warp 0 (one thread) copies the box blocks, warp 1 (one thread) the
// weight chunks, warps 2 and 3 (one thread each) issue the 4 MMAs of
// 128 x COUT x 16 of each chunk for tile 2p and tile 2p + 1 into their TMEM
// accumulators (double-buffered while 2 x 2 x COUT columns fit in TMEM,
// else single); epilogue group t (four warps) drains issuer t's accumulator
// of every pair, adds the bias, applies the ReLU and stores BF16 pixels.
// Every wait is bounded, with the abort protocol of the kernel above.
template <int CIN, int COUT>
struct HaloStreamCfg {
  static constexpr int TY = 16, TX = 8;
  static constexpr int BY = TY + 2, BX = TX + 2;
  static constexpr int NKC = CIN / 64;                             // 64-channel blocks
  static constexpr int HPL = 8;                                    // 16-byte channel planes per block
  static constexpr uint32_t BOX = (uint32_t)BY * BX * 16;          // bytes of one plane's copy
  static constexpr uint32_t PLANE = (BOX + 127u) / 128u * 128u;
  static constexpr uint32_t HSTAGE = HPL * PLANE;                  // one block of one box
  static constexpr int X = 2;                                      // issuers: tiles of a pair
  static constexpr int NB = NKC < 2 ? NKC : 2;                     // block slots per issuer
  static constexpr int NCHUNK = 9 * NKC;                           // weight chunks per pair
  static constexpr uint32_t WCH = (uint32_t)COUT * 128;            // bytes of one chunk
  static constexpr uint32_t BOXES = (uint32_t)X * NB * HSTAGE;
  static constexpr int R0 = (int)((226u * 1024u - 1024u - 4u * COUT - BOXES) / WCH);
  static constexpr int R = R0 > 8 ? 8 : R0;                        // weight ring slots
  static constexpr uint32_t WRING = R * WCH;
  static constexpr int kEpiGroups = X;                             // group t drains issuer t
  static constexpr int kEpiWarp = 2 + X;
  static constexpr int THREADS = 32 * (kEpiWarp + 4 * kEpiGroups);
  static constexpr int NBUF = 2 * X * COUT <= 512 ? 2 : 1;         // accumulators per issuer
  static constexpr uint32_t NCOLS = (uint32_t)NBUF * X * COUT;
  static constexpr uint32_t SMEM = WRING + BOXES + 4 * COUT + 1024;   // + bias, 1024-byte alignment slack
  static_assert(CIN % 64 == 0 && (COUT == 64 || COUT == 128 || COUT == 256), "streamed halo conv shapes");
  static_assert(R >= 4, "weight ring too shallow");
  static_assert(NCOLS <= 512, "accumulators exceed TMEM");
  static_assert(SMEM <= 226u * 1024u, "shared memory");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(HaloStreamCfg<CIN, COUT>::THREADS, 1)
    conv3x3_halo_stream_kernel(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw,
                               const HaloArgs a, unsigned* err) {
  using C = HaloStreamCfg<CIN, COUT>;
  constexpr int R = C::R, NKC = C::NKC, NB = C::NB, HPL = C::HPL, NCHUNK = C::NCHUNK, X = C::X, NBUF = C::NBUF;
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, COUT);
  extern __shared__ __align__(1024) uint8_t smem_stream[];
  uint8_t* smem = smem_stream + ((1024u - (smem_u32(smem_stream) & 1023u)) & 1023u);
  uint8_t* wring = smem;                         // R weight chunks (1024-byte aligned swizzle atoms)
  uint8_t* box = smem + C::WRING;                // block slot j of issuer t at (t NB + j) HSTAGE
  float* sbias = reinterpret_cast<float*>(box + C::BOXES);
  __shared__ uint64_t hfull[X][NB], hempty[X][NB], wfull[R], wempty[R], tfull[X][NBUF], tempty[X][NBUF], done[X];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(&tmem_base, C::NCOLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int t = 0; t < X; ++t) {
      for (int j = 0; j < NB; ++j) {
        mbar_init(&hfull[t][j], 1);
        mbar_init(&hempty[t][j], 1);
      }
      for (int q = 0; q < NBUF; ++q) {
        mbar_init(&tfull[t][q], 1);
        mbar_init(&tempty[t][q], 128);   // the four warps of epilogue group t
      }
      mbar_init(&done[t], 1);
    }
    for (int r = 0; r < R; ++r) {
      mbar_init(&wfull[r], 1);
      mbar_init(&wempty[r], X);          // both issuers release a chunk
    }
    abort_flag = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int n_local = a.n_tiles > (int)blockIdx.x ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int n_pairs = (n_local + 1) / 2;
  // tile g of this CTA; g = n_local (the missing second tile of a last
  // pair) lies past the batch, where the box copies read zeros
  auto tile_of = [&](int g, int& b, int& y0, int& x0) {
    const int t = (int)blockIdx.x + g * (int)gridDim.x;
    const int per = a.tiles_y * a.tiles_x;
    b = t / per;
    const int r = t - b * per, ty = r / a.tiles_x;
    y0 = ty * C::TY;
    x0 = (r - ty * a.tiles_x) * C::TX;
  };

  if (warp == 0) {
    // -------------------------------------------------------- box blocks
    if (lane == 0) {
      int fills[X][NB] = {};   // copies issued into each slot
      bool ok = true;
      for (int p = 0; p < n_pairs && ok && !abort_flag; ++p) {
        for (int k = 0; k < NKC && ok; ++k) {
          const int u = p * NKC + k, j = u % NB, n = u / NB;   // n: this slot's fill index
          for (int t = 0; t < X; ++t) {
            if (n >= 1 && !wait_or_abort(&hempty[t][j], (uint32_t)((n - 1) & 1), &abort_flag, err)) {
              ok = false;
              break;
            }
            int b, y0, x0;
            tile_of(2 * p + t, b, y0, x0);
            mbar_arrive_expect_tx(&hfull[t][j], HPL * C::BOX);
            const uint32_t dst = smem_u32(box + (size_t)(t * NB + j) * C::HSTAGE), bar = smem_u32(&hfull[t][j]);
#pragma unroll
            for (int pl = 0; pl < HPL; ++pl)
              tma_load_4d(dst + pl * C::PLANE, &tx, (k * HPL + pl) * 8, x0 - 1, y0 - 1, b, bar);
            ++fills[t][j];
          }
        }
      }
      // every issued copy must land before the CTA may exit: the last fill of each slot
#pragma unroll
      for (int t = 0; t < X; ++t)
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (fills[t][j] > 0 && !mbar_wait(&hfull[t][j], (uint32_t)((fills[t][j] - 1) & 1)))
            atomicOr(err, kErrWaitTimeout);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------- weight chunks
    if (lane == 0) {
      const int nq = n_pairs * NCHUNK;
      int q = 0;
      for (; q < nq && !abort_flag; ++q) {
        const int r = q % R;
        if (q >= R && !wait_or_abort(&wempty[r], (uint32_t)((q / R - 1) & 1), &abort_flag, err)) break;
        const int c = q % NCHUNK, k = c / 9, tap = c - 9 * k;
        mbar_arrive_expect_tx(&wfull[r], C::WCH);
        tma_load_2d(smem_u32(wring + (size_t)r * C::WCH), &tw, tap * CIN + k * 64, 0, smem_u32(&wfull[r]));
      }
      for (int p = q > R ? q - R : 0; p < q; ++p)
        if (!mbar_wait(&wfull[p % R], (uint32_t)((p / R) & 1))) atomicOr(err, kErrWaitTimeout);
    }
    __syncwarp();
  } else if (warp < C::kEpiWarp) {
    // ------------------------------------------------------- MMA issue
    // issuer t takes tile 2p + t of every pair.  The chunk loop is
    // unrolled: every A descriptor is the block slot's base descriptor plus
    // a constant offset (in 16-byte units, added to the low word: addresses
    // stay below 256 KB, so the address field cannot carry), every B
    // descriptor the ring slot's plus 2 per K step of 16.
    const int t = warp - 2;
    if (lane == 0) {
      const uint64_t bdesc0 = smem_desc_sw128(smem_u32(wring));
      const uint32_t b_hi = (uint32_t)(bdesc0 >> 32);
      for (int p = 0; p < n_pairs && !abort_flag; ++p) {
        const int buf = p % NBUF, jp = p / NBUF;   // accumulator, and its use index
        if (p >= NBUF && !wait_or_abort(&tempty[t][buf], (uint32_t)((jp - 1) & 1), &abort_flag, err)) break;
        const uint32_t acc = tmem + (uint32_t)(t * NBUF + buf) * COUT;
        const unsigned q0 = (unsigned)p * NCHUNK;   // ring position of the pair's first chunk
        bool ok = true;
#pragma unroll
        for (int k = 0; k < NKC && ok; ++k) {
          const unsigned u = (unsigned)p * NKC + (unsigned)k, j = u % NB;
          if (!wait_or_abort(&hfull[t][j], (u / NB) & 1u, &abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t adesc0 = smem_desc_kmajor(smem_u32(box + (size_t)(t * NB + j) * C::HSTAGE), C::PLANE,
                                                   (uint32_t)C::BX * 16u);
          const uint32_t a_lo = (uint32_t)adesc0, a_hi = (uint32_t)(adesc0 >> 32);
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int c = k * 9 + tap, ky = tap / 3, kx = tap - 3 * ky;
            const unsigned q = q0 + (unsigned)c, r = q % R;
            if (!wait_or_abort(&wfull[r], (q / R) & 1u, &abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t b_lo = (uint32_t)bdesc0 + r * (C::WCH >> 4);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const uint32_t aoff = ((uint32_t)(2 * jj) * C::PLANE + (uint32_t)(ky * C::BX + kx) * 16u) >> 4;
              const uint64_t ad = ((uint64_t)a_hi << 32) | (uint64_t)(a_lo + aoff);
              const uint64_t bd = ((uint64_t)b_hi << 32) | (uint64_t)(b_lo + 2u * (uint32_t)jj);
              mma_bf16(acc, ad, bd, IDESC, (c > 0 || jj > 0) ? 1u : 0u);
            }
            mma_commit(&wempty[r]);
          }
          if (!ok) break;
          mma_commit(&hempty[t][j]);
        }
        if (!ok) break;
        mma_commit(&tfull[t][buf]);
      }
      mma_commit(&done[t]);   // tracks every MMA this thread issued
      if (!mbar_wait(&done[t], 0)) atomicOr(err, kErrWaitTimeout);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------- epilogue
    // group e drains issuer e's accumulator of every pair (tile 2p + e),
    // so it sees each accumulator's phases in order; warp (index mod 4)
    // reads its TMEM lane quarter
    const int e = (warp - C::kEpiWarp) >> 2;
    const int qd = warp & 3;
    const int m = qd * 32 + lane;          // tile row: pixel (m / 8, m % 8)
    for (int i = (warp - C::kEpiWarp) * 32 + lane; i < COUT; i += 32 * 4 * C::kEpiGroups) sbias[i] = __ldg(&a.bias[i]);
    asm volatile("bar.sync 1, %0;" ::"r"(32 * 4 * C::kEpiGroups));
    bool ok = true;
    for (int p = 0; p < n_pairs && ok; ++p) {
      const int buf = p % NBUF, jp = p / NBUF;
      if (!wait_or_abort(&tfull[e][buf], (uint32_t)(jp & 1), &abort_flag, err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int g = 2 * p + e;
      int b, y0, x0;
      tile_of(g, b, y0, x0);
      const int yy = y0 + (m >> 3), xx = x0 + (m & 7);
      const bool valid = g < n_local && yy < a.H && xx < a.W;
      const size_t pix = valid ? (size_t)((size_t)b * a.H + yy) * a.W + xx : 0;
      __nv_bfloat16* dst = a.y ? a.y + pix * a.y_cs + a.y_co : nullptr;
      const uint32_t acc = tmem + (uint32_t)(e * NBUF + buf) * COUT + ((uint32_t)(qd * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 32) {
        uint32_t rr[32];
        tmem_ld16_nowait(acc + (uint32_t)c0, rr);
        tmem_ld16_nowait(acc + (uint32_t)c0 + 16u, rr + 16);
        tmem_wait_ld();
        if (c0 + 32 >= COUT) {
          tc_fence_before();
          mbar_arrive(&tempty[e][buf]);    // the accumulator is free once it is in registers
        }
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
          __align__(16) __nv_bfloat16 o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float v = __uint_as_float(rr[c + i]) + sbias[c0 + c + i];
            o[i] = __float2bfloat16_rn(a.relu ? fmaxf(v, 0.f) : v);
          }
          if (valid && dst) *reinterpret_cast<uint4*>(dst + c0 + c) = *reinterpret_cast<const uint4*>(o);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, C::NCOLS);
}

}  // namespace umma
}  // namespace ussim
