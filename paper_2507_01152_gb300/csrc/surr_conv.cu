// Convolution operators of the surrogate on the tcgen05 tile GEMM.
//
//  conv3x3 forward   D[(b,yo,xo)][co]     = sum_(ky,kx,ci) X[b, yo*s-1+ky, xo*s-1+kx, ci] W[co][ky][kx][ci]
//  conv3x3 dgrad     dX[(b,yi,xi)][ci]    = sum_(ky,kx,co) dY[b, (yi+1-ky)/s, (xi+1-kx)/s, co] W[co][ky][kx][ci]
//                                          (terms whose (yi+1-ky)/s is not an integer drop out)
//  conv3x3 wgrad     dW^T[(ky,kx,ci)][co] = sum_(b,yo,xo) X[b, yo*s-1+ky, xo*s-1+kx, ci] dY[b,yo,xo,co]
//  convT2x2 forward  D[(b,y,x)][(d,co)]   = sum_ci X[b,y,x,ci] W4[(d,co)][ci], scattered to (2y+dy, 2x+dx)
//  convT2x2 dgrad    dX[(b,y,x)][ci]      = sum_(d,co) dY[b, 2y+dy, 2x+dx, co] W4[(d,co)][ci]
//  convT2x2 wgrad    dW4[(d,co)][ci]      = sum_(b,y,x) dY[b, 2y+dy, 2x+dx, co] X[b,y,x,ci]
//
// Activations are NHWC BF16 views (pointer, channel stride, channel offset),
// so a layer reads or writes a channel slice of a concatenated tensor in
// place.  Epilogues fuse bias + ReLU + BF16 conversion (forward), the ReLU
// mask of the layer input (+ optional accumulation into an existing
// gradient, for tensors that feed two layers) (dgrad), and FP32 atomic
// reduction of split-K partial sums (wgrad).
#include <cuda_bf16.h>

#include "conv_halo.cuh"
#include "surr_internal.h"
#include "ussim_surrogate.h"
#include "umma_tma.cuh"

namespace ussim {
namespace surr {

using namespace umma;
using bf16 = __nv_bfloat16;

struct View {
  const bf16* p;
  int cs, co;   // channel stride (elements per pixel) and channel offset
};
struct OutView {
  bf16* p;
  int cs, co;
};

// rows of an implicit GEMM walk the pixels of a B x H x W grid
struct Grid {
  int B, H, W;
  __device__ __forceinline__ void pix(int m, int& b, int& y, int& x) const {
    const int hw = H * W;
    b = m / hw;
    const int r = m - b * hw;
    y = r / W;
    x = r - y * W;
  }
};

// each producer thread stages a fixed 16-byte column chunk kc of kRows rows
// per A tile (rows r0 + kRowStep i), so per-row pixel coordinates are
// computed once per tile
constexpr int kRows = kBM * 8 / kProducers;        // 4
constexpr int kRowStep = kBM / kRows;               // 32
__device__ __forceinline__ void a_chunk(int tid, int& kc, int& r0) {
  kc = (tid >> 3) & 7;
  r0 = (tid & 7) + ((tid >> 6) << 3);
}

// ------------------------------------------------------------ forward conv
struct ConvFwdLoader {
  static constexpr bool kAsync = true;
  View x;
  const bf16* w;   // [N][K]
  Grid in, out;
  int Cin, K, N, stride, M, bn;
  struct State {
    int pix[kRows], y0[kRows], x0[kRows];   // per staged row: first pixel of its image (-1: row past M), yo*s-1, xo*s-1
  };
  __device__ void prepare(State& st, int m0, int, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int m = m0 + r0 + kRowStep * i;
      if (m < M) {
        int b, yo, xo;
        out.pix(m, b, yo, xo);
        st.pix[i] = b * in.H * in.W;
        st.y0[i] = yo * stride - 1;
        st.x0[i] = xo * stride - 1;
      } else {
        st.pix[i] = -1;
        st.y0[i] = st.x0[i] = 0;
      }
    }
  }
  __device__ void load(const State& st, uint8_t* as, uint8_t* bs, int m0, int n0, int kt, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
    const int k = kt * kBK + kc * 8;
    const bool kval = k < K;
    const int tap = kval ? k / Cin : 0, ci = k - tap * Cin;
    const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + kRowStep * i;
      const void* src = x.p;
      uint32_t bytes = 0;
      const int yi = st.y0[i] + ky, xi = st.x0[i] + kx;
      if (kval && st.pix[i] >= 0 && (unsigned)yi < (unsigned)in.H && (unsigned)xi < (unsigned)in.W) {
        src = x.p + ((size_t)st.pix[i] + (size_t)yi * in.W + xi) * x.cs + x.co + ci;
        bytes = 16;
      }
      cp_async16(as + tile_off(r, kc, kBK), src, bytes);
    }
    for (int c = tid; c < bn * 8; c += kProducers) {
      const int r = (c & 7) + ((c >> 6) << 3), kc2 = (c >> 3) & 7;
      const int n = n0 + r, kk = kt * kBK + kc2 * 8;
      const bool v = n < N && kk < K;
      cp_async16(bs + tile_off(r, kc2, kBK), v ? (const void*)(w + (size_t)n * K + kk) : (const void*)w, v ? 16u : 0u);
    }
  }
};

// 16 consecutive bias values (the same addresses in every lane: broadcast
// loads), four 16-byte loads where the run is 16-byte aligned
__device__ __forceinline__ void load_bias16(const float* b, float* out) {
  if ((reinterpret_cast<uintptr_t>(b) & 15u) == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(b) + i);
      out[4 * i] = q.x;
      out[4 * i + 1] = q.y;
      out[4 * i + 2] = q.z;
      out[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = __ldg(b + i);
  }
}

struct BiasActStore {
  OutView y;
  const float* bias;
  int relu;
  __device__ void store(int m, int n0, const float* v, bool valid) const {
    if (!valid) return;
    float bv[16];
    load_bias16(bias + n0, bv);
    __align__(16) bf16 o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float t = v[i] + bv[i];
      o[i] = __float2bfloat16_rn(relu ? fmaxf(t, 0.f) : t);
    }
    uint4* dst = reinterpret_cast<uint4*>(y.p + (size_t)m * y.cs + y.co + n0);
    dst[0] = reinterpret_cast<const uint4*>(o)[0];
    dst[1] = reinterpret_cast<const uint4*>(o)[1];
  }
};

// ------------------------------------------------------------ conv dgrad
struct ConvDgradLoader {
  static constexpr bool kAsync = true;
  View dy;
  const bf16* wd;   // [Cin][9 Cout]: wd[ci][(ky,kx,co)] = W[co][ky][kx][ci]
  Grid in, out;     // in = dX grid (forward input), out = dY grid
  int Cout, K, N, stride, M, bn;
  struct State {
    int pix[kRows], yi[kRows], xi[kRows];   // per staged row: first pixel of its dY image (-1: past M), and its dX pixel
  };
  __device__ void prepare(State& st, int m0, int, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int m = m0 + r0 + kRowStep * i;
      if (m < M) {
        int b, yi, xi;
        in.pix(m, b, yi, xi);
        st.pix[i] = b * out.H * out.W;
        st.yi[i] = yi;
        st.xi[i] = xi;
      } else {
        st.pix[i] = -1;
        st.yi[i] = st.xi[i] = 0;
      }
    }
  }
  __device__ void load(const State& st, uint8_t* as, uint8_t* bs, int m0, int n0, int kt, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
    const int k = kt * kBK + kc * 8;
    const bool kval = k < K;
    const int tap = kval ? k / Cout : 0, co = k - tap * Cout;
    const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + kRowStep * i;
      const void* src = dy.p;
      uint32_t bytes = 0;
      const int ys = st.yi[i] + 1 - ky, xs = st.xi[i] + 1 - kx;
      if (kval && st.pix[i] >= 0 && ys >= 0 && xs >= 0) {
        const bool div = stride == 1 || (((ys | xs) & 1) == 0);
        const int yo = stride == 1 ? ys : (ys >> 1), xo = stride == 1 ? xs : (xs >> 1);
        if (div && yo < out.H && xo < out.W) {
          src = dy.p + ((size_t)st.pix[i] + (size_t)yo * out.W + xo) * dy.cs + dy.co + co;
          bytes = 16;
        }
      }
      cp_async16(as + tile_off(r, kc, kBK), src, bytes);
    }
    for (int c = tid; c < bn * 8; c += kProducers) {
      const int r = (c & 7) + ((c >> 6) << 3), kc2 = (c >> 3) & 7;
      const int n = n0 + r, kk = kt * kBK + kc2 * 8;
      const bool v = n < N && kk < K;
      cp_async16(bs + tile_off(r, kc2, kBK), v ? (const void*)(wd + (size_t)n * K + kk) : (const void*)wd, v ? 16u : 0u);
    }
  }
};

// gradient w.r.t. a post-ReLU activation x: g * [x > 0], optionally added to
// the gradient already stored there (the tensor also feeds another layer)
struct MaskedGradStore {
  OutView dx;
  View x;
  int accumulate;
  __device__ void store(int m, int n0, const float* v, bool valid) const {
    if (!valid) return;
    store_pixel(m, n0, v);
  }
  __device__ void store_pixel(long long m, int n0, const float* v) const {
    const uint4* xp = reinterpret_cast<const uint4*>(x.p + (size_t)m * x.cs + x.co + n0);
    __align__(16) bf16 xv[16];
    reinterpret_cast<uint4*>(xv)[0] = __ldg(xp);
    reinterpret_cast<uint4*>(xv)[1] = __ldg(xp + 1);
    uint4* dst = reinterpret_cast<uint4*>(dx.p + (size_t)m * dx.cs + dx.co + n0);
    __align__(16) bf16 old[16];
    if (accumulate) {
      reinterpret_cast<uint4*>(old)[0] = dst[0];
      reinterpret_cast<uint4*>(old)[1] = dst[1];
    }
    __align__(16) bf16 o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float g = __bfloat162float(xv[i]) > 0.f ? v[i] : 0.f;
      if (accumulate) g += __bfloat162float(old[i]);
      o[i] = __float2bfloat16_rn(g);
    }
    dst[0] = reinterpret_cast<const uint4*>(o)[0];
    dst[1] = reinterpret_cast<const uint4*>(o)[1];
  }
};

// the same for one parity class of a stride-2 data gradient: GEMM row m is
// pixel (y', x') of the class grid (Ho x Wo), i.e. input pixel
// (2 y' + py, 2 x' + px) of the 2Ho x 2Wo input grid
struct MaskedGradStoreS2 {
  MaskedGradStore base;
  int Ho, Wo, py, px;
  __device__ void store(int m, int n0, const float* v, bool valid) const {
    if (!valid) return;
    const int hw = Ho * Wo, b = m / hw, r = m - b * hw, y = r / Wo, xx = r - y * Wo;
    base.store_pixel(((long long)b * 2 * Ho + 2 * y + py) * (2 * Wo) + 2 * xx + px, n0, v);
  }
};

// ------------------------------------------------------- transposed conv
struct ConvTFwdLoader {
  static constexpr bool kAsync = true;
  View x;
  const bf16* w4;   // [4 Cout][Cin]
  int Cin, N, M, bn;
  struct State {};
  __device__ void prepare(State&, int, int, int) const {}
  __device__ void load(const State&, uint8_t* as, uint8_t* bs, int m0, int n0, int kt, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
    const int k = kt * kBK + kc * 8;
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + kRowStep * i, m = m0 + r;
      const bool v = m < M && k < Cin;
      cp_async16(as + tile_off(r, kc, kBK), v ? (const void*)(x.p + (size_t)m * x.cs + x.co + k) : (const void*)x.p,
                 v ? 16u : 0u);
    }
    for (int c = tid; c < bn * 8; c += kProducers) {
      const int r = (c & 7) + ((c >> 6) << 3), kc2 = (c >> 3) & 7;
      const int n = n0 + r, kk = kt * kBK + kc2 * 8;
      const bool v = n < N && kk < Cin;
      cp_async16(bs + tile_off(r, kc2, kBK), v ? (const void*)(w4 + (size_t)n * Cin + kk) : (const void*)w4,
                 v ? 16u : 0u);
    }
  }
};

struct ConvTStore {
  OutView y;
  const float* bias;
  Grid in;     // input grid; output is 2H x 2W
  int Cout, relu;
  __device__ void store(int m, int n0, const float* v, bool valid) const {
    if (!valid) return;
    const int d = n0 / Cout, co = n0 - d * Cout;   // 16 consecutive n stay in one (dy, dx)
    const int dyy = d >> 1, dxx = d & 1;
    int b, yy, xx;
    in.pix(m, b, yy, xx);
    const size_t op = ((size_t)(b * 2 * in.H + 2 * yy + dyy) * (2 * in.W) + 2 * xx + dxx);
    float bv[16];
    load_bias16(bias + co, bv);
    __align__(16) bf16 o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float t = v[i] + bv[i];
      o[i] = __float2bfloat16_rn(relu ? fmaxf(t, 0.f) : t);
    }
    uint4* dst = reinterpret_cast<uint4*>(y.p + op * y.cs + y.co + co);
    dst[0] = reinterpret_cast<const uint4*>(o)[0];
    dst[1] = reinterpret_cast<const uint4*>(o)[1];
  }
};

struct ConvTDgradLoader {
  static constexpr bool kAsync = true;
  View dy;
  const bf16* w4t;   // [Cin][4 Cout]
  Grid in;           // dX grid (convT input); dY is 2H x 2W
  int Cout, K, N, M, bn;
  struct State {
    int base[kRows];     // per staged row: dY pixel index of (2y, 2x), -1 past M
  };
  __device__ void prepare(State& st, int m0, int, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int m = m0 + r0 + kRowStep * i;
      if (m < M) {
        int b, yy, xx;
        in.pix(m, b, yy, xx);
        st.base[i] = (b * 2 * in.H + 2 * yy) * (2 * in.W) + 2 * xx;
      } else {
        st.base[i] = -1;
      }
    }
  }
  __device__ void load(const State& st, uint8_t* as, uint8_t* bs, int m0, int n0, int kt, int tid) const {
    int kc, r0;
    a_chunk(tid, kc, r0);
    const int k = kt * kBK + kc * 8;
    const bool kval = k < K;
    const int d = kval ? k / Cout : 0, co = k - d * Cout;
    const int off = (d >> 1) * (2 * in.W) + (d & 1);
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + kRowStep * i;
      const bool v = kval && st.base[i] >= 0;
      cp_async16(as + tile_off(r, kc, kBK),
                 v ? (const void*)(dy.p + ((size_t)st.base[i] + off) * dy.cs + dy.co + co) : (const void*)dy.p,
                 v ? 16u : 0u);
    }
    for (int c = tid; c < bn * 8; c += kProducers) {
      const int r = (c & 7) + ((c >> 6) << 3), kc2 = (c >> 3) & 7;
      const int n = n0 + r, kk = kt * kBK + kc2 * 8;
      const bool v = n < N && kk < K;
      cp_async16(bs + tile_off(r, kc2, kBK), v ? (const void*)(w4t + (size_t)n * K + kk) : (const void*)w4t,
                 v ? 16u : 0u);
    }
  }
};

// ------------------------------------------------------ TMA loaders
// A 3x3 convolution (or the data gradient of a stride-1 one) whose operand
// channels C are a multiple of CB (64, 32 or 8): every CB-wide slice of a
// 64-wide K step lies in one tap, and the tile's 128 output pixels are
// Yb rows x Xb columns of one image, so each slice of the step's A tile
// is one tensor copy of the input box shifted by the tap's offset
// (stride 2: every other pixel), the copy's zero fill standing in for the
// padding; slices past K copy a box wholly outside the image (zeros).
// B: the 64 x BN box of the weights [N][K].
template <int CB>
struct ConvTmaLoader {
  static constexpr bool kTma = true;
  static constexpr int kALayout = CB == 64 ? 0 : (CB == 32 ? 1 : 2);
  static constexpr int kSlices = kBK / CB;
  static constexpr uint32_t kSliceBytes = kBM * CB * 2;
  CUtensorMap ta;   // activations: (C, W, H, B), traversal steps (1, s, s, 1)
  CUtensorMap tb;   // weights: (K, N)
  int Ho, Wo;       // grid of the GEMM rows
  int Hi;           // input rows
  int C, stride, sign;   // channels per tap; sign +1: tap offset k - 1 (forward), -1: 1 - k (data gradient)
  // tiles past the last row (m0 >= B Ho Wo) land wholly outside the batch: zeros
  __device__ void issue_a(uint32_t as, int m0, int kt, uint32_t bar) const {
    const int hw = Ho * Wo, b = m0 / hw, r = m0 - b * hw, y0 = r / Wo, x0 = r - y0 * Wo;
    const int k = kt * kBK;
#pragma unroll
    for (int j = 0; j < kSlices; ++j) {
      const int kk = k + j * CB, tap = kk / C, c0 = kk - tap * C, ky = tap / 3, kx = tap - 3 * ky;
      if (tap < 9)
        tma_load_4d(as + j * kSliceBytes, &ta, c0, x0 * stride + sign * (kx - 1), y0 * stride + sign * (ky - 1), b,
                    bar);
      else
        tma_load_4d(as + j * kSliceBytes, &ta, 0, 0, Hi, b, bar);
    }
  }
  __device__ void issue_b(uint32_t bs, int n0, int kt, uint32_t bar) const { tma_load_2d(bs, &tb, kt * kBK, n0, bar); }
};

// 128 pixels of one image as Yb rows x Xb columns
inline bool conv_tma_box(int Ho, int Wo, int& Xb, int& Yb) {
  if (Wo % kBM == 0) {
    Xb = kBM;
    Yb = 1;
    return true;
  }
  if (kBM % Wo == 0 && Ho % (kBM / Wo) == 0) {
    Xb = Wo;
    Yb = kBM / Wo;
    return true;
  }
  return false;
}

// activations x (C channels of a view on an Hi x Wi grid, B images) feeding
// GEMM rows on an Ho x Wo grid; weights w [N][K]
template <int CB>
inline bool make_conv_tma(ConvTmaLoader<CB>& L, View x, int C, int B, int Hi, int Wi, int Ho, int Wo, int stride,
                          int sign, const bf16* w, int K, int N, int bn) {
  int Xb, Yb;
  if (C % CB || !conv_tma_box(Ho, Wo, Xb, Yb)) return false;
  const uint64_t pitch = (uint64_t)x.cs * 2;
  const uint64_t d[4] = {(uint64_t)C, (uint64_t)Wi, (uint64_t)Hi, (uint64_t)B};
  const uint64_t st[3] = {pitch, pitch * Wi, pitch * Wi * Hi};
  const uint32_t bx[4] = {(uint32_t)CB, (uint32_t)(Xb * stride), (uint32_t)(Yb * stride), 1};
  const uint32_t e[4] = {1, (uint32_t)stride, (uint32_t)stride, 1};
  if (!tma::encode_bf16(&L.ta, x.p + x.co, 4, d, st, bx, e, CB == 8 ? 0 : 2 * CB) || !rows_map(&L.tb, w, K, N, K, bn))
    return false;
  L.Ho = Ho;
  L.Wo = Wo;
  L.Hi = Hi;
  L.C = C;
  L.stride = stride;
  L.sign = sign;
  return true;
}

// run a convolution GEMM through the TMA loader with the widest channel
// slice that divides C; false if its shape does not fit one
template <class Ep>
bool conv_tma(cudaError_t& e, View x, int C, int B, int Hi, int Wi, int Ho, int Wo, int stride, int sign,
              const bf16* w, int K, int N, int bn, const Ep& ep, int M, unsigned* err, cudaStream_t st) {
  if (C % 64 == 0) {
    ConvTmaLoader<64> L;
    if (!make_conv_tma(L, x, C, B, Hi, Wi, Ho, Wo, stride, sign, w, K, N, bn)) return false;
    e = gemm_bn(bn, L, ep, M, N, K, err, st);
    return true;
  }
  if (C % 32 == 0) {
    ConvTmaLoader<32> L;
    if (!make_conv_tma(L, x, C, B, Hi, Wi, Ho, Wo, stride, sign, w, K, N, bn)) return false;
    e = gemm_bn(bn, L, ep, M, N, K, err, st);
    return true;
  }
  if (C % 8 == 0 && bn == 32) {   // only the first layer (8 input channels) takes this path
    ConvTmaLoader<8> L;
    if (!make_conv_tma(L, x, C, B, Hi, Wi, Ho, Wo, stride, sign, w, K, N, bn)) return false;
    e = launch_umma_gemm<32, 4>(L, ep, M, N, K, err, st);
    return true;
  }
  return false;
}

// Data gradient of a stride-2 3x3 convolution, one output-parity class
// (py, px) at a time: input pixel (2y' + py, 2x' + px) receives dY at
// (y' + oy, x' + ox) through the taps ky = py + 1 - 2 oy (kx likewise) that
// land on it - 1, 2, 2 or 4 taps instead of 9 with three quarters zero.  A
// = tensor copies of the dY box of the tile's 128 class pixels shifted by
// (oy, ox) per tap (64 output channels per K step); B = the columns of the
// transposed weights [Cin][9 Cout] of the class's taps.
struct DgradS2TmaLoader {
  static constexpr bool kTma = true;
  CUtensorMap ta;   // dY: (Cout, Wo, Ho, B)
  CUtensorMap tb;   // transposed weights: (9 Cout, Cin)
  int Ho, Wo, Cout, ntaps;
  int tap[4], oy[4], ox[4];
  __device__ void issue_a(uint32_t as, int m0, int kt, uint32_t bar) const {
    const int hw = Ho * Wo, b = m0 / hw, r = m0 - b * hw, y0 = r / Wo, x0 = r - y0 * Wo;
    const int k = kt * kBK, i = k / Cout, c0 = k - i * Cout;
    tma_load_4d(as, &ta, c0, x0 + ox[i], y0 + oy[i], b, bar);
  }
  __device__ void issue_b(uint32_t bs, int n0, int kt, uint32_t bar) const {
    const int k = kt * kBK, i = k / Cout, c0 = k - i * Cout;
    tma_load_2d(bs, &tb, tap[i] * Cout + c0, n0, bar);
  }
};

// Weight gradient of a 3x3 convolution through tensor copies, both operands
// MN-major (channels contiguous, as the NHWC tensors already are): for the
// K step of 64 output pixels (a box of Yb rows x Xb columns of one image),
// A = the input pixels under tap (ky, kx), CB (64 or 32) channels per
// swizzled box (128 / CB boxes per tile, each inside one tap), B = the
// output gradient of the same pixels, BN channels in boxes of up to 64.
// Rows past the last tap copy a box wholly outside the image.
template <int CB>
struct WgradTmaLoader {
  static constexpr bool kTma = true;
  static constexpr int kALayout = CB == 64 ? 3 : 4;
  static constexpr bool kBMajorMN = true;
  static constexpr int kBoxes = kBM / CB;
  static constexpr uint32_t kBoxBytes = 64u * 2u * CB;
  CUtensorMap ta;   // X: (Cin, Wi, Hi, B), traversal steps (1, s, s, 1), box (64, Xb s, Yb s, 1)
  CUtensorMap tb;   // dY: (Cout, Wo, Ho, B), box (bb, Xb, Yb, 1)
  int Ho, Wo, Hi, Cin, stride, bb, nbox;   // bb channels per B box, nbox boxes per B tile
  __device__ __forceinline__ void pix(int kt, int& b, int& y0, int& x0) const {
    const int p0 = kt * kBK, hw = Ho * Wo;
    b = p0 / hw;
    const int r = p0 - b * hw;
    y0 = r / Wo;
    x0 = r - y0 * Wo;
  }
  __device__ void issue_a(uint32_t as, int m0, int kt, uint32_t bar) const {
    int b, y0, x0;
    pix(kt, b, y0, x0);
#pragma unroll
    for (int h = 0; h < kBoxes; ++h) {
      const int r = m0 + CB * h, tap = r / Cin, c = r - tap * Cin, ky = tap / 3, kx = tap - 3 * ky;
      if (tap < 9)
        tma_load_4d(as + h * kBoxBytes, &ta, c, x0 * stride + kx - 1, y0 * stride + ky - 1, b, bar);
      else
        tma_load_4d(as + h * kBoxBytes, &ta, 0, 0, Hi, b, bar);
    }
  }
  __device__ void issue_b(uint32_t bs, int n0, int kt, uint32_t bar) const {
    int b, y0, x0;
    pix(kt, b, y0, x0);
    for (int j = 0; j < nbox; ++j) tma_load_4d(bs + (uint32_t)j * 64u * 2u * (uint32_t)bb, &tb, n0 + j * bb, x0, y0, b, bar);
  }
};

// 64 pixels of one image as Yb rows x Xb columns
inline bool pix64_box(int Ho, int Wo, int& Xb, int& Yb) {
  if (Wo % 64 == 0) {
    Xb = 64;
    Yb = 1;
    return true;
  }
  if (64 % Wo == 0 && Ho % (64 / Wo) == 0) {
    Xb = Wo;
    Yb = 64 / Wo;
    return true;
  }
  return false;
}

template <int CB>
inline bool make_wgrad_tma(WgradTmaLoader<CB>& L, View x, View dy, int Cin, int Cout, int B, int Hi, int Wi, int Ho,
                           int Wo, int stride, int bn) {
  int Xb, Yb;
  // B tiles of 32 or more channels (64- and 128-byte swizzled MN-major
  // boxes); 16-channel outputs gather with the register-transpose loader
  if (Cin % CB || bn < 32 || !pix64_box(Ho, Wo, Xb, Yb)) return false;
  const int bb = bn < 64 ? bn : 64;
  {
    const uint64_t pitch = (uint64_t)x.cs * 2;
    const uint64_t d[4] = {(uint64_t)Cin, (uint64_t)Wi, (uint64_t)Hi, (uint64_t)B};
    const uint64_t st[3] = {pitch, pitch * Wi, pitch * Wi * Hi};
    const uint32_t bx[4] = {(uint32_t)CB, (uint32_t)(Xb * stride), (uint32_t)(Yb * stride), 1};
    const uint32_t e[4] = {1, (uint32_t)stride, (uint32_t)stride, 1};
    if (!tma::encode_bf16(&L.ta, x.p + x.co, 4, d, st, bx, e, 2 * CB)) return false;
  }
  {
    const uint64_t pitch = (uint64_t)dy.cs * 2;
    const uint64_t d[4] = {(uint64_t)Cout, (uint64_t)Wo, (uint64_t)Ho, (uint64_t)B};
    const uint64_t st[3] = {pitch, pitch * Wo, pitch * Wo * Ho};
    const uint32_t bx[4] = {(uint32_t)bb, (uint32_t)Xb, (uint32_t)Yb, 1};
    const uint32_t e[4] = {1, 1, 1, 1};
    if (!tma::encode_bf16(&L.tb, dy.p + dy.co, 4, d, st, bx, e, 2 * bb)) return false;
  }
  L.Ho = Ho;
  L.Wo = Wo;
  L.Hi = Hi;
  L.Cin = Cin;
  L.stride = stride;
  L.bb = bb;
  L.nbox = bn / bb;
  return true;
}

// --------------------------------------------------------------- wgrad
// Both operands of a weight gradient are stored pixel-major (channels
// contiguous), while the GEMM reduces over pixels.  The loader reads
// 8 channels x 8 pixels (eight 16-byte loads), transposes the 8 x 8 BF16
// block in registers with byte permutes, and stores 8 pixels x 8 channels.
__device__ __forceinline__ void transpose8x8(const uint4* in, uint4* out) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(in);   // w[4 p + j]: channels 2j, 2j+1 of pixel p
  uint32_t* o = reinterpret_cast<uint32_t*>(out);               // o[4 c + j]: pixels 2j, 2j+1 of channel c
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      o[4 * c + j] = __byte_perm(w[4 * (2 * j) + (c >> 1)], w[4 * (2 * j + 1) + (c >> 1)], (c & 1) ? 0x7632 : 0x5410);
}

// source of one operand of a weight gradient: channel group (8 channels)
// `r8` of pixel p, or zeros
struct ConvIm2col {   // rows (ky, kx, ci) of the forward input's im2col
  View x;
  Grid in, out;
  int Cin, stride, rows;
  __device__ __forceinline__ uint4 get(int row, int p, int P) const {
    if (row >= rows || p >= P) return make_uint4(0, 0, 0, 0);
    const int tap = row / Cin, ci = row - tap * Cin, ky = tap / 3, kx = tap - ky * 3;
    int b, yo, xo;
    out.pix(p, b, yo, xo);
    const int yi = yo * stride - 1 + ky, xi = xo * stride - 1 + kx;
    if ((unsigned)yi >= (unsigned)in.H || (unsigned)xi >= (unsigned)in.W) return make_uint4(0, 0, 0, 0);
    return __ldg(reinterpret_cast<const uint4*>(x.p + ((size_t)(b * in.H + yi) * in.W + xi) * x.cs + x.co + ci));
  }
};
struct PixelRows {    // rows = channels of a tensor on the reduction grid
  View t;
  int rows;
  __device__ __forceinline__ uint4 get(int row, int p, int P) const {
    if (row >= rows || p >= P) return make_uint4(0, 0, 0, 0);
    return __ldg(reinterpret_cast<const uint4*>(t.p + (size_t)p * t.cs + t.co + row));
  }
};
struct ConvTGather {  // rows (d, co) of the transposed conv's output gradient, on its input grid
  View dy;
  Grid in;
  int Cout, rows;
  __device__ __forceinline__ uint4 get(int row, int p, int P) const {
    if (row >= rows || p >= P) return make_uint4(0, 0, 0, 0);
    const int d = row / Cout, co = row - d * Cout;
    int b, yy, xx;
    in.pix(p, b, yy, xx);
    const size_t op = (size_t)(b * 2 * in.H + 2 * yy + (d >> 1)) * (2 * in.W) + 2 * xx + (d & 1);
    return __ldg(reinterpret_cast<const uint4*>(dy.p + op * dy.cs + dy.co + co));
  }
};

template <class SrcA, class SrcB>
struct WgradLoader {
  static constexpr bool kAsync = false;
  SrcA a;
  SrcB b;
  int P, bn;   // pixels in the reduction
  struct State {};
  __device__ void prepare(State&, int, int, int) const {}
  __device__ void load(const State&, uint8_t* as, uint8_t* bs, int m0, int n0, int kt, int tid) const {
    const int p0 = kt * kBK;
    // A: 16 row groups x 8 pixel groups = 128 blocks; B: bn / 8 x 8 = bn blocks
    for (int blk = tid; blk < 128 + bn; blk += kProducers) {
      const bool isA = blk < 128;
      const int id = isA ? blk : blk - 128;
      const int rg = id >> 3, pg = id & 7;
      uint4 in[8], out[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) in[q] = isA ? a.get(m0 + rg * 8, p0 + pg * 8 + q, P) : b.get(n0 + rg * 8, p0 + pg * 8 + q, P);
      transpose8x8(in, out);
      uint8_t* dst = isA ? as : bs;
#pragma unroll
      for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4*>(dst + tile_off(rg * 8 + c, pg, kBK)) = out[c];
    }
  }
};

struct AtomicF32Store {   // G[m][n] += v (FP32), rows < M
  float* g;
  int N, M;
  __device__ void store(int m, int n0, const float* v, bool valid) const {
    if (!valid || m >= M) return;
    float* dst = g + (size_t)m * N + n0;
#pragma unroll
    for (int i = 0; i < 16; ++i) atomicAdd(dst + i, v[i]);
  }
};

// --------------------------------------------------------------- launch
// TMA loaders run narrow tiles with several issuing warps (tiles per group):
// 4 up to BN = 64, 2 at 128, 1 at 256
template <class Ld, class Ep>
cudaError_t gemm_bn(int bn, const Ld& ld, const Ep& ep, int M, int N, int K, unsigned* err, cudaStream_t st,
                    int splits = 1) {
  constexpr bool T = is_tma_loader<Ld>::value;
  switch (bn) {
    case 256: return launch_umma_gemm<256, 1>(ld, ep, M, N, K, err, st, splits);
    case 128: return launch_umma_gemm<128, T ? 2 : 1>(ld, ep, M, N, K, err, st, splits);
    case 64: return launch_umma_gemm<64, T ? 4 : 1>(ld, ep, M, N, K, err, st, splits);
    case 32: return launch_umma_gemm<32, T ? 4 : 1>(ld, ep, M, N, K, err, st, splits);
    case 16: return launch_umma_gemm<16, T ? 4 : 1>(ld, ep, M, N, K, err, st, splits);
    default: return cudaErrorInvalidValue;
  }
}

// Stride-1 forward of the narrow layers through the haloed-box kernel
// (conv_halo.cuh): CIN, COUT in {32, 64}, and the first layer's 8 -> 32.  False (e untouched) if the shape
// has no instantiation or the tensor map cannot describe the input.
template <int CIN, int COUT>
bool halo_fwd(cudaError_t& e, View x, const bf16* w, const float* bias, OutView y, int relu, int B, int H, int W,
              unsigned* err, cudaStream_t st, const float* head_w = nullptr, const float* head_b = nullptr,
              float* head_out = nullptr) {
  using Cf = HaloCfg<CIN, COUT>;
  CUtensorMap m;
  const uint64_t pitch = (uint64_t)x.cs * 2;
  const uint64_t d[4] = {(uint64_t)CIN, (uint64_t)W, (uint64_t)H, (uint64_t)B};
  const uint64_t strd[3] = {pitch, pitch * W, pitch * W * H};
  const uint32_t bx[4] = {8, (uint32_t)Cf::BX, (uint32_t)Cf::BY, 1}, es[4] = {1, 1, 1, 1};
  if (!tma::encode_bf16(&m, x.p + x.co, 4, d, strd, bx, es, 0)) return false;
  HaloArgs a;
  a.w = w;
  a.bias = bias;
  a.y = y.p;
  a.y_cs = y.cs;
  a.y_co = y.co;
  a.relu = relu;
  a.head_w = head_w;
  a.head_b = head_b;
  a.head_out = head_out;
  a.B = B;
  a.H = H;
  a.W = W;
  a.tiles_y = (H + Cf::TY - 1) / Cf::TY;
  a.tiles_x = (W + Cf::TX - 1) / Cf::TX;
  const long long nt = (long long)B * a.tiles_y * a.tiles_x;
  if (nt > (1ll << 30)) return false;
  a.n_tiles = (int)nt;
  auto kern = conv3x3_halo_kernel<CIN, COUT>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM)) != cudaSuccess)
    return true;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<long long>(nt, sms);
  kern<<<grid, Cf::THREADS, Cf::SMEM, st>>>(m, a, err);
  e = cudaGetLastError();
  return true;
}

// Stride-1 forward of a wide-input layer (CIN 128 or 256; COUT 64, 128 or 256)
// through the haloed-box kernel with streamed weights.  False (e untouched)
// if a tensor map cannot describe the operands.
template <int CIN, int COUT>
bool halo_stream_fwd(cudaError_t& e, View x, const bf16* w, const float* bias, OutView y, int relu, int B, int H,
                     int W, unsigned* err, cudaStream_t st) {
  using Cf = HaloStreamCfg<CIN, COUT>;
  CUtensorMap mx, mw;
  const uint64_t pitch = (uint64_t)x.cs * 2;
  const uint64_t d[4] = {(uint64_t)CIN, (uint64_t)W, (uint64_t)H, (uint64_t)B};
  const uint64_t strd[3] = {pitch, pitch * W, pitch * W * H};
  const uint32_t bx[4] = {8, (uint32_t)Cf::BX, (uint32_t)Cf::BY, 1}, es[4] = {1, 1, 1, 1};
  // weights w [COUT][3][3][CIN]: rows of 9 CIN, chunks of 64 x COUT
  if (!tma::encode_bf16(&mx, x.p + x.co, 4, d, strd, bx, es, 0) || !rows_map(&mw, w, 9 * CIN, COUT, 9 * CIN, COUT))
    return false;
  HaloArgs a;
  a.w = w;
  a.bias = bias;
  a.y = y.p;
  a.y_cs = y.cs;
  a.y_co = y.co;
  a.relu = relu;
  a.B = B;
  a.H = H;
  a.W = W;
  a.tiles_y = (H + Cf::TY - 1) / Cf::TY;
  a.tiles_x = (W + Cf::TX - 1) / Cf::TX;
  const long long nt = (long long)B * a.tiles_y * a.tiles_x;
  if (nt > (1ll << 26)) return false;
  a.n_tiles = (int)nt;
  auto kern = conv3x3_halo_stream_kernel<CIN, COUT>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM)) != cudaSuccess)
    return true;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<long long>(nt, sms);
  kern<<<grid, Cf::THREADS, Cf::SMEM, st>>>(mx, mw, a, err);
  e = cudaGetLastError();
  return true;
}

bool halo_fwd_any(cudaError_t& e, View x, int Cin, int Cout, const bf16* w, const float* bias, OutView y, int relu,
                  int B, int H, int W, unsigned* err, cudaStream_t st) {
  // 512 frames: 128 -> 128 at 64 x 64, 1,385 TFLOP/s here against 1,053 tap by tap; 128 -> 64 at
  // 128 x 128, 1,057 against 701
  if (Cin == 128 && Cout == 128) return halo_stream_fwd<128, 128>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 128 && Cout == 64) return halo_stream_fwd<128, 64>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 256 && Cout == 128) return halo_stream_fwd<256, 128>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 256 && Cout == 256) return halo_stream_fwd<256, 256>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 8 && Cout == 32) return halo_fwd<8, 32>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 32 && Cout == 32) return halo_fwd<32, 32>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 64 && Cout == 32) return halo_fwd<64, 32>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 32 && Cout == 64) return halo_fwd<32, 64>(e, x, w, bias, y, relu, B, H, W, err, st);
  if (Cin == 64 && Cout == 64) return halo_fwd<64, 64>(e, x, w, bias, y, relu, B, H, W, err, st);
  return false;
}

bool aligned16(const void* p);

bool conv3x3_head_fwd(cudaError_t& e, const uint16_t* x, int x_cs, int x_co, int Cin, const uint16_t* w,
                      const float* bias, uint16_t* y, int y_cs, int y_co, int B, int H, int W, const float* head_w,
                      const float* head_b, float* head_out, unsigned* err, cudaStream_t st) {
  if (!x || !w || !bias || !head_w || !head_b || !head_out || (x_cs % 8) || (x_co % 8) || x_co + Cin > x_cs ||
      !aligned16(x) || !aligned16(w) || (y && ((y_cs % 8) || (y_co % 8) || y_co + 32 > y_cs || !aligned16(y))))
    return false;
  const View xv{(const bf16*)x, x_cs, x_co};
  const OutView yv{(bf16*)y, y_cs, y_co};
  if (Cin == 32)
    return halo_fwd<32, 32>(e, xv, (const bf16*)w, bias, yv, 1, B, H, W, err, st, head_w, head_b, head_out);
  if (Cin == 64)
    return halo_fwd<64, 32>(e, xv, (const bf16*)w, bias, yv, 1, B, H, W, err, st, head_w, head_b, head_out);
  return false;
}

int pick_bn(int N) {
  return (N % 256 == 0) ? 256 : (N % 128 == 0) ? 128 : (N % 64 == 0) ? 64 : (N % 32 == 0) ? 32 : (N % 16 == 0) ? 16 : 0;
}

// split the pixel reduction of a weight gradient so that the grid covers
// about four waves of the GPU
int wgrad_splits(int mt, int nt, long long P, int X = 1) {
  mt = (mt + X - 1) / X;   // tile groups along M
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = 4LL * sms;
  long long s = (want + (long long)mt * nt - 1) / ((long long)mt * nt);
  const long long ktot = (P + kBK - 1) / kBK;
  if (s > ktot) s = ktot;
  return (int)(s < 1 ? 1 : s);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace surr
}  // namespace ussim

using namespace ussim;
using namespace ussim::surr;

#define US_CHECK(cond) \
  do {                 \
    if (!(cond)) return US_ERR_INVALID_ARG; \
  } while (0)

static us_status to_status(cudaError_t e) { return e == cudaSuccess ? US_OK : US_ERR_CUDA; }

extern "C" {

us_status us_conv3x3_fwd(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* w, const float* bias,
                         uint16_t* y, int32_t y_cs, int32_t y_co, int32_t B, int32_t H, int32_t W, int32_t Cin,
                         int32_t Cout, int32_t stride, int32_t relu, uint32_t* err, void* stream) {
  US_CHECK(x && w && bias && y && err && B > 0 && H > 0 && W > 0 && (stride == 1 || stride == 2));
  US_CHECK(Cin % 8 == 0 && Cin > 0 && pick_bn(Cout) && x_cs % 8 == 0 && x_co % 8 == 0 && x_co + Cin <= x_cs);
  US_CHECK(y_cs % 8 == 0 && y_co % 8 == 0 && y_co + Cout <= y_cs && aligned16(x) && aligned16(y) && aligned16(w));
  const Grid in{B, H, W}, out{B, (H - 1) / stride + 1, (W - 1) / stride + 1};
  const int M = B * out.H * out.W, K = 9 * Cin, bn = pick_bn(Cout);
  BiasActStore ep{{(bf16*)y, y_cs, y_co}, bias, relu};
  cudaError_t e;
  if (stride == 1 && halo_fwd_any(e, {(const bf16*)x, x_cs, x_co}, Cin, Cout, (const bf16*)w, bias,
                                  {(bf16*)y, y_cs, y_co}, relu, B, H, W, err, (cudaStream_t)stream))
    return to_status(e);
  if (conv_tma(e, {(const bf16*)x, x_cs, x_co}, Cin, B, H, W, out.H, out.W, stride, 1, (const bf16*)w, K, Cout, bn, ep,
               M, err, (cudaStream_t)stream))
    return to_status(e);
  ConvFwdLoader ld{{(const bf16*)x, x_cs, x_co}, (const bf16*)w, in, out, Cin, K, Cout, stride, M, bn};
  return to_status(gemm_bn(bn, ld, ep, M, Cout, K, err, (cudaStream_t)stream));
}

us_status us_conv3x3_dgrad(const uint16_t* dy, int32_t dy_cs, int32_t dy_co, const uint16_t* wd, const uint16_t* x,
                           int32_t x_cs, int32_t x_co, uint16_t* dx, int32_t dx_cs, int32_t dx_co, int32_t accumulate,
                           int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout, int32_t stride, uint32_t* err,
                           void* stream) {
  US_CHECK(dy && wd && x && dx && err && B > 0 && H > 0 && W > 0 && (stride == 1 || stride == 2));
  US_CHECK(Cout % 8 == 0 && pick_bn(Cin) && dy_cs % 8 == 0 && dy_co % 8 == 0 && x_cs % 8 == 0 && x_co % 8 == 0);
  US_CHECK(dx_cs % 8 == 0 && dx_co % 8 == 0 && aligned16(dy) && aligned16(wd) && aligned16(x) && aligned16(dx));
  const Grid in{B, H, W}, out{B, (H - 1) / stride + 1, (W - 1) / stride + 1};
  const int M = B * H * W, K = 9 * Cout, bn = pick_bn(Cin);
  MaskedGradStore ep{{(bf16*)dx, dx_cs, dx_co}, {(const bf16*)x, x_cs, x_co}, accumulate};
  cudaError_t e;
  if (stride == 1 && conv_tma(e, {(const bf16*)dy, dy_cs, dy_co}, Cout, B, H, W, H, W, 1, -1, (const bf16*)wd, K, Cin,
                              bn, ep, M, err, (cudaStream_t)stream))
    return to_status(e);
  int Xb, Yb;
  if (stride == 2 && H % 2 == 0 && W % 2 == 0 && Cout % kBK == 0 && conv_tma_box(out.H, out.W, Xb, Yb)) {
    // four parity classes, each a dense convolution over dY with its own taps
    DgradS2TmaLoader tl;
    const uint64_t pitch = (uint64_t)dy_cs * 2;
    const uint64_t d[4] = {(uint64_t)Cout, (uint64_t)out.W, (uint64_t)out.H, (uint64_t)B};
    const uint64_t st[3] = {pitch, pitch * out.W, pitch * out.W * out.H};
    const uint32_t bx[4] = {(uint32_t)kBK, (uint32_t)Xb, (uint32_t)Yb, 1}, es[4] = {1, 1, 1, 1};
    if (tma::encode_bf16(&tl.ta, (const bf16*)dy + dy_co, 4, d, st, bx, es) &&
        rows_map(&tl.tb, (const bf16*)wd, K, Cin, K, bn)) {
      tl.Ho = out.H;
      tl.Wo = out.W;
      tl.Cout = Cout;
      const int Mc = B * out.H * out.W;
      for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px) {
          tl.ntaps = 0;
          for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx)
              if (((py + 1 - ky) & 1) == 0 && ((px + 1 - kx) & 1) == 0) {
                tl.tap[tl.ntaps] = 3 * ky + kx;
                tl.oy[tl.ntaps] = (py + 1 - ky) / 2;
                tl.ox[tl.ntaps] = (px + 1 - kx) / 2;
                ++tl.ntaps;
              }
          MaskedGradStoreS2 eps{ep, out.H, out.W, py, px};
          if ((e = gemm_bn(bn, tl, eps, Mc, Cin, tl.ntaps * Cout, err, (cudaStream_t)stream)) != cudaSuccess)
            return to_status(e);
        }
      return US_OK;
    }
  }
  ConvDgradLoader ld{{(const bf16*)dy, dy_cs, dy_co}, (const bf16*)wd, in, out, Cout, K, Cin, stride, M, bn};
  return to_status(gemm_bn(bn, ld, ep, M, Cin, K, err, (cudaStream_t)stream));
}

us_status us_conv3x3_wgrad(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* dy, int32_t dy_cs,
                           int32_t dy_co, float* gwt, int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout,
                           int32_t stride, uint32_t* err, void* stream) {
  US_CHECK(x && dy && gwt && err && B > 0 && H > 0 && W > 0 && (stride == 1 || stride == 2));
  US_CHECK(Cin % 8 == 0 && pick_bn(Cout) && x_cs % 8 == 0 && x_co % 8 == 0 && dy_cs % 8 == 0 && dy_co % 8 == 0);
  US_CHECK(aligned16(x) && aligned16(dy));
  const Grid in{B, H, W}, out{B, (H - 1) / stride + 1, (W - 1) / stride + 1};
  const int rows = 9 * Cin, P = B * out.H * out.W, bn = pick_bn(Cout);
  AtomicF32Store ep{gwt, Cout, rows};
  const int mt = (rows + kBM - 1) / kBM, nt = Cout / bn;
  const int X = bn <= 64 ? 4 : (bn <= 128 ? 2 : 1);
  const View xv{(const bf16*)x, x_cs, x_co}, dyv{(const bf16*)dy, dy_cs, dy_co};
  if (Cin % 64 == 0) {
    WgradTmaLoader<64> tl;
    if (make_wgrad_tma(tl, xv, dyv, Cin, Cout, B, H, W, out.H, out.W, stride, bn))
      return to_status(gemm_bn(bn, tl, ep, rows, Cout, P, err, (cudaStream_t)stream, wgrad_splits(mt, nt, P, X)));
  } else if (Cin % 32 == 0) {
    WgradTmaLoader<32> tl;
    if (make_wgrad_tma(tl, xv, dyv, Cin, Cout, B, H, W, out.H, out.W, stride, bn))
      return to_status(gemm_bn(bn, tl, ep, rows, Cout, P, err, (cudaStream_t)stream, wgrad_splits(mt, nt, P, X)));
  }
  WgradLoader<ConvIm2col, PixelRows> ld{{{(const bf16*)x, x_cs, x_co}, in, out, Cin, stride, rows},
                                        {{(const bf16*)dy, dy_cs, dy_co}, Cout}, P, bn};
  return to_status(gemm_bn(bn, ld, ep, rows, Cout, P, err, (cudaStream_t)stream, wgrad_splits(mt, nt, P)));
}

us_status us_convT2x2_fwd(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* w4, const float* bias,
                          uint16_t* y, int32_t y_cs, int32_t y_co, int32_t B, int32_t H, int32_t W, int32_t Cin,
                          int32_t Cout, int32_t relu, uint32_t* err, void* stream) {
  US_CHECK(x && w4 && bias && y && err && B > 0 && H > 0 && W > 0);
  US_CHECK(Cin % 8 == 0 && Cout % 16 == 0 && pick_bn(4 * Cout) && x_cs % 8 == 0 && x_co % 8 == 0);
  US_CHECK(y_cs % 8 == 0 && y_co % 8 == 0 && aligned16(x) && aligned16(w4) && aligned16(y));
  const int M = B * H * W, N = 4 * Cout, bn = pick_bn(N);   // 16-column chunks never straddle a (dy, dx) block
  ConvTStore ep{{(bf16*)y, y_cs, y_co}, bias, {B, H, W}, Cout, relu};
  RowsTmaLoader tl;
  if (rows_map(&tl.ta, (const bf16*)x + x_co, x_cs, M, Cin, kBM) && rows_map(&tl.tb, (const bf16*)w4, Cin, N, Cin, bn))
    return to_status(gemm_bn(bn, tl, ep, M, N, Cin, err, (cudaStream_t)stream));
  ConvTFwdLoader ld{{(const bf16*)x, x_cs, x_co}, (const bf16*)w4, Cin, N, M, bn};
  return to_status(gemm_bn(bn, ld, ep, M, N, Cin, err, (cudaStream_t)stream));
}

us_status us_convT2x2_dgrad(const uint16_t* dy, int32_t dy_cs, int32_t dy_co, const uint16_t* w4t, const uint16_t* x,
                            int32_t x_cs, int32_t x_co, uint16_t* dx, int32_t dx_cs, int32_t dx_co,
                            int32_t accumulate, int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout,
                            uint32_t* err, void* stream) {
  US_CHECK(dy && w4t && x && dx && err && B > 0 && H > 0 && W > 0);
  US_CHECK(Cout % 8 == 0 && pick_bn(Cin) && dy_cs % 8 == 0 && dy_co % 8 == 0 && x_cs % 8 == 0 && x_co % 8 == 0);
  US_CHECK(dx_cs % 8 == 0 && dx_co % 8 == 0 && aligned16(dy) && aligned16(w4t) && aligned16(x) && aligned16(dx));
  const int M = B * H * W, K = 4 * Cout, bn = pick_bn(Cin);
  ConvTDgradLoader ld{{(const bf16*)dy, dy_cs, dy_co}, (const bf16*)w4t, {B, H, W}, Cout, K, Cin, M, bn};
  MaskedGradStore ep{{(bf16*)dx, dx_cs, dx_co}, {(const bf16*)x, x_cs, x_co}, accumulate};
  return to_status(gemm_bn(bn, ld, ep, M, Cin, K, err, (cudaStream_t)stream));
}

us_status us_convT2x2_wgrad(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* dy, int32_t dy_cs,
                            int32_t dy_co, float* g4, int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout,
                            uint32_t* err, void* stream) {
  US_CHECK(x && dy && g4 && err && B > 0 && H > 0 && W > 0);
  US_CHECK(Cout % 8 == 0 && pick_bn(Cin) && x_cs % 8 == 0 && x_co % 8 == 0 && dy_cs % 8 == 0 && dy_co % 8 == 0);
  US_CHECK(aligned16(x) && aligned16(dy));
  const int rows = 4 * Cout, P = B * H * W, bn = pick_bn(Cin);
  WgradLoader<ConvTGather, PixelRows> ld{{{(const bf16*)dy, dy_cs, dy_co}, {B, H, W}, Cout, rows},
                                         {{(const bf16*)x, x_cs, x_co}, Cin}, P, bn};
  AtomicF32Store ep{g4, Cin, rows};
  const int mt = (rows + kBM - 1) / kBM, nt = Cin / bn;
  return to_status(gemm_bn(bn, ld, ep, rows, Cin, P, err, (cudaStream_t)stream, wgrad_splits(mt, nt, P)));
}

}  // extern "C"
