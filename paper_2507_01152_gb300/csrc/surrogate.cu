// The learned surrogate: a convolutional encoder-decoder with skip
// connections (the kind of network SonoGym's learning-based simulator uses,
// Sec. 4 and App. B.2), trained on frames the physics path renders.
//
// Layers (c = base channels, level l has c 2^l channels, 4 levels):
//   enc0a conv(8 -> c), enc0b conv(c -> c)                          -> e0
//   down_l conv stride 2, enc_l a/b conv                            -> e_l
//   up_l convT2x2 into the first half of cat_l = [up_l, e_l],
//   dec_l a conv(2 c_l -> c_l), dec_l b conv(c_l -> c_l)            (l = 2, 1, 0)
//   head 1x1 conv (c -> 1) + sigmoid
// every conv / convT followed by ReLU.  e_l is written straight into the
// second half of cat_l, so concatenation costs nothing; its gradient is
// accumulated there by both consumers.
// Loss per frame: L1 + (1 - SSIM) (Wang et al. 2004: 11 x 11 Gaussian,
// sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, valid region); batch mean.  Adam.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "surr_internal.h"
#include "ussim_surrogate.h"

namespace ussim {
namespace surr {

using bf16 = __nv_bfloat16;
constexpr int kInCh = 8;
constexpr int kLevels = 4;
constexpr int kWin = 11;
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;

struct LayerDesc {
  int kind;            // 0 conv3x3, 1 convT2x2, 2 head
  int cin, cout, stride;
  long long w_off, b_off, w_size;   // into the flat parameter vector
  int hin, win;        // input spatial size
};

// ------------------------------------------------------------------ kernels

// out[p] = sigmoid(sum_c f[p][c] w[c] + b); a pixel's channels are read
// as 16-byte vectors (C a multiple of 8, rows 16-byte aligned).  Each group
// of 8 channels is summed in channel order, then b and the group sums in
// group order (the fused head of the last convolution sums the same way).
__global__ void head_fwd(const bf16* f, int C, const float* w, const float* b, float* out, long long P) {
  __shared__ float sw[256];
  for (int i = threadIdx.x; i < C; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint4* fp = reinterpret_cast<const uint4*>(f + p * C);
  float z = b[0];
  for (int c8 = 0; c8 < C / 8; ++c8) {
    const uint4 q = __ldg(fp + c8);
    const bf16* h = reinterpret_cast<const bf16*>(&q);
    float zg = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) zg = fmaf(__bfloat162float(h[i]), sw[c8 * 8 + i], zg);
    z += zg;
  }
  out[p] = 1.f / (1.f + expf(-z));
}

// through the sigmoid and the head: dz = dout * y (1 - y); df = dz w [f > 0];
// gw[c] += sum dz f[c]; gb += sum dz
__global__ void head_bwd(const bf16* f, int C, const float* w, const float* y, const float* dout, bf16* df,
                         float* gw, float* gb, long long P) {
  __shared__ float sw[256 + 1];
  for (int i = threadIdx.x; i <= C; i += blockDim.x) sw[i] = 0.f;
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < P) {
    const float yy = y[p];
    const float dz = dout[p] * yy * (1.f - yy);
    const bf16* fp = f + p * C;
    bf16* dp = df + p * C;
    for (int c = 0; c < C; ++c) {
      const float fv = __bfloat162float(fp[c]);
      dp[c] = __float2bfloat16_rn(fv > 0.f ? dz * w[c] : 0.f);
      atomicAdd(&sw[c], dz * fv);
    }
    atomicAdd(&sw[C], dz);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(&gw[i], sw[i]);
  if (threadIdx.x == 0) atomicAdd(gb, sw[C]);
}

// gb[c] += sum over pixels of g[p][co + c] (channel stride cs), C <= 256
__global__ void bias_grad(const bf16* g, int cs, int co, int C, long long P, int pix_per_block, float* gb) {
  __shared__ float acc[256];
  for (int i = threadIdx.x; i < C; i += blockDim.x) acc[i] = 0.f;
  __syncthreads();
  const int lanes = blockDim.x / C;          // threads per channel
  const int c = threadIdx.x % C, j = threadIdx.x / C;
  if (j < lanes) {
    float s = 0.f;
    const long long p0 = (long long)blockIdx.x * pix_per_block;
    const long long p1 = min(P, p0 + pix_per_block);
    for (long long p = p0 + j; p < p1; p += lanes) s += __bfloat162float(g[p * cs + co + c]);
    atomicAdd(&acc[c], s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(&gb[i], acc[i]);
}

// normalised 11-tap Gaussian (sigma 1.5), set from FP64 on the host
__constant__ float c_gauss[kWin];
__device__ __forceinline__ float gauss_w(int k) { return c_gauss[k]; }

// deterministic per-frame sums: every block of a (chunk, frame) grid
// reduces its values in a fixed order into partial[frame][chunk]
constexpr int kRedThreads = 256;
__device__ __forceinline__ void block_sum_to(float* partial, float v) {
  __shared__ float red[kRedThreads];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = kRedThreads / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// horizontal Gaussian pass of (x, y, x^2, y^2, x y): out [B][5][H][W-10]
__global__ void ssim_hpass(const float* x, const float* y, float* out, int B, int H, int W) {
  const int Wv = W - kWin + 1;
  const long long n = (long long)B * H * Wv;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % Wv);
  const long long rowi = i / Wv;                 // b * H + r
  const int b = (int)(rowi / H), r = (int)(rowi % H);
  float s[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k < kWin; ++k) {
    const float w = gauss_w(k);
    const long long q = rowi * W + c + k;
    const float a = x[q], t = y[q];
    s[0] += w * a;
    s[1] += w * t;
    s[2] += w * a * a;
    s[3] += w * t * t;
    s[4] += w * a * t;
  }
  const long long plane = (long long)H * Wv;
  for (int q = 0; q < 5; ++q) out[((long long)b * 5 + q) * plane + (long long)r * Wv + c] = s[q];
}

// vertical pass -> statistics at valid pixels, SSIM map, and the three maps
// of its derivative: A' = dS/dmux - 2 dS/dsxx mux - dS/dsxy muy, Bm = dS/dsxx,
// Cm = dS/dsxy; per-block SSIM partial sums.  maps: [B][3][Hv][Wv].
// grid (chunks of the valid region, frames)
__global__ void ssim_vpass(const float* h, float* maps, float* ssim_part, int H, int W) {
  const int Wv = W - kWin + 1, Hv = H - kWin + 1;
  const int b = blockIdx.y;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float S = 0.f;
  if (i < (long long)Hv * Wv) {
    const int c = (int)(i % Wv), r = (int)(i / Wv);
    const long long plane = (long long)H * Wv;
    float s[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < kWin; ++k) {
      const float w = gauss_w(k);
      for (int q = 0; q < 5; ++q) s[q] += w * h[((long long)b * 5 + q) * plane + (long long)(r + k) * Wv + c];
    }
    const float mx = s[0], my = s[1];
    const float sxx = s[2] - mx * mx, syy = s[3] - my * my, sxy = s[4] - mx * my;
    const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
    const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
    const float D = d1 * d2;
    S = n1 * n2 / D;
    const float dmux = 2.f * my * n2 / D - 2.f * mx * S / d1;
    const float dsxx = -S / d2;
    const float dsxy = 2.f * n1 / D;
    const long long vp = (long long)Hv * Wv, o = (long long)r * Wv + c;
    maps[((long long)b * 3 + 0) * vp + o] = dmux - 2.f * dsxx * mx - dsxy * my;
    maps[((long long)b * 3 + 1) * vp + o] = dsxx;
    maps[((long long)b * 3 + 2) * vp + o] = dsxy;
  }
  block_sum_to(ssim_part, S);
}

// full correlation of the three valid-region maps with the window, then
// d loss / d pred (if dx); per-block |x - y| partial sums.
// loss = (1/B) sum_b [ mean|x - y| + 1 - mean S ].  grid (chunks of the frame, frames)
__global__ void ssim_grad(const float* maps, const float* x, const float* y, float* dx, float* l1_part, int B, int H,
                          int W) {
  const int Wv = W - kWin + 1, Hv = H - kWin + 1;
  const int b = blockIdx.y;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float ad = 0.f;
  if (j < (long long)H * W) {
    const int c = (int)(j % W), r = (int)(j / W);
    const long long i = (long long)b * H * W + j;
    const long long vp = (long long)Hv * Wv;
    float g[3] = {0, 0, 0};
    for (int ky = 0; ky < kWin; ++ky) {
      const int pr = r - ky;
      if (pr < 0 || pr >= Hv) continue;
      const float wy = gauss_w(ky);
      for (int kx = 0; kx < kWin; ++kx) {
        const int pc = c - kx;
        if (pc < 0 || pc >= Wv) continue;
        const float w = wy * gauss_w(kx);
        const long long o = (long long)pr * Wv + pc;
        for (int q = 0; q < 3; ++q) g[q] += w * maps[((long long)b * 3 + q) * vp + o];
      }
    }
    const float xv = x[i], yv = y[i];
    const float dS = g[0] + 2.f * xv * g[1] + yv * g[2];
    const float d = xv - yv;
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    if (dx) dx[i] = (sgn / (float)(H * W) - dS / (float)vp) / (float)B;
    ad = fabsf(d);
  }
  block_sum_to(l1_part, ad);
}

// loss out: [0] batch loss, [1 + b] frame L1, [1 + B + b] frame SSIM;
// partial sums added in a fixed order
__global__ void loss_finish(const float* l1_part, int n_l1, const float* ss_part, int n_ss, float* out, int B, int H,
                            int W) {
  const int Hv = H - kWin + 1, Wv = W - kWin + 1;
  float tot = 0.f;
  for (int b = 0; b < B; ++b) {
    float l1 = 0.f, ss = 0.f;
    for (int k = 0; k < n_l1; ++k) l1 += l1_part[(size_t)b * n_l1 + k];
    for (int k = 0; k < n_ss; ++k) ss += ss_part[(size_t)b * n_ss + k];
    l1 /= (float)(H * W);
    ss /= (float)(Hv * Wv);
    out[1 + b] = l1;
    out[1 + B + b] = ss;
    tot += l1 + 1.f - ss;
  }
  out[0] = tot / (float)B;
}

// Adam on the flat FP32 parameters.  Conv weight gradients arrive in the
// [9 Cin][Cout] layout of the weight-gradient GEMM (seg_kind 1).
struct Seg {
  long long off, size;
  int kind, cin, cout;
};

__global__ void adam_kernel(float* p, float* m, float* v, const float* g, const Seg* segs, int nseg, long long n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = 0;
  while (s + 1 < nseg && segs[s + 1].off <= i) ++s;
  const Seg sg = segs[s];
  long long gi = i;
  if (sg.kind == 1) {   // p layout [co][tap][ci] ; g layout [tap][ci][co]
    const long long j = i - sg.off;
    const long long K9 = 9LL * sg.cin;
    const long long co = j / K9, r = j - co * K9;
    gi = sg.off + r * sg.cout + co;
  }
  const float gg = g[gi];
  const float mm = b1 * m[i] + (1.f - b1) * gg;
  const float vv = b2 * v[i] + (1.f - b2) * gg * gg;
  m[i] = mm;
  v[i] = vv;
  p[i] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// BF16 copies of a layer's weights: forward layout (same as FP32) and the
// input-gradient layout (conv: [ci][tap][co]; convT: [ci][4 Cout])
__global__ void relayout_conv(const float* w, bf16* wf, bf16* wd, int cin, int cout) {
  const long long n = 9LL * cin * cout;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ci = (int)(i % cin);
  const long long t = i / cin;
  const int tap = (int)(t % 9), co = (int)(t / 9);
  const bf16 v = __float2bfloat16_rn(w[i]);
  wf[i] = v;
  wd[((long long)ci * 9 + tap) * cout + co] = v;
}
__global__ void relayout_convT(const float* w, bf16* wf, bf16* wt, int cin, int cout4) {
  const long long n = (long long)cin * cout4;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ci = (int)(i % cin), r = (int)(i / cin);
  const bf16 v = __float2bfloat16_rn(w[i]);
  wf[i] = v;
  wt[(long long)ci * cout4 + r] = v;
}

// per-frame features for the error head: channel means of the bottleneck
// activation, feat[b][c] = mean over pixels of x[b][p][c].  One block of
// 1024 threads per frame: thread t sums channel t mod C over the pixels
// p = t / C (mod 1024 / C) with four accumulators, then the groups'
// partial sums are added in a fixed order (deterministic).  C <= 1024;
// threads past the last whole group of C only join the barrier.
__global__ void __launch_bounds__(1024) pool_features(const bf16* x, int P, int C, float* feat) {
  __shared__ float part[1024];
  const int b = blockIdx.x, t = threadIdx.x, c = t % C, grp = t / C, ngrp = 1024 / C;
  if (grp < ngrp) {
    const bf16* xb = x + (size_t)b * P * C + c;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int p = grp;
    for (; p + 3 * ngrp < P; p += 4 * ngrp) {
      s0 += __bfloat162float(xb[(size_t)p * C]);
      s1 += __bfloat162float(xb[(size_t)(p + ngrp) * C]);
      s2 += __bfloat162float(xb[(size_t)(p + 2 * ngrp) * C]);
      s3 += __bfloat162float(xb[(size_t)(p + 3 * ngrp) * C]);
    }
    for (; p < P; p += ngrp) s0 += __bfloat162float(xb[(size_t)p * C]);
    part[t] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
  if (grp == 0) {
    float s = 0.f;
    for (int g = 0; g < ngrp; ++g) s += part[g * C + c];
    feat[(size_t)b * C + c] = s / (float)P;
  }
}

// predicted per-frame L1 gap: w . feat + bias
__global__ void error_head(const float* feat, const float* w, int F, int B, float* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = w[F];
  for (int f = 0; f < F; ++f) s = fmaf(w[f], feat[(size_t)b * F + f], s);
  out[b] = s;
}

// gradient in the flat parameter layout (conv segments transposed back)
__global__ void grads_to_param_layout(const float* g, float* out, const Seg* segs, int nseg, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = 0;
  while (s + 1 < nseg && segs[s + 1].off <= i) ++s;
  const Seg sg = segs[s];
  long long gi = i;
  if (sg.kind == 1) {
    const long long j = i - sg.off, K9 = 9LL * sg.cin, co = j / K9, r = j - co * K9;
    gi = sg.off + r * sg.cout + co;
  }
  out[i] = g[gi];
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------ GAN term
// discriminator input: the 8 channels of the slice, the frame (BF16), 7 zeros
__global__ void disc_input(const bf16* x, const float* y, bf16* out, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint4 xv = reinterpret_cast<const uint4*>(x)[p];
  __align__(16) bf16 o[8];
  o[0] = __float2bfloat16_rn(y[p]);
#pragma unroll
  for (int k = 1; k < 8; ++k) o[k] = __float2bfloat16_rn(0.f);
  reinterpret_cast<uint4*>(out)[2 * p] = xv;
  reinterpret_cast<uint4*>(out)[2 * p + 1] = *reinterpret_cast<const uint4*>(o);
}

// patch logits z[p] = sum_c f[p][c] w[c] + b
__global__ void disc_head_fwd(const bf16* f, int C, const float* w, const float* b, float* z, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const bf16* fp = f + p * C;
  float acc = b[0];
  for (int c = 0; c < C; ++c) acc = fmaf(__bfloat162float(fp[c]), w[c], acc);
  z[p] = acc;
}

// BCE of logits against a constant target t: per block, the fixed-order sum
// of log(1 + e^z) - t z into partial[block]; dz[p] = scale (s(z) - t)
__global__ void bce_logits_kernel(const float* z, float t, float scale, float* dz, float* partial, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (p < P) {
    const float v = z[p];
    // log(1 + e^v) without overflow: max(v, 0) + log1p(e^-|v|)
    l = fmaxf(v, 0.f) + log1pf(expf(-fabsf(v))) - t * v;
    dz[p] = scale * (1.f / (1.f + expf(-v)) - t);
  }
  block_sum_to(partial, l);
}

// out[0] (+)= weight * (sum of the partials) / P, in order
__global__ void bce_finish(const float* partial, int n, long long P, float weight, int accumulate, float* out) {
  float s = 0.f;
  for (int k = 0; k < n; ++k) s += partial[k];
  const float v = weight * s / (float)P;
  out[0] = accumulate ? out[0] + v : v;
}

// through the head: df = dz w [f > 0]; gw[c] += sum dz f[c], gb += sum dz
// (gw, gb may be null: no parameter gradients)
__global__ void disc_head_bwd(const bf16* f, int C, const float* w, const float* dz, bf16* df, float* gw, float* gb,
                              long long P) {
  __shared__ float sw[256 + 1];
  for (int i = threadIdx.x; i <= C; i += blockDim.x) sw[i] = 0.f;
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < P) {
    const float d = dz[p];
    const bf16* fp = f + p * C;
    bf16* dp = df + p * C;
    for (int c = 0; c < C; ++c) {
      const float fv = __bfloat162float(fp[c]);
      dp[c] = __float2bfloat16_rn(fv > 0.f ? d * w[c] : 0.f);
      if (gw) atomicAdd(&sw[c], d * fv);
    }
    if (gb) atomicAdd(&sw[C], d);
  }
  __syncthreads();
  if (gw)
    for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(&gw[i], sw[i]);
  if (gb && threadIdx.x == 0) atomicAdd(gb, sw[C]);
}

// dout[p] += g[p * cs + ch]: the frame channel of the discriminator's input
// gradient, added to the generator's output gradient
__global__ void add_channel(const bf16* g, int cs, int ch, float* dout, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < P) dout[p] += __bfloat162float(g[p * cs + ch]);
}

__global__ void fill_bf16(bf16* p, float v, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = __float2bfloat16_rn(v);
}

}  // namespace surr
}  // namespace ussim

using namespace ussim;
using namespace ussim::surr;

struct us_surr {
  us_surr_config cfg{};
  std::vector<LayerDesc> layers;
  std::vector<Seg> segs;
  long long n_params = 0;
  int step = 0;
  // parameters and optimiser state (FP32)
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *g_host_layout = nullptr;
  Seg* d_segs = nullptr;
  // BF16 weights: forward and input-gradient layouts, per layer
  std::vector<bf16*> wf, wd;
  // activations / gradients (BF16 NHWC), per named buffer
  struct Buf {
    bf16* a = nullptr;
    bf16* g = nullptr;
    int C = 0, H = 0, W = 0;
  };
  std::vector<Buf> bufs;
  float *out = nullptr, *dout = nullptr, *sh = nullptr, *smaps = nullptr, *l1s = nullptr, *sss = nullptr;
  float *feat = nullptr, *ehead = nullptr;   // bottleneck features of the last forward, error-head weights
  unsigned* err = nullptr;
  std::string last_error;
  // GAN term (App. B.2: L1 and GAN terms, weights 1 and 0.01): the patch
  // discriminator's parameters, optimiser state, BF16 weights and buffers
  int gan_cd = 0;
  float gan_weight = 0.f, gan_lr = 0.f;
  int gan_step = 0;
  std::vector<LayerDesc> dlayers;   // d1, d2, d3 (conv3x3 stride 2), head
  std::vector<Seg> dsegs;
  long long dn = 0;
  float *dp = nullptr, *dm = nullptr, *dv = nullptr, *dg = nullptr, *dg_host = nullptr;
  Seg* d_dsegs = nullptr;
  bf16 *dwf[3] = {}, *dwd[3] = {};
  bf16 *din = nullptr, *din_g = nullptr, *dones = nullptr;
  bf16 *dact[3] = {}, *dgr[3] = {};
  float *dlogit = nullptr, *ddz = nullptr, *dpart = nullptr;
};

namespace {

// buffer ids
enum {
  B_IN, B_A0, B_CAT0, B_D1, B_A1, B_CAT1, B_D2, B_A2, B_CAT2, B_D3, B_A3, B_E3, B_X2A, B_X2, B_X1A, B_X1, B_X0A, B_X0,
  B_COUNT
};

void build_layers(us_surr* s) {
  const int c = s->cfg.base_channels;
  int ch[kLevels];
  for (int l = 0; l < kLevels; ++l) ch[l] = c << l;
  const int H = s->cfg.height, W = s->cfg.width;
  auto add = [&](int kind, int cin, int cout, int stride, int hin, int win) {
    LayerDesc d{kind, cin, cout, stride, 0, 0, 0, hin, win};
    d.w_size = kind == 0 ? 9LL * cin * cout : (kind == 1 ? 4LL * cout * cin : cin);
    d.w_off = s->n_params;
    d.b_off = d.w_off + d.w_size;
    s->n_params = d.b_off + cout;
    s->layers.push_back(d);
    s->segs.push_back(Seg{d.w_off, d.w_size, kind == 0 ? 1 : 0, cin, cout});
    s->segs.push_back(Seg{d.b_off, cout, 0, 0, 0});
  };
  add(0, kInCh, ch[0], 1, H, W);                         // enc0a
  add(0, ch[0], ch[0], 1, H, W);                         // enc0b
  for (int l = 1; l < kLevels; ++l) {
    const int h = H >> l, w = W >> l;
    add(0, ch[l - 1], ch[l], 2, h * 2, w * 2);           // down_l
    add(0, ch[l], ch[l], 1, h, w);                       // enc_l a
    add(0, ch[l], ch[l], 1, h, w);                       // enc_l b
  }
  for (int l = kLevels - 2; l >= 0; --l) {
    const int h = H >> l, w = W >> l;
    add(1, ch[l + 1], ch[l], 2, h / 2, w / 2);           // up_l
    add(0, 2 * ch[l], ch[l], 1, h, w);                   // dec_l a
    add(0, ch[l], ch[l], 1, h, w);                       // dec_l b
  }
  add(2, ch[0], 1, 1, H, W);                             // head
}

us_status fail(us_surr* s, us_status st, const std::string& msg) {
  if (s) s->last_error = msg;
  return st;
}

us_status cfail(us_surr* s, cudaError_t e, const char* where) {
  if (s) s->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? US_ERR_OOM : US_ERR_CUDA;
}

us_status refresh_weights(us_surr* s, cudaStream_t st) {
  for (size_t i = 0; i < s->layers.size(); ++i) {
    const LayerDesc& d = s->layers[i];
    if (d.kind == 0)
      relayout_conv<<<blocks(d.w_size), 256, 0, st>>>(s->p + d.w_off, s->wf[i], s->wd[i], d.cin, d.cout);
    else if (d.kind == 1)
      relayout_convT<<<blocks(d.w_size), 256, 0, st>>>(s->p + d.w_off, s->wf[i], s->wd[i], d.cin, 4 * d.cout);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "weight relayout");
}

void free_surr(us_surr* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  cudaFree(s->p);
  cudaFree(s->m);
  cudaFree(s->v);
  cudaFree(s->g);
  cudaFree(s->g_host_layout);
  cudaFree(s->d_segs);
  for (auto* q : s->wf) cudaFree(q);
  for (auto* q : s->wd) cudaFree(q);
  for (auto& b : s->bufs) {
    cudaFree(b.a);
    cudaFree(b.g);
  }
  cudaFree(s->out);
  cudaFree(s->dout);
  cudaFree(s->sh);
  cudaFree(s->smaps);
  cudaFree(s->l1s);
  cudaFree(s->sss);
  cudaFree(s->feat);
  cudaFree(s->ehead);
  cudaFree(s->err);
  cudaFree(s->dp);
  cudaFree(s->dm);
  cudaFree(s->dv);
  cudaFree(s->dg);
  cudaFree(s->dg_host);
  cudaFree(s->d_dsegs);
  for (int i = 0; i < 3; ++i) {
    cudaFree(s->dwf[i]);
    cudaFree(s->dwd[i]);
    cudaFree(s->dact[i]);
    cudaFree(s->dgr[i]);
  }
  cudaFree(s->din);
  cudaFree(s->din_g);
  cudaFree(s->dones);
  cudaFree(s->dlogit);
  cudaFree(s->ddz);
  cudaFree(s->dpart);
  delete s;
}

const uint16_t* A(const us_surr* s, int id) { return reinterpret_cast<const uint16_t*>(s->bufs[id].a); }
uint16_t* Aw(us_surr* s, int id) { return reinterpret_cast<uint16_t*>(s->bufs[id].a); }
uint16_t* G(us_surr* s, int id) { return reinterpret_cast<uint16_t*>(s->bufs[id].g); }
const uint16_t* Wf(const us_surr* s, int l) { return reinterpret_cast<const uint16_t*>(s->wf[l]); }
const uint16_t* Wd(const us_surr* s, int l) { return reinterpret_cast<const uint16_t*>(s->wd[l]); }

#define TRY(x)                        \
  do {                                \
    us_status _r = (x);               \
    if (_r != US_OK) return _r;       \
  } while (0)

// layer index -> (input buffer, input channel offset, output buffer, output channel offset)
struct Wiring {
  int in, in_co, out, out_co;
};

std::vector<Wiring> wiring(const us_surr* s) {
  const int c = s->cfg.base_channels;
  return {
      {B_IN, 0, B_A0, 0},              // enc0a
      {B_A0, 0, B_CAT0, c},            // enc0b -> e0 = cat0[c:2c]
      {B_CAT0, c, B_D1, 0},            // down1
      {B_D1, 0, B_A1, 0},              // enc1a
      {B_A1, 0, B_CAT1, 2 * c},        // enc1b -> e1 = cat1[2c:4c]
      {B_CAT1, 2 * c, B_D2, 0},        // down2
      {B_D2, 0, B_A2, 0},              // enc2a
      {B_A2, 0, B_CAT2, 4 * c},        // enc2b -> e2 = cat2[4c:8c]
      {B_CAT2, 4 * c, B_D3, 0},        // down3
      {B_D3, 0, B_A3, 0},              // enc3a
      {B_A3, 0, B_E3, 0},              // enc3b -> e3
      {B_E3, 0, B_CAT2, 0},            // up2 -> cat2[0:4c]
      {B_CAT2, 0, B_X2A, 0},           // dec2a
      {B_X2A, 0, B_X2, 0},             // dec2b
      {B_X2, 0, B_CAT1, 0},            // up1 -> cat1[0:2c]
      {B_CAT1, 0, B_X1A, 0},           // dec1a
      {B_X1A, 0, B_X1, 0},             // dec1b
      {B_X1, 0, B_CAT0, 0},            // up0 -> cat0[0:c]
      {B_CAT0, 0, B_X0A, 0},           // dec0a
      {B_X0A, 0, B_X0, 0},             // dec0b
      {B_X0, 0, -1, 0},                // head
  };
}

// keep_act: store the last convolution's activation (the backward pass
// reads it); without it the head may be fused into that convolution
us_status forward_impl(us_surr* s, int B, cudaStream_t st, bool keep_act = true) {
  const auto wr = wiring(s);
  const LayerDesc& hd = s->layers.back();
  bool head_done = false;
  for (size_t i = 0; i + 1 < s->layers.size(); ++i) {
    const LayerDesc& d = s->layers[i];
    const auto& bi = s->bufs[wr[i].in];
    const auto& bo = s->bufs[wr[i].out];
    us_status r;
    if (i + 2 == s->layers.size() && d.kind == 0 && d.stride == 1 && d.cout == 32 && hd.cin == 32) {
      cudaError_t e = cudaSuccess;
      if (surr::conv3x3_head_fwd(e, A(s, wr[i].in), bi.C, wr[i].in_co, d.cin, Wf(s, (int)i), s->p + d.b_off,
                                 keep_act ? Aw(s, wr[i].out) : nullptr, bo.C, wr[i].out_co, B, d.hin, d.win,
                                 s->p + hd.w_off, s->p + hd.b_off, s->out, s->err, st)) {
        if (e != cudaSuccess) return cfail(s, e, "last convolution with the head");
        head_done = true;
        continue;
      }
    }
    if (d.kind == 0)
      r = us_conv3x3_fwd(A(s, wr[i].in), bi.C, wr[i].in_co, Wf(s, (int)i), s->p + d.b_off, Aw(s, wr[i].out), bo.C,
                         wr[i].out_co, B, d.hin, d.win, d.cin, d.cout, d.stride, 1, s->err, st);
    else
      r = us_convT2x2_fwd(A(s, wr[i].in), bi.C, wr[i].in_co, Wf(s, (int)i), s->p + d.b_off, Aw(s, wr[i].out), bo.C,
                          wr[i].out_co, B, d.hin, d.win, d.cin, d.cout, 1, s->err, st);
    if (r != US_OK) return fail(s, r, "forward layer " + std::to_string(i));
  }
  const long long P = (long long)B * s->cfg.height * s->cfg.width;
  if (!head_done)
    head_fwd<<<blocks(P), 256, 0, st>>>(s->bufs[B_X0].a, hd.cin, s->p + hd.w_off, s->p + hd.b_off, s->out, P);
  const auto& e3 = s->bufs[B_E3];
  pool_features<<<B, 1024, 0, st>>>(e3.a, e3.H * e3.W, e3.C, s->feat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "head");
}

us_status backward_impl(us_surr* s, int B, cudaStream_t st) {
  const auto wr = wiring(s);
  const LayerDesc& hd = s->layers.back();
  const long long P = (long long)B * s->cfg.height * s->cfg.width;
  cudaError_t e = cudaMemsetAsync(s->g, 0, sizeof(float) * s->n_params, st);
  if (e != cudaSuccess) return cfail(s, e, "zero grads");
  head_bwd<<<blocks(P), 256, 0, st>>>(s->bufs[B_X0].a, hd.cin, s->p + hd.w_off, s->out, s->dout, s->bufs[B_X0].g,
                                      s->g + hd.w_off, s->g + hd.b_off, P);
  for (int i = (int)s->layers.size() - 2; i >= 0; --i) {
    const LayerDesc& d = s->layers[i];
    const auto& bi = s->bufs[wr[i].in];
    const auto& bo = s->bufs[wr[i].out];
    const int Ho = d.kind == 1 ? 2 * d.hin : (d.hin - 1) / d.stride + 1;
    const int Wo = d.kind == 1 ? 2 * d.win : (d.win - 1) / d.stride + 1;
    const long long Pout = (long long)B * Ho * Wo;
    // gradient at this layer's output lives in the output buffer's gradient slice
    const uint16_t* dy = G(s, wr[i].out);
    const int dy_cs = bo.C, dy_co = wr[i].out_co;
    const int ppb = 4096;
    bias_grad<<<blocks(Pout, ppb), 256, 0, st>>>(s->bufs[wr[i].out].g, dy_cs, dy_co, d.cout, Pout, ppb,
                                                 s->g + d.b_off);
    us_status r;
    if (d.kind == 0) {
      r = us_conv3x3_wgrad(A(s, wr[i].in), bi.C, wr[i].in_co, dy, dy_cs, dy_co, s->g + d.w_off, B, d.hin, d.win, d.cin,
                           d.cout, d.stride, s->err, st);
      if (r == US_OK && i > 0) {
        // e_l (second half of cat_l) gets its decoder gradient first, so the
        // down-sampling layer that also reads it accumulates
        const bool acc = (wr[i].in == B_CAT0 || wr[i].in == B_CAT1 || wr[i].in == B_CAT2) && wr[i].in_co > 0;
        r = us_conv3x3_dgrad(dy, dy_cs, dy_co, Wd(s, i), A(s, wr[i].in), bi.C, wr[i].in_co, G(s, wr[i].in), bi.C,
                             wr[i].in_co, acc ? 1 : 0, B, d.hin, d.win, d.cin, d.cout, d.stride, s->err, st);
      }
    } else {
      r = us_convT2x2_wgrad(A(s, wr[i].in), bi.C, wr[i].in_co, dy, dy_cs, dy_co, s->g + d.w_off, B, d.hin, d.win, d.cin,
                            d.cout, s->err, st);
      if (r == US_OK)
        r = us_convT2x2_dgrad(dy, dy_cs, dy_co, Wd(s, i), A(s, wr[i].in), bi.C, wr[i].in_co, G(s, wr[i].in), bi.C,
                              wr[i].in_co, 0, B, d.hin, d.win, d.cin, d.cout, s->err, st);
    }
    if (r != US_OK) return fail(s, r, "backward layer " + std::to_string(i));
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "backward");
}

// ---------------------------------------------------------- GAN term
constexpr int kDiscIn = 16;   // discriminator input channels: slice 8, frame 1, zeros 7

void build_disc(us_surr* s, int cd) {
  s->dlayers.clear();
  s->dsegs.clear();
  s->dn = 0;
  const int H = s->cfg.height, W = s->cfg.width;
  const int cin[3] = {kDiscIn, cd, 2 * cd}, cout[3] = {cd, 2 * cd, 2 * cd};
  for (int i = 0; i < 4; ++i) {
    LayerDesc d{};
    d.kind = i < 3 ? 0 : 2;
    d.cin = i < 3 ? cin[i] : 2 * cd;
    d.cout = i < 3 ? cout[i] : 1;
    d.stride = i < 3 ? 2 : 1;
    d.hin = H >> i;
    d.win = W >> i;
    d.w_size = d.kind == 0 ? 9LL * d.cin * d.cout : d.cin;
    d.w_off = s->dn;
    d.b_off = d.w_off + d.w_size;
    s->dn = d.b_off + d.cout;
    s->dlayers.push_back(d);
    s->dsegs.push_back(Seg{d.w_off, d.w_size, d.kind == 0 ? 1 : 0, d.cin, d.cout});
    s->dsegs.push_back(Seg{d.b_off, d.cout, 0, 0, 0});
  }
}

us_status refresh_disc_weights(us_surr* s, cudaStream_t st) {
  for (int i = 0; i < 3; ++i) {
    const LayerDesc& d = s->dlayers[i];
    relayout_conv<<<blocks(d.w_size), 256, 0, st>>>(s->dp + d.w_off, s->dwf[i], s->dwd[i], d.cin, d.cout);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "discriminator weight relayout");
}

// discriminator forward on (slice x, frame y): logits of the B frames' patches
us_status disc_forward(us_surr* s, const bf16* x, const float* y, int B, cudaStream_t st) {
  const int H = s->cfg.height, W = s->cfg.width;
  const long long P = (long long)B * H * W;
  disc_input<<<blocks(P), 256, 0, st>>>(x, y, s->din, P);
  const bf16* in = s->din;
  int in_c = kDiscIn;
  for (int i = 0; i < 3; ++i) {
    const LayerDesc& d = s->dlayers[i];
    const us_status r = us_conv3x3_fwd(reinterpret_cast<const uint16_t*>(in), in_c, 0,
                                       reinterpret_cast<const uint16_t*>(s->dwf[i]), s->dp + d.b_off,
                                       reinterpret_cast<uint16_t*>(s->dact[i]), d.cout, 0, B, d.hin, d.win, d.cin,
                                       d.cout, 2, 1, s->err, st);
    if (r != US_OK) return fail(s, r, "discriminator layer " + std::to_string(i));
    in = s->dact[i];
    in_c = d.cout;
  }
  const LayerDesc& hd = s->dlayers[3];
  const long long Pd = (long long)B * (H >> 3) * (W >> 3);
  disc_head_fwd<<<blocks(Pd), 256, 0, st>>>(s->dact[2], hd.cin, s->dp + hd.w_off, s->dp + hd.b_off, s->dlogit, Pd);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "discriminator forward");
}

// BCE of the last logits against t: out[0] (+)= weight * mean; dz = scale (s(z) - t)
us_status disc_bce(us_surr* s, int B, float t, float weight, float scale, int accumulate, float* out,
                   cudaStream_t st) {
  const long long Pd = (long long)B * (s->cfg.height >> 3) * (s->cfg.width >> 3);
  const unsigned nb = blocks(Pd, kRedThreads);
  bce_logits_kernel<<<nb, kRedThreads, 0, st>>>(s->dlogit, t, scale, s->ddz, s->dpart, Pd);
  bce_finish<<<1, 1, 0, st>>>(s->dpart, (int)nb, Pd, weight, accumulate, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "discriminator loss");
}

// from dz back through the discriminator: with_params adds the parameter
// gradients to dg; with_input leaves the gradient of its input in din_g
us_status disc_backward(us_surr* s, int B, bool with_params, bool with_input, cudaStream_t st) {
  const int H = s->cfg.height, W = s->cfg.width;
  const LayerDesc& hd = s->dlayers[3];
  const long long Pd = (long long)B * (H >> 3) * (W >> 3);
  disc_head_bwd<<<blocks(Pd), 256, 0, st>>>(s->dact[2], hd.cin, s->dp + hd.w_off, s->ddz, s->dgr[2],
                                            with_params ? s->dg + hd.w_off : nullptr,
                                            with_params ? s->dg + hd.b_off : nullptr, Pd);
  for (int i = 2; i >= 0; --i) {
    const LayerDesc& d = s->dlayers[i];
    const long long Pout = (long long)B * (d.hin / 2) * (d.win / 2);
    const uint16_t* dy = reinterpret_cast<const uint16_t*>(s->dgr[i]);
    const bf16* xin = i > 0 ? s->dact[i - 1] : s->din;
    us_status r = US_OK;
    if (with_params) {
      bias_grad<<<blocks(Pout, 4096), 256, 0, st>>>(s->dgr[i], d.cout, 0, d.cout, Pout, 4096, s->dg + d.b_off);
      r = us_conv3x3_wgrad(reinterpret_cast<const uint16_t*>(xin), d.cin, 0, dy, d.cout, 0, s->dg + d.w_off, B, d.hin,
                           d.win, d.cin, d.cout, 2, s->err, st);
    }
    if (r == US_OK && (i > 0 || with_input)) {
      // inner layers: the input is a post-ReLU activation (its mask applies);
      // the first layer's input is not, so its gradient is taken through an
      // all-ones mask
      const bf16* mask = i > 0 ? xin : s->dones;
      bf16* dx = i > 0 ? s->dgr[i - 1] : s->din_g;
      r = us_conv3x3_dgrad(dy, d.cout, 0, reinterpret_cast<const uint16_t*>(s->dwd[i]),
                           reinterpret_cast<const uint16_t*>(mask), d.cin, 0, reinterpret_cast<uint16_t*>(dx), d.cin,
                           0, 0, B, d.hin, d.win, d.cin, d.cout, 2, s->err, st);
    }
    if (r != US_OK) return fail(s, r, "discriminator backward layer " + std::to_string(i));
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "discriminator backward");
}

// the generator's GAN term: loss_out[0] += w BCE(D(x, pred), 1) and
// dout += d/dpred of it (the discriminator held fixed)
us_status gan_generator_term(us_surr* s, const bf16* x, int B, float* loss_out, cudaStream_t st) {
  const long long Pd = (long long)B * (s->cfg.height >> 3) * (s->cfg.width >> 3);
  TRY(disc_forward(s, x, s->out, B, st));
  TRY(disc_bce(s, B, 1.f, s->gan_weight, s->gan_weight / (float)Pd, 1, loss_out, st));
  TRY(disc_backward(s, B, false, true, st));
  const long long P = (long long)B * s->cfg.height * s->cfg.width;
  add_channel<<<blocks(P), 256, 0, st>>>(s->din_g, kDiscIn, kInCh, s->dout, P);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "GAN term");
}

us_status loss_impl(us_surr* s, const float* pred, const float* target, int B, float* loss_out, float* dpred,
                    cudaStream_t st, int H = 0, int W = 0) {
  if (H == 0) H = s->cfg.height;
  if (W == 0) W = s->cfg.width;
  const int n_ss = (int)blocks((long long)(H - kWin + 1) * (W - kWin + 1), kRedThreads);
  const int n_l1 = (int)blocks((long long)H * W, kRedThreads);
  ssim_hpass<<<blocks((long long)B * H * (W - kWin + 1)), 256, 0, st>>>(pred, target, s->sh, B, H, W);
  ssim_vpass<<<dim3(n_ss, B), kRedThreads, 0, st>>>(s->sh, s->smaps, s->sss, H, W);
  ssim_grad<<<dim3(n_l1, B), kRedThreads, 0, st>>>(s->smaps, pred, target, dpred, s->l1s, B, H, W);
  loss_finish<<<1, 1, 0, st>>>(s->l1s, n_l1, s->sss, n_ss, loss_out, B, H, W);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "loss");
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

uint32_t crc32(const void* data, size_t n, uint32_t crc = 0) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= b[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

}  // namespace

extern "C" {

int32_t us_surr_param_segments(const us_surr_config* cfg, int32_t max_segs, int64_t* offsets, int64_t* sizes,
                               int32_t* fan_in) {
  if (!cfg || cfg->base_channels < 16 || cfg->base_channels % 16) return -1;
  us_surr tmp;
  tmp.cfg = *cfg;
  build_layers(&tmp);
  const int n = (int)tmp.segs.size();
  if (offsets && sizes && fan_in) {
    if (max_segs < n) return -1;
    for (int i = 0; i < n; ++i) {
      const LayerDesc& d = tmp.layers[i / 2];
      offsets[i] = tmp.segs[i].off;
      sizes[i] = tmp.segs[i].size;
      fan_in[i] = (i & 1) ? 0 : (d.kind == 0 ? 9 * d.cin : d.cin);
    }
  }
  return n;
}

int64_t us_surr_num_params(const us_surr_config* cfg) {
  if (!cfg || cfg->base_channels < 16 || cfg->base_channels % 16) return -1;
  us_surr tmp;
  tmp.cfg = *cfg;
  build_layers(&tmp);
  return tmp.n_params;
}

us_status us_surr_create(const us_surr_config* cfg, const float* init_params, us_surr** out) {
  if (!out) return US_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || !init_params) return US_ERR_INVALID_ARG;
  const int c = cfg->base_channels, H = cfg->height, W = cfg->width;
  if (c < 16 || c > 64 || c % 16 || H < 16 || W < 16 || H % 8 || W % 8 || cfg->max_batch < 1 ||
      !(cfg->lr > 0) || !(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) || !(cfg->eps > 0))
    return US_ERR_INVALID_ARG;
  us_surr* s = new us_surr();
  s->cfg = *cfg;
  build_layers(s);
  {
    float gw[kWin];
    double tot = 0, w64[kWin];
    for (int k = 0; k < kWin; ++k) {
      const double d = k - kWin / 2;
      w64[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
      tot += w64[k];
    }
    for (int k = 0; k < kWin; ++k) gw[k] = (float)(w64[k] / tot);
    if (cudaMemcpyToSymbol(c_gauss, gw, sizeof gw) != cudaSuccess) {
      delete s;
      return US_ERR_CUDA;
    }
  }
  const int Bm = cfg->max_batch;
  cudaError_t e;
  auto falloc = [&](float** p, long long n) { return cudaMalloc(p, sizeof(float) * (size_t)std::max(1LL, n)); };
  if ((e = falloc(&s->p, s->n_params)) != cudaSuccess || (e = falloc(&s->m, s->n_params)) != cudaSuccess ||
      (e = falloc(&s->v, s->n_params)) != cudaSuccess || (e = falloc(&s->g, s->n_params)) != cudaSuccess ||
      (e = falloc(&s->g_host_layout, s->n_params)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_segs, sizeof(Seg) * s->segs.size())) != cudaSuccess ||
      (e = cudaMalloc(&s->err, sizeof(unsigned))) != cudaSuccess) {
    free_surr(s);
    return US_ERR_OOM;
  }
  cudaMemcpy(s->p, init_params, sizeof(float) * s->n_params, cudaMemcpyHostToDevice);
  cudaMemset(s->m, 0, sizeof(float) * s->n_params);
  cudaMemset(s->v, 0, sizeof(float) * s->n_params);
  cudaMemset(s->err, 0, sizeof(unsigned));
  cudaMemcpy(s->d_segs, s->segs.data(), sizeof(Seg) * s->segs.size(), cudaMemcpyHostToDevice);
  for (const LayerDesc& d : s->layers) {
    bf16 *a = nullptr, *b = nullptr;
    if (d.kind != 2) {
      if ((e = cudaMalloc(&a, sizeof(bf16) * d.w_size)) != cudaSuccess || (e = cudaMalloc(&b, sizeof(bf16) * d.w_size)) != cudaSuccess) {
        cudaFree(a);
        free_surr(s);
        return US_ERR_OOM;
      }
    }
    s->wf.push_back(a);
    s->wd.push_back(b);
  }
  // activation buffers: channels and spatial size per id
  s->bufs.resize(B_COUNT);
  auto setb = [&](int id, int C, int lvl) {
    s->bufs[id].C = C;
    s->bufs[id].H = H >> lvl;
    s->bufs[id].W = W >> lvl;
  };
  setb(B_IN, kInCh, 0);
  setb(B_A0, c, 0);
  setb(B_CAT0, 2 * c, 0);
  setb(B_D1, 2 * c, 1);
  setb(B_A1, 2 * c, 1);
  setb(B_CAT1, 4 * c, 1);
  setb(B_D2, 4 * c, 2);
  setb(B_A2, 4 * c, 2);
  setb(B_CAT2, 8 * c, 2);
  setb(B_D3, 8 * c, 3);
  setb(B_A3, 8 * c, 3);
  setb(B_E3, 8 * c, 3);
  setb(B_X2A, 4 * c, 2);
  setb(B_X2, 4 * c, 2);
  setb(B_X1A, 2 * c, 1);
  setb(B_X1, 2 * c, 1);
  setb(B_X0A, c, 0);
  setb(B_X0, c, 0);
  for (int id = 0; id < B_COUNT; ++id) {
    auto& b = s->bufs[id];
    const size_t n = (size_t)Bm * b.H * b.W * b.C;
    if (id == B_IN) continue;   // the caller's input, read in place; no gradient needed
    if ((e = cudaMalloc(&b.a, n * sizeof(bf16))) != cudaSuccess) {
      free_surr(s);
      return US_ERR_OOM;
    }
    if ((e = cudaMalloc(&b.g, n * sizeof(bf16))) != cudaSuccess) {
      free_surr(s);
      return US_ERR_OOM;
    }
  }
  const size_t P = (size_t)Bm * H * W;
  if ((e = cudaMalloc(&s->out, P * 4)) != cudaSuccess || (e = cudaMalloc(&s->dout, P * 4)) != cudaSuccess ||
      (e = cudaMalloc(&s->sh, (size_t)Bm * 5 * H * (W - kWin + 1) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&s->smaps, (size_t)Bm * 3 * (H - kWin + 1) * (W - kWin + 1) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&s->feat, (size_t)Bm * 8 * c * 4)) != cudaSuccess ||
      (e = cudaMalloc(&s->ehead, (size_t)(8 * c + 1) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&s->l1s, (size_t)Bm * 4 * blocks((long long)H * W))) != cudaSuccess ||
      (e = cudaMalloc(&s->sss, (size_t)Bm * 4 * blocks((long long)(H - kWin + 1) * (W - kWin + 1)))) != cudaSuccess) {
    free_surr(s);
    return US_ERR_OOM;
  }
  cudaMemset(s->ehead, 0, (size_t)(8 * c + 1) * 4);
  if (refresh_weights(s, 0) != US_OK || cudaDeviceSynchronize() != cudaSuccess) {
    free_surr(s);
    return US_ERR_CUDA;
  }
  *out = s;
  return US_OK;
}

void us_surr_destroy(us_surr* s) { free_surr(s); }

const char* us_surr_last_error(const us_surr* s) { return s ? s->last_error.c_str() : "NULL handle"; }

us_status us_surr_forward(us_surr* s, const uint16_t* x, float* y, int32_t B, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!x || !y || B < 1 || B > s->cfg.max_batch || !aligned16(x)) return fail(s, US_ERR_INVALID_ARG, "bad forward arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s->bufs[B_IN].a = const_cast<bf16*>(reinterpret_cast<const bf16*>(x));
  TRY(forward_impl(s, B, st, false));
  const size_t P = (size_t)B * s->cfg.height * s->cfg.width;
  cudaError_t e = cudaMemcpyAsync(y, s->out, P * 4, cudaMemcpyDeviceToDevice, st);
  s->bufs[B_IN].a = nullptr;
  return e == cudaSuccess ? US_OK : cfail(s, e, "copy out");
}

us_status us_surr_train_step(us_surr* s, const uint16_t* x, const float* target, int32_t B, float* loss_out,
                             int32_t update, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!x || !target || !loss_out || B < 1 || B > s->cfg.max_batch || !aligned16(x))
    return fail(s, US_ERR_INVALID_ARG, "bad train-step arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s->bufs[B_IN].a = const_cast<bf16*>(reinterpret_cast<const bf16*>(x));
  us_status r = forward_impl(s, B, st);
  if (r == US_OK) r = loss_impl(s, s->out, target, B, loss_out, s->dout, st);
  if (r == US_OK && s->gan_weight > 0.f) r = gan_generator_term(s, reinterpret_cast<const bf16*>(x), B, loss_out, st);
  if (r == US_OK) r = backward_impl(s, B, st);
  s->bufs[B_IN].a = nullptr;
  if (r != US_OK) return r;
  if (update) {
    s->step += 1;
    const float c1 = 1.f - std::pow(s->cfg.beta1, (float)s->step), c2 = 1.f - std::pow(s->cfg.beta2, (float)s->step);
    adam_kernel<<<blocks(s->n_params), 256, 0, st>>>(s->p, s->m, s->v, s->g, s->d_segs, (int)s->segs.size(),
                                                     s->n_params, s->cfg.lr, s->cfg.beta1, s->cfg.beta2, s->cfg.eps, c1,
                                                     c2);
    TRY(refresh_weights(s, st));
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "train step");
}

us_status us_surr_metrics(us_surr* s, const float* pred, const float* target, int32_t B, float* out, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!pred || !target || !out || B < 1 || B > s->cfg.max_batch) return fail(s, US_ERR_INVALID_ARG, "bad metrics arguments");
  return loss_impl(s, pred, target, B, out, nullptr, static_cast<cudaStream_t>(stream));
}

us_status us_surr_metrics_hw(us_surr* s, const float* pred, const float* target, int32_t B, int32_t H, int32_t W,
                             float* out, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!pred || !target || !out || B < 1 || B > s->cfg.max_batch || H < kWin || W < kWin || H > s->cfg.height ||
      W > s->cfg.width)
    return fail(s, US_ERR_INVALID_ARG, "bad metrics arguments");
  return loss_impl(s, pred, target, B, out, nullptr, static_cast<cudaStream_t>(stream), H, W);
}

int32_t us_surr_num_features(const us_surr* s) { return s ? 8 * s->cfg.base_channels : -1; }

us_status us_surr_features(us_surr* s, int32_t B, float* out, void* stream) {
  if (!s || !out || B < 1 || B > s->cfg.max_batch) return US_ERR_INVALID_ARG;
  const cudaError_t e = cudaMemcpyAsync(out, s->feat, (size_t)B * 8 * s->cfg.base_channels * 4, cudaMemcpyDeviceToDevice,
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? US_OK : cfail(s, e, "features");
}

us_status us_surr_predict_error(us_surr* s, int32_t B, float* out, void* stream) {
  if (!s || !out || B < 1 || B > s->cfg.max_batch) return US_ERR_INVALID_ARG;
  error_head<<<blocks(B), 256, 0, static_cast<cudaStream_t>(stream)>>>(s->feat, s->ehead, 8 * s->cfg.base_channels, B, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "error head");
}

// Ridge least squares for the error head: minimise sum (w.f + b - y)^2 +
// ridge |w|^2 over n (feature, true L1) pairs given on the host, by the
// normal equations (Cholesky, FP64).
us_status us_surr_fit_error_head(us_surr* s, const float* feat, const float* target, int32_t n, float ridge) {
  if (!s || !feat || !target || n < 2 || !(ridge >= 0)) return US_ERR_INVALID_ARG;
  const int F = 8 * s->cfg.base_channels, D = F + 1;
  std::vector<double> A((size_t)D * D, 0.0), rhs(D, 0.0), w(D, 0.0);
  std::vector<double> x(D);
  for (int i = 0; i < n; ++i) {
    for (int f = 0; f < F; ++f) x[f] = feat[(size_t)i * F + f];
    x[F] = 1.0;
    for (int a = 0; a < D; ++a) {
      rhs[a] += x[a] * target[i];
      for (int b = 0; b <= a; ++b) A[(size_t)a * D + b] += x[a] * x[b];
    }
  }
  for (int a = 0; a < F; ++a) A[(size_t)a * D + a] += ridge;
  A[(size_t)F * D + F] += 1e-9;
  // Cholesky A = L L^T (lower triangle in place)
  for (int j = 0; j < D; ++j) {
    double d = A[(size_t)j * D + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * D + k] * A[(size_t)j * D + k];
    if (!(d > 0)) return fail(s, US_ERR_INVALID_ARG, "error-head normal equations are singular");
    d = std::sqrt(d);
    A[(size_t)j * D + j] = d;
    for (int i = j + 1; i < D; ++i) {
      double v = A[(size_t)i * D + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * D + k] * A[(size_t)j * D + k];
      A[(size_t)i * D + j] = v / d;
    }
  }
  std::vector<double> y(D);
  for (int i = 0; i < D; ++i) {
    double v = rhs[i];
    for (int k = 0; k < i; ++k) v -= A[(size_t)i * D + k] * y[k];
    y[i] = v / A[(size_t)i * D + i];
  }
  for (int i = D - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < D; ++k) v -= A[(size_t)k * D + i] * w[k];
    w[i] = v / A[(size_t)i * D + i];
  }
  std::vector<float> wf(D);
  for (int i = 0; i < D; ++i) wf[i] = (float)w[i];
  return cudaMemcpy(s->ehead, wf.data(), (size_t)D * 4, cudaMemcpyHostToDevice) == cudaSuccess ? US_OK : US_ERR_CUDA;
}

us_status us_surr_get_params(const us_surr* s, float* host_out) {
  if (!s || !host_out) return US_ERR_INVALID_ARG;
  return cudaMemcpy(host_out, s->p, sizeof(float) * s->n_params, cudaMemcpyDeviceToHost) == cudaSuccess ? US_OK
                                                                                                          : US_ERR_CUDA;
}

int64_t us_surr_gan_num_params(int32_t cd) {
  if (cd < 16 || cd > 128 || cd % 16) return -1;
  us_surr tmp;
  tmp.cfg.height = tmp.cfg.width = 64;
  build_disc(&tmp, cd);
  return tmp.dn;
}

us_status us_surr_gan_enable(us_surr* s, int32_t cd, const float* init, float gan_weight, float lr) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!init || cd < 16 || cd > 128 || cd % 16 || !(gan_weight >= 0.f) || !(lr > 0.f) || s->gan_cd)
    return fail(s, US_ERR_INVALID_ARG, "bad GAN arguments (or the GAN term is already enabled)");
  build_disc(s, cd);
  const int H = s->cfg.height, W = s->cfg.width, Bm = s->cfg.max_batch;
  const long long P = (long long)Bm * H * W;
  cudaError_t e = cudaSuccess;
  auto fa = [&](float** p, long long n) {
    if (e == cudaSuccess) e = cudaMalloc(p, sizeof(float) * (size_t)std::max(1LL, n));
  };
  auto ba = [&](bf16** p, long long n) {
    if (e == cudaSuccess) e = cudaMalloc(p, sizeof(bf16) * (size_t)std::max(1LL, n));
  };
  fa(&s->dp, s->dn);
  fa(&s->dm, s->dn);
  fa(&s->dv, s->dn);
  fa(&s->dg, s->dn);
  fa(&s->dg_host, s->dn);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_dsegs, sizeof(Seg) * s->dsegs.size());
  for (int i = 0; i < 3; ++i) {
    const LayerDesc& d = s->dlayers[i];
    ba(&s->dwf[i], d.w_size);
    ba(&s->dwd[i], d.w_size);
    ba(&s->dact[i], (long long)Bm * (d.hin / 2) * (d.win / 2) * d.cout);
    ba(&s->dgr[i], (long long)Bm * (d.hin / 2) * (d.win / 2) * d.cout);
  }
  ba(&s->din, P * kDiscIn);
  ba(&s->din_g, P * kDiscIn);
  ba(&s->dones, P * kDiscIn);
  const long long Pd = (long long)Bm * (H >> 3) * (W >> 3);
  fa(&s->dlogit, Pd);
  fa(&s->ddz, Pd);
  fa(&s->dpart, (long long)blocks(Pd, kRedThreads));
  if (e == cudaSuccess) e = cudaMemcpy(s->dp, init, sizeof(float) * s->dn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->dm, 0, sizeof(float) * s->dn);
  if (e == cudaSuccess) e = cudaMemset(s->dv, 0, sizeof(float) * s->dn);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_dsegs, s->dsegs.data(), sizeof(Seg) * s->dsegs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fill_bf16<<<blocks(P * kDiscIn), 256>>>(s->dones, 1.f, P * kDiscIn);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cfail(s, e, "GAN buffers");
  s->gan_cd = cd;
  s->gan_weight = gan_weight;
  s->gan_lr = lr;
  TRY(refresh_disc_weights(s, nullptr));
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? US_OK : cfail(s, e, "GAN set-up");
}

us_status us_surr_gan_disc_step(us_surr* s, const uint16_t* x, const float* real, int32_t B, float* loss_out,
                                int32_t update, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!s->gan_cd) return fail(s, US_ERR_INVALID_ARG, "the GAN term is not enabled");
  if (!x || !real || !loss_out || B < 1 || B > s->cfg.max_batch || !aligned16(x))
    return fail(s, US_ERR_INVALID_ARG, "bad discriminator-step arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long Pd = (long long)B * (s->cfg.height >> 3) * (s->cfg.width >> 3);
  const bf16* xb = reinterpret_cast<const bf16*>(x);
  cudaError_t e = cudaMemsetAsync(s->dg, 0, sizeof(float) * s->dn, st);
  if (e != cudaSuccess) return cfail(s, e, "zero discriminator grads");
  // (BCE(D(x, real), 1) + BCE(D(x, fake), 0)) / 2, the fake frames being the
  // last forward's output; loss_out [3]: the loss, its real and fake terms
  TRY(disc_forward(s, xb, real, B, st));
  TRY(disc_bce(s, B, 1.f, 1.f, 0.5f / (float)Pd, 0, loss_out + 1, st));
  TRY(disc_backward(s, B, true, false, st));
  TRY(disc_forward(s, xb, s->out, B, st));
  TRY(disc_bce(s, B, 0.f, 1.f, 0.5f / (float)Pd, 0, loss_out + 2, st));
  TRY(disc_backward(s, B, true, false, st));
  bce_finish<<<1, 1, 0, st>>>(loss_out + 1, 2, 2, 1.f, 0, loss_out);
  if (update) {
    s->gan_step += 1;
    const float c1 = 1.f - std::pow(s->cfg.beta1, (float)s->gan_step), c2 = 1.f - std::pow(s->cfg.beta2, (float)s->gan_step);
    adam_kernel<<<blocks(s->dn), 256, 0, st>>>(s->dp, s->dm, s->dv, s->dg, s->d_dsegs, (int)s->dsegs.size(), s->dn,
                                               s->gan_lr, s->cfg.beta1, s->cfg.beta2, s->cfg.eps, c1, c2);
    TRY(refresh_disc_weights(s, st));
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? US_OK : cfail(s, e, "discriminator step");
}

us_status us_surr_gan_get(us_surr* s, float* params_host, float* grads_host) {
  if (!s || !s->gan_cd) return US_ERR_INVALID_ARG;
  if (params_host && cudaMemcpy(params_host, s->dp, sizeof(float) * s->dn, cudaMemcpyDeviceToHost) != cudaSuccess)
    return US_ERR_CUDA;
  if (grads_host) {
    grads_to_param_layout<<<blocks(s->dn), 256>>>(s->dg, s->dg_host, s->d_dsegs, (int)s->dsegs.size(), s->dn);
    if (cudaMemcpy(grads_host, s->dg_host, sizeof(float) * s->dn, cudaMemcpyDeviceToHost) != cudaSuccess)
      return US_ERR_CUDA;
  }
  return US_OK;
}

us_status us_surr_get_grads(us_surr* s, float* host_out) {
  if (!s || !host_out) return US_ERR_INVALID_ARG;
  grads_to_param_layout<<<blocks(s->n_params), 256>>>(s->g, s->g_host_layout, s->d_segs, (int)s->segs.size(),
                                                      s->n_params);
  return cudaMemcpy(host_out, s->g_host_layout, sizeof(float) * s->n_params, cudaMemcpyDeviceToHost) == cudaSuccess
             ? US_OK
             : US_ERR_CUDA;
}

us_status us_surr_check(us_surr* s, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return US_ERR_CUDA;
  unsigned w = 0;
  if (cudaMemcpy(&w, s->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return US_ERR_CUDA;
  if (w) {
    cudaMemset(s->err, 0, 4);
    return fail(s, US_ERR_TIMEOUT, "a tensor-core wait ran out");
  }
  return US_OK;
}

// checkpoint: magic, version, config, step, n_params, params, m, v, CRC32
us_status us_surr_save(const us_surr* s, const char* path) {
  if (!s || !path) return US_ERR_INVALID_ARG;
  const size_t n = (size_t)s->n_params;
  std::vector<float> buf(3 * n);
  if (cudaMemcpy(buf.data(), s->p, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + n, s->m, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * n, s->v, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return US_ERR_CUDA;
  FILE* f = std::fopen(path, "wb");
  if (!f) return US_ERR_INVALID_ARG;
  const char magic[8] = {'U', 'S', 'S', 'U', 'R', 'R', '0', '1'};
  const int64_t np = s->n_params;
  const int32_t step = s->step;
  uint32_t crc = crc32(&s->cfg, sizeof s->cfg);
  crc = crc32(&step, sizeof step, crc);
  crc = crc32(buf.data(), buf.size() * 4, crc);
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&s->cfg, sizeof s->cfg, 1, f) == 1 &&
            std::fwrite(&step, 4, 1, f) == 1 && std::fwrite(&np, 8, 1, f) == 1 &&
            std::fwrite(buf.data(), 4, buf.size(), f) == buf.size() && std::fwrite(&crc, 4, 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? US_OK : US_ERR_INTERNAL;
}

us_status us_surr_load(us_surr* s, const char* path) {
  if (!s || !path) return US_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(s, US_ERR_INVALID_ARG, "cannot open checkpoint");
  char magic[8];
  us_surr_config cfg;
  int32_t step;
  int64_t np;
  const size_t n = (size_t)s->n_params;
  std::vector<float> buf(3 * n);
  uint32_t crc_file = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "USSURR01", 8) == 0 &&
            std::fread(&cfg, sizeof cfg, 1, f) == 1 && std::fread(&step, 4, 1, f) == 1 &&
            std::fread(&np, 8, 1, f) == 1 && np == s->n_params && std::fread(buf.data(), 4, buf.size(), f) == buf.size() &&
            std::fread(&crc_file, 4, 1, f) == 1;
  std::fclose(f);
  if (!ok) return fail(s, US_ERR_INVALID_ARG, "checkpoint does not match this network");
  uint32_t crc = crc32(&cfg, sizeof cfg);
  crc = crc32(&step, sizeof step, crc);
  crc = crc32(buf.data(), buf.size() * 4, crc);
  if (crc != crc_file) return fail(s, US_ERR_INVALID_ARG, "checkpoint CRC mismatch");
  if (cfg.base_channels != s->cfg.base_channels) return fail(s, US_ERR_INVALID_ARG, "checkpoint of another network");
  if (cudaMemcpy(s->p, buf.data(), n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->m, buf.data() + n, n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->v, buf.data() + 2 * n, n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return US_ERR_CUDA;
  s->step = step;
  TRY(refresh_weights(s, 0));
  return cudaDeviceSynchronize() == cudaSuccess ? US_OK : US_ERR_CUDA;
}

}  // extern "C"
