/*
 * ussim_surrogate.h — C ABI of the learned surrogate of the ultrasound
 * render and of the tensor-core operators it is built from.
 *
 * SonoGym's learning-based simulator translates CT slices to ultrasound
 * images with a pix2pix U-Net (Sec. 4 "Ultrasound simulation"; App. B.2
 * "Learning-based approach", Fig. U-Net).  Here the network is a
 * convolutional encoder-decoder that maps the label/HU slice sampled on the
 * output grid to the physics frame, trained on frames the physics path
 * renders; BF16 operands, FP32 accumulation in tensor memory (tcgen05).
 *
 * Conventions as in ussim.h: DEVICE pointers, caller-owned, asynchronous on
 * `stream` (a cudaStream_t as void*), status codes, no traps.  BF16 tensors
 * are passed as uint16_t* (raw bfloat16 bits).
 */
#ifndef USSIM_SURROGATE_H
#define USSIM_SURROGATE_H

#include <stdint.h>

#include "ussim.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C[M][N] (FP32) = A[M][K] (BF16, row-major) * B[N][K]^T (BF16, row-major)
 * on the tcgen05 tile kernel (128 x N tiles, FP32 accumulation in TMEM).
 * The building block of the surrogate's implicit-GEMM convolutions; the
 * paper has no counterpart (it is a plain dense contraction).
 * N multiple of 32, K multiple of 8, pointers 16-byte aligned.
 * err: DEVICE uint32 word; bit 4 is set if a bounded tensor-core wait ran
 * out (then C is not written). */
US_API us_status us_gemm_bf16_nt(const uint16_t* A, const uint16_t* B, float* C, int32_t M, int32_t N, int32_t K,
                                 uint32_t* err, void* stream);

/* ---- convolution operators (implicit GEMM on tcgen05) -----------------
 * Tensors are NHWC BF16 views: base pointer, channel stride (elements per
 * pixel, multiple of 8) and channel offset (multiple of 8), so an operator
 * can read or write a channel slice of a concatenated tensor.  Channel
 * counts are multiples of 8 (Cout of the forward ops a multiple of 32 /
 * 16 for convT).  All pointers 16-byte aligned.  `err` as above.
 * The paper's U-Net (App. B.2, Fig. U-Net) is built from such layers:
 * 3x3 convolutions (stride 1, or 2 to downsample, zero padding 1) and
 * 2x2 stride-2 transposed convolutions to upsample. */

/* y[b,yo,xo,co] = act(bias[co] + sum_{ky,kx,ci} x[b, yo*s-1+ky, xo*s-1+kx, ci] w[co][ky][kx][ci]);
 * input B x H x W x Cin, output B x ceil(H/s) x ceil(W/s) x Cout; act = ReLU if relu. */
US_API us_status us_conv3x3_fwd(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* w, const float* bias,
                                uint16_t* y, int32_t y_cs, int32_t y_co, int32_t B, int32_t H, int32_t W,
                                int32_t Cin, int32_t Cout, int32_t stride, int32_t relu, uint32_t* err, void* stream);

/* gradient w.r.t. the input of a 3x3 convolution whose input x is a
 * post-ReLU activation: dx = [x > 0] * sum_{ky,kx,co} dy[b,(yi+1-ky)/s,(xi+1-kx)/s,co] w[co][ky][kx][ci]
 * (terms with a non-integer quotient drop out); wd[ci][ky][kx][co] =
 * w[co][ky][kx][ci].  accumulate = 1 adds to the values already in dx. */
US_API us_status us_conv3x3_dgrad(const uint16_t* dy, int32_t dy_cs, int32_t dy_co, const uint16_t* wd,
                                  const uint16_t* x, int32_t x_cs, int32_t x_co, uint16_t* dx, int32_t dx_cs,
                                  int32_t dx_co, int32_t accumulate, int32_t B, int32_t H, int32_t W, int32_t Cin,
                                  int32_t Cout, int32_t stride, uint32_t* err, void* stream);

/* weight gradient, accumulated: gwt[(ky,kx,ci)][co] += sum_{b,yo,xo} x[b, yo*s-1+ky, xo*s-1+kx, ci] dy[b,yo,xo,co]
 * (FP32, [9 Cin][Cout], the transpose of the weight layout). */
US_API us_status us_conv3x3_wgrad(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* dy, int32_t dy_cs,
                                  int32_t dy_co, float* gwt, int32_t B, int32_t H, int32_t W, int32_t Cin,
                                  int32_t Cout, int32_t stride, uint32_t* err, void* stream);

/* y[b, 2y+dy, 2x+dx, co] = act(bias[co] + sum_ci x[b,y,x,ci] w4[(2 dy + dx) Cout + co][ci]);
 * input B x H x W x Cin, output B x 2H x 2W x Cout. */
US_API us_status us_convT2x2_fwd(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* w4, const float* bias,
                                 uint16_t* y, int32_t y_cs, int32_t y_co, int32_t B, int32_t H, int32_t W,
                                 int32_t Cin, int32_t Cout, int32_t relu, uint32_t* err, void* stream);

/* dx = [x > 0] * sum_{dy,dx,co} dy[b, 2y+dy, 2x+dx, co] w4[(2 dy + dx) Cout + co][ci];
 * w4t[ci][(d, co)] = w4[(d, co)][ci]; x is the (post-ReLU) input, B x H x W x Cin. */
US_API us_status us_convT2x2_dgrad(const uint16_t* dy, int32_t dy_cs, int32_t dy_co, const uint16_t* w4t,
                                   const uint16_t* x, int32_t x_cs, int32_t x_co, uint16_t* dx, int32_t dx_cs,
                                   int32_t dx_co, int32_t accumulate, int32_t B, int32_t H, int32_t W, int32_t Cin,
                                   int32_t Cout, uint32_t* err, void* stream);

/* g4[(d, co)][ci] += sum_{b,y,x} dy[b, 2y+dy, 2x+dx, co] x[b,y,x,ci]  (FP32, [4 Cout][Cin]) */
US_API us_status us_convT2x2_wgrad(const uint16_t* x, int32_t x_cs, int32_t x_co, const uint16_t* dy, int32_t dy_cs,
                                   int32_t dy_co, float* g4, int32_t B, int32_t H, int32_t W, int32_t Cin,
                                   int32_t Cout, uint32_t* err, void* stream);

/* ---- the surrogate network ---------------------------------------------
 * Encoder-decoder with skip connections (a U-Net as in App. B.2's
 * learning-based simulator; the figure giving its exact widths is not in
 * the text, this layer list is the library's reading):
 *   level l = 0..3 has c 2^l channels (c = base_channels);
 *   enc0: conv3x3(8 -> c), conv3x3(c -> c) -> e0;
 *   enc l: conv3x3 stride 2 (c_{l-1} -> c_l), conv3x3, conv3x3 -> e_l;
 *   dec l = 2..0: convT2x2(c_{l+1} -> c_l), concat [up, e_l],
 *                 conv3x3(2 c_l -> c_l), conv3x3(c_l -> c_l);
 *   head: 1x1 conv (c -> 1) + sigmoid; every conv / convT followed by ReLU.
 * Input: [B][H][W][8] BF16 (channels: label / 4, clamp(HU / 1000, -1, 3),
 * inside-fan mask, 5 zeros).  Output: [B][H][W] FP32 in (0, 1), the
 * log-compressed frame.  Loss per frame L1 + (1 - SSIM) (Wang et al. 2004,
 * 11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, valid
 * region), batch mean; the paper's pix2pix training uses the L1 term.
 * Adam (Kingma & Ba) on FP32 master weights; BF16 copies feed the tensor
 * cores.  Parameter vector (FP32): per layer in the order above, weights
 * ([Cout][3][3][Cin], convT [(2 dy + dx) Cout + co][Cin], head [c]) then
 * bias. */
typedef struct {
  int32_t base_channels;  /* c: 16, 32, 48 or 64 */
  int32_t height, width;  /* multiples of 8, >= 16 */
  int32_t max_batch;      /* activations are allocated for this many frames */
  float lr, beta1, beta2, eps;
} us_surr_config;

typedef struct us_surr us_surr;

/* parameter segments in order (each layer: weights, then bias): offset,
 * size and fan-in (0 for biases), so that a caller can draw the initial
 * parameters.  Returns the number of segments (-1 on a bad config or if
 * max_segs is too small); NULL arrays just return the count.  Host only. */
US_API int32_t us_surr_param_segments(const us_surr_config* cfg, int32_t max_segs, int64_t* offsets,
                                      int64_t* sizes, int32_t* fan_in);
/* number of FP32 parameters of the network, or -1 for a bad config */
US_API int64_t us_surr_num_params(const us_surr_config* cfg);
/* Create the network of the layer list above (App. B.2, learning-based
 * approach: the U-Net the paper trains on CT-US pairs).  init_params: HOST,
 * us_surr_num_params floats (copied); the handle owns its weights, Adam
 * moments and activations for max_batch frames.  Errors: US_ERR_INVALID_ARG
 * (bad config, NULL), US_ERR_OOM, US_ERR_CUDA. */
US_API us_status us_surr_create(const us_surr_config* cfg, const float* init_params, us_surr** out);
US_API void us_surr_destroy(us_surr* s);
US_API const char* us_surr_last_error(const us_surr* s);
/* Forward pass (App. B.2: the learned simulator maps the CT / label slice
 * to the ultrasound image): y[B][H][W] = net(x); x [B][H][W][8] BF16, y FP32,
 * DEVICE, caller-owned; 1 <= B <= max_batch.  Keeps the activations of this
 * call for us_surr_features / us_surr_predict_error.  Errors:
 * US_ERR_INVALID_ARG, US_ERR_CUDA; a bounded tensor-core wait that runs out
 * is reported by us_surr_check. */
US_API us_status us_surr_forward(us_surr* s, const uint16_t* x, float* y, int32_t B, void* stream);
/* One training step on (x, target) (App. B.2: the network is trained on
 * paired slices and images with an L1 term; here the images are the
 * physics renders): forward, loss, backward, and (update = 1) an Adam
 * update.  x as us_surr_forward; target DEVICE [B][H][W] FP32.  loss_out:
 * DEVICE [1 + 2B]: batch loss, per-frame L1, per-frame SSIM (before the
 * update).  Errors as us_surr_forward. */
US_API us_status us_surr_train_step(us_surr* s, const uint16_t* x, const float* target, int32_t B, float* loss_out,
                                    int32_t update, void* stream);
/* per-frame L1 and SSIM of any prediction (the quality the paper reports
 * for its learned simulator includes SSIM, Sec. 5): pred, target DEVICE
 * [B][H][W]; out DEVICE [1 + 2B] as above.  Errors: US_ERR_INVALID_ARG. */
US_API us_status us_surr_metrics(us_surr* s, const float* pred, const float* target, int32_t B, float* out,
                                 void* stream);
/* The same per-frame L1 and SSIM for B frames of an explicit H x W
 * (11 <= H <= height, 11 <= W <= width of the network's config, B <=
 * max_batch): quality of frames of other probe sizes against physics.
 * Errors: US_ERR_INVALID_ARG. */
US_API us_status us_surr_metrics_hw(us_surr* s, const float* pred, const float* target, int32_t B, int32_t H,
                                    int32_t W, float* out, void* stream);
/* ---- error gate ----------------------------------------------------------
 * The physics render is the surrogate's judge and fallback: a linear error
 * head on the surrogate's bottleneck features (channel means of the
 * deepest activation, 8 c values per frame) predicts each frame's L1 gap
 * to physics; frames predicted above a threshold are re-rendered by
 * physics (us_sim_render_gated).  The head is fitted by ridge regression
 * on (features, true L1) pairs that physics provides. */
US_API int32_t us_surr_num_features(const us_surr* s);
/* features of the frames of the last us_surr_forward: DEVICE [B][8 c] */
US_API us_status us_surr_features(us_surr* s, int32_t B, float* out, void* stream);
/* predicted L1 gap of the frames of the last forward: DEVICE [B] */
US_API us_status us_surr_predict_error(us_surr* s, int32_t B, float* out, void* stream);
/* fit the head: feat HOST [n][8 c], target HOST [n] (true per-frame L1),
 * ridge >= 0; minimises sum_i (w . feat_i + w0 - target_i)^2 + ridge |w|^2
 * (intercept w0 not penalised) through the FP64 normal equations and a
 * Cholesky solve; synchronous.  The paper has no counterpart (its learned
 * simulator has no error gate).  Errors: US_ERR_INVALID_ARG (n < 2, NULL,
 * ridge < 0, singular system), US_ERR_CUDA. */
US_API us_status us_surr_fit_error_head(us_surr* s, const float* feat, const float* target, int32_t n, float ridge);

/* ---- GAN term -----------------------------------------------------------
 * App. B.2 trains the learned simulator with an L1 term and a GAN term,
 * weights 1 and 0.01.  The discriminator (the library's reading of
 * pix2pix's patch classifier) sees the input slice and a frame as 16
 * channels (the 8 slice channels, the frame, 7 zeros) through three 3x3
 * stride-2 convolutions with ReLU (16 -> cd -> 2 cd -> 2 cd) and a 1x1 head
 * to one logit per 8 x 8 patch; BCE on logits averaged over every patch.
 * Parameters (FP32, this order): d1 w [cd][3][3][16], d1 b [cd], d2 w
 * [2cd][3][3][cd], d2 b, d3 w [2cd][3][3][2cd], d3 b, head w [2cd], head b [1].
 * With the term enabled, us_surr_train_step minimises
 *   L1 + (1 - SSIM) + gan_weight * BCE(D(x, G(x)), 1)
 * over the generator (the discriminator held fixed; loss_out[0] includes
 * the term), and us_surr_gan_disc_step minimises
 *   (BCE(D(x, real), 1) + BCE(D(x, G(x)), 0)) / 2
 * over the discriminator, the fake frames being those of the last forward
 * pass (call it after the train step of the same x).  Requires height and
 * width multiples of 8. */
/* parameter count of a discriminator of width cd (16 .. 128, multiple of 16), -1 otherwise */
US_API int64_t us_surr_gan_num_params(int32_t cd);
/* enable the GAN term: init HOST [us_surr_gan_num_params(cd)] (copied),
 * gan_weight >= 0 (the paper's 0.01), lr > 0 (the discriminator's Adam step;
 * its betas and eps are the network's).  Allocates the discriminator's
 * buffers for max_batch frames (synchronous).  Errors: US_ERR_INVALID_ARG
 * (bad arguments, already enabled), US_ERR_OOM, US_ERR_CUDA. */
US_API us_status us_surr_gan_enable(us_surr* s, int32_t cd, const float* init, float gan_weight, float lr);
/* one discriminator step on (x, real) and the last forward's frames: loss_out
 * DEVICE [3] = (loss, real term, fake term); update = 1 applies Adam.
 * Errors: US_ERR_INVALID_ARG (not enabled, bad arguments), US_ERR_CUDA. */
US_API us_status us_surr_gan_disc_step(us_surr* s, const uint16_t* x, const float* real, int32_t B, float* loss_out,
                                       int32_t update, void* stream);
/* discriminator parameters and the gradients of its last step, HOST
 * [us_surr_gan_num_params(cd)], parameter layout; either may be NULL (synchronous) */
US_API us_status us_surr_gan_get(us_surr* s, float* params, float* grads);

/* parameters / gradients of the last train step, HOST, parameter layout (synchronous) */
US_API us_status us_surr_get_params(const us_surr* s, float* host_out);
US_API us_status us_surr_get_grads(us_surr* s, float* host_out);
/* wait for `stream`; US_ERR_TIMEOUT if a bounded tensor-core wait ran out */
US_API us_status us_surr_check(us_surr* s, void* stream);
/* checkpoint: config, step, parameters, Adam moments, CRC32; resuming
 * reproduces the next step exactly (the paper trains its networks for
 * 15-25 epochs, App. B.2; long runs need resumable state).  Errors:
 * US_ERR_INVALID_ARG (bad path, config mismatch, CRC mismatch), US_ERR_CUDA. */
US_API us_status us_surr_save(const us_surr* s, const char* path);
US_API us_status us_surr_load(us_surr* s, const char* path);

#ifdef __cplusplus
}
#endif

#endif /* USSIM_SURROGATE_H */
