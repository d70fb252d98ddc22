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

#ifdef __cplusplus
}
#endif

#endif /* USSIM_SURROGATE_H */
