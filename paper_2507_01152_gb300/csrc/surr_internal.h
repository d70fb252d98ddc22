// Entry points shared between the surrogate's translation units (not part
// of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ussim {
namespace surr {

// Stride-1 3x3 convolution Cin -> 32 (Cin 32 or 64, ReLU) with the 1x1
// sigmoid head fused into its epilogue: head_out[p] = sigmoid(head_b[0] +
// sum_c y[p][c] head_w[c]), over the BF16 outputs in channel order, as the
// separate head computes it.  y may be null (the activation is then not
// stored).  Returns false, launching nothing, if the shape or the views have
// no fused form; e holds the launch status otherwise.
bool conv3x3_head_fwd(cudaError_t& e, const uint16_t* x, int x_cs, int x_co, int Cin, const uint16_t* w,
                      const float* bias, uint16_t* y, int y_cs, int y_co, int B, int H, int W, const float* head_w,
                      const float* head_b, float* head_out, unsigned* err, cudaStream_t st);

}  // namespace surr
}  // namespace ussim
