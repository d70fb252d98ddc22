// Elevation sweep of a 3-D probe (Sec. 4, Task 3: volumetric images
// H x W x E): each environment's pose is replicated over E parallel planes
// offset along the probe's elevation axis (y), so that the 2-D render of the
// expanded batch yields the E slices of each volumetric image.
#include "us_internal.h"

namespace ussim {

// out[b E + e] = pose b translated by y_e = (e - (E - 1) / 2) * pitch along
// its own y axis: t' = t + R[:, 1] y_e (FP32, one rounding per product and sum)
__global__ void expand_elevation(const float* poses, int B, int E, float pitch, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * E) return;
  const int b = i / E, e = i - b * E;
  const float* M = poses + 12 * b;
  float* O = out + 12 * i;
  const float y = __fmul_rn((float)e - 0.5f * (float)(E - 1), pitch);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    O[4 * r + 0] = M[4 * r + 0];
    O[4 * r + 1] = M[4 * r + 1];
    O[4 * r + 2] = M[4 * r + 2];
    O[4 * r + 3] = __fadd_rn(M[4 * r + 3], __fmul_rn(M[4 * r + 1], y));
  }
}

cudaError_t launch_expand_elevation(const float* poses, int B, int E, float pitch, float* out, cudaStream_t st) {
  const int n = B * E;
  expand_elevation<<<(n + 127) / 128, 128, 0, st>>>(poses, B, E, pitch, out);
  return cudaGetLastError();
}

}  // namespace ussim
