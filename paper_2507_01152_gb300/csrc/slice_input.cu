// Input of the learned surrogate: the label and CT slices on each env's
// output pixel grid (Fig. 2 caption: image plane -> 2-D CT and label
// slices), as 8-channel BF16 pixels (label / 4, clamp(HU / 1000, -1, 3),
// inside-fan flag, five zeros).  Same FP32 voxel-coordinate path as the
// render's beam samples.
#include <cuda_bf16.h>

#include "us_internal.h"

namespace ussim {

// hu_raw / in_fan (optional): the unscaled trilinear HU and the inside-fan
// flag of every pixel, for the histogram matching that follows
__global__ void slice_input_kernel(RenderParams p, const EnvItem* items, int H, int W, uint4* out, float* hu_raw,
                                   uint8_t* in_fan) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W) return;
  const EnvItem it = items[b];
  const DevProbe& P = p.probes[it.probe];
  const DevVolume V = p.vols[it.vol];
  bool finite;
  const Pose M = load_pose(p.poses, it.b, finite);
  const int r = q / W, c = q - r * W;
  float x, z, mask = 1.f;
  if (P.kind == 1) {
    x = P.px[c];
    z = P.pz[r];
    mask = P.lut[q].x >= 0.f ? 1.f : 0.f;
  } else {
    beam_point(P, P.lines[c], r, x, z);
  }
  const float3 u = to_voxel(M, V.inv_h, x, z);
  int vi;
  const float lab = (float)nearest_label(V, u, vi);
  const float hu_v = trilinear_hu(V, u);
  const float hu = fminf(fmaxf(hu_v * 1e-3f, -1.f), 3.f);
  if (hu_raw) {
    hu_raw[(size_t)b * H * W + q] = hu_v;
    in_fan[(size_t)b * H * W + q] = mask != 0.f;
  }
  __align__(16) __nv_bfloat16 v[8];
  v[0] = __float2bfloat16_rn(0.25f * lab);
  v[1] = __float2bfloat16_rn(hu);
  v[2] = __float2bfloat16_rn(mask);
#pragma unroll
  for (int k = 3; k < 8; ++k) v[k] = __float2bfloat16_rn(0.f);
  out[(size_t)b * H * W + q] = *reinterpret_cast<const uint4*>(v);
}

cudaError_t launch_slice_input(const RenderParams& p, const EnvItem* items_batch, int B, int H, int W, void* out,
                               float* hu_raw, uint8_t* in_fan, cudaStream_t st) {
  const dim3 grid((H * W + 255) / 256, B);
  slice_input_kernel<<<grid, 256, 0, st>>>(p, items_batch, H, W, reinterpret_cast<uint4*>(out), hu_raw, in_fan);
  return cudaGetLastError();
}

}  // namespace ussim
