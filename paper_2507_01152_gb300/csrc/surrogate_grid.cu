// The learned surrogate on a batch of mixed probes (SonoGym App. B.2:
// the learning-based simulator maps CT / label slices to images; here it
// runs on one H x W grid for every environment, whatever its probe):
//  * grid_slice_kernel samples each environment's label / CT slice on an
//    H x W grid spanning that environment's output field (curvilinear: the
//    fan's bounding box; linear: the image rectangle), through the render's
//    FP32 voxel-coordinate path;
//  * resize_kernel maps the H x W surrogate frames back onto each
//    environment's own output grid (bilinear, zero outside a curvilinear
//    fan), so the physics fallback and the consumer see frames of the
//    probe's size;
//  * audit_compact picks the physics audit of the surrogate's error gate: a
//    seeded fraction of the frames the gate let through, rendered by
//    physics beside the surrogate frame to check the error predictor.
#include <cuda_bf16.h>

#include "us_internal.h"

namespace ussim {

__global__ void grid_slice_kernel(RenderParams p, const EnvItem* items, int H, int W, const DevGridTab* tabs,
                                  uint4* out) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W) return;
  const EnvItem it = items[b];
  const DevGridTab t = tabs[it.probe];
  const DevVolume V = p.vols[it.vol];
  bool finite;
  const Pose M = load_pose(p.poses, it.b, finite);
  const int r = q / W, c = q - r * W;
  const float3 u = to_voxel(M, V.inv_h, __ldg(&t.px[c]), __ldg(&t.pz[r]));
  int vi;
  const float lab = (float)nearest_label(V, u, vi);
  const float hu = fminf(fmaxf(trilinear_hu(V, u) * 1e-3f, -1.f), 3.f);
  __align__(16) __nv_bfloat16 v[8];
  v[0] = __float2bfloat16_rn(0.25f * lab);
  v[1] = __float2bfloat16_rn(hu);
  v[2] = __float2bfloat16_rn(__ldg(&t.mask[q]) ? 1.f : 0.f);
#pragma unroll
  for (int k = 3; k < 8; ++k) v[k] = __float2bfloat16_rn(0.f);
  out[(size_t)b * H * W + q] = *reinterpret_cast<const uint4*>(v);
}

cudaError_t launch_grid_slices(const RenderParams& p, const EnvItem* items_batch, int B, int H, int W,
                               const DevGridTab* tabs, void* out, cudaStream_t st) {
  const dim3 grid((H * W + 255) / 256, B);
  grid_slice_kernel<<<grid, 256, 0, st>>>(p, items_batch, H, W, tabs, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

// Output pixel (r, c) of an out_h x out_w frame reads the H x W source at
// fy = (r + 1/2) H / out_h - 1/2, fx = (c + 1/2) W / out_w - 1/2 (pixel
// centres of the same field), clamped to the source, bilinear; curvilinear
// pixels outside the fan are 0, as in the physics frame.
__global__ void resize_kernel(RenderParams p, const EnvItem* items, const float* src, int H, int W) {
  const int b = blockIdx.y;
  const EnvItem it = items[b];
  const DevProbe& P = p.probes[it.probe];
  const int OH = P.out_h, OW = P.out_w;
  const float sy = (float)H / (float)OH, sx = (float)W / (float)OW;
  const float* s = src + (size_t)b * H * W;
  float* out = p.frames + it.frame_off;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < OH * OW; q += gridDim.x * blockDim.x) {
    const int r = q / OW, c = q - r * OW;
    float v = 0.f;
    if (P.kind == 0 || P.lut[q].x >= 0.f) {
      const float fy = fminf(fmaxf(fmaf((float)r + 0.5f, sy, -0.5f), 0.f), (float)(H - 1));
      const float fx = fminf(fmaxf(fmaf((float)c + 0.5f, sx, -0.5f), 0.f), (float)(W - 1));
      const int y0 = min((int)fy, H - 2), x0 = min((int)fx, W - 2);
      const float a = fy - (float)y0, bb = fx - (float)x0;
      const float* r0 = s + (size_t)y0 * W + x0;
      const float top = fmaf(bb, r0[1] - r0[0], r0[0]);
      const float bot = fmaf(bb, r0[W + 1] - r0[W], r0[W]);
      v = fmaf(a, bot - top, top);
    }
    __stcs(&out[q], v);
  }
}

cudaError_t launch_resize(const RenderParams& p, const EnvItem* items_batch, int B, const float* src, int H, int W,
                          int max_out, cudaStream_t st) {
  const dim3 grid((unsigned)std::min(64, (max_out + 255) / 256), B);
  resize_kernel<<<grid, 256, 0, st>>>(p, items_batch, src, H, W);
  return cudaGetLastError();
}

// Frames the gate keeps (score <= thr) enter the audit when word 0 of
// Philox-4x32-10 on counter (0, 0, env, 2), key = the render key of
// (seed, step), is below t_audit = floor(fraction 2^32): a fixed,
// reproducible subset of about that fraction, fresh every step.  One block,
// B <= 32 * 1024; out[0 .. *count) in batch order, flags[b] = 1 if audited.
__global__ void audit_compact(const EnvItem* items, int B, const float* score, float thr, uint2 key,
                              unsigned long long t_audit, EnvItem* out, int* count, uint8_t* flags) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < B; c0 += blockDim.x) {
    const int b = c0 + threadIdx.x;
    int keep = 0;
    if (b < B && !(score[b] > thr)) {
      const uint4 w = philox4x32_10(make_uint4(0u, 0u, (unsigned)b, 2u), key);
      keep = (unsigned long long)w.x < t_audit ? 1 : 0;
    }
    if (b < B && flags) flags[b] = (uint8_t)keep;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    if (lane == 0) warp_tot[wi] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int i = 0; i < wi; ++i) before += warp_tot[i];
    if (keep) out[base + before + __popc(m & ((1u << lane) - 1u))] = items[b];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) base += warp_tot[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

cudaError_t launch_audit_compact(const EnvItem* items, int B, const float* score, float thr, uint2 key,
                                 unsigned long long t_audit, EnvItem* out, int* count, uint8_t* flags,
                                 cudaStream_t st) {
  audit_compact<<<1, 1024, 0, st>>>(items, B, score, thr, key, t_audit, out, count, flags);
  return cudaGetLastError();
}

}  // namespace ussim
