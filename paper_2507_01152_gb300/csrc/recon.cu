// Reconstruction observation of the bone-surface task (Sec. 4, Task 2; App.
// C): each frame's ground-truth bone-surface points, thinned by a missing
// probability, accumulate into a per-environment reconstruction; the
// observation is that reconstruction in the current probe frame, voxelized
// to 40 x 40 x 40 voxels of 3 mm.
//
// Surface point: beam sample s whose nearest label is the bone label while
// sample s - 1's is not.  Kept unless word 0 of Philox-4x32-10 on counter
// (s, line, env, 1) with the render key of (seed, step) is below
// floor(p_miss 2^32).  The reconstruction is a bitmap over the voxels of the
// environment's volume (the point's nearest voxel) plus the list of its set
// voxels in the order they were first set (the set itself does not depend on
// that order).
#include <algorithm>

#include "us_internal.h"

namespace ussim {

// one warp per line, lanes over samples; the previous sample's label comes
// from the neighbouring lane (or the last lane of the previous chunk)
__global__ void recon_update(RenderParams p, const EnvItem* items, int B, int bone, unsigned thr, unsigned* bitmaps,
                             long long words, int* points, int* counts, int cap) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int b = blockIdx.y;
  if (b >= B) return;
  const EnvItem it = items[b];
  const DevProbe P = p.probes[it.probe];
  const DevVolume V = p.vols[it.vol];
  bool finite;
  const Pose M = load_pose(p.poses, it.b, finite);
  unsigned* bm = bitmaps + (long long)b * words;
  for (int l = blockIdx.x * nw + warp; l < P.nl; l += gridDim.x * nw) {
    const float2 ln = P.lines[l];
    int carry = -1;   // label of the sample before this chunk
    for (int c = 0; c < P.ns; c += 32) {
      const int s = c + lane;
      int lab = -2, vi = -1;
      if (s < P.ns) {
        float x, z;
        beam_point(P, ln, s, x, z);
        lab = (int)nearest_label(V, to_voxel(M, V.inv_h, x, z), vi);
      }
      int prev = __shfl_up_sync(0xffffffffu, lab, 1);
      if (lane == 0) prev = carry;
      carry = __shfl_sync(0xffffffffu, lab, 31);
      if (s > 0 && s < P.ns && lab == bone && prev != bone) {
        const uint4 w = philox4x32_10(make_uint4((unsigned)s, (unsigned)l, (unsigned)it.b, 1u), p.key);
        if (w.x >= thr) {
          const unsigned bit = 1u << (vi & 31);
          if (!(atomicOr(&bm[vi >> 5], bit) & bit)) {
            const int k = atomicAdd(&counts[b], 1);
            if (k < cap)
              points[(long long)b * cap + k] = vi;
            else
              atomicOr(p.err, kErrReconOverflow);
          }
        }
      }
    }
  }
}

// one thread per reconstructed voxel: probe-frame position, observation voxel
__global__ void recon_observe(RenderParams p, const EnvItem* items, int B, const int* points, const int* counts,
                              int cap, unsigned char* obs) {
  const int b = blockIdx.y;
  if (b >= B) return;
  // the grid covers the lists' capacity; blocks past this list's count
  // leave before loading anything else
  const int n = min(counts[b], cap);
  if (blockIdx.x * blockDim.x >= n) return;
  const EnvItem it = items[b];
  const DevVolume V = p.vols[it.vol];
  bool finite;
  const Pose M = load_pose(p.poses, it.b, finite);
  const float third = 0.333333343267f;   // (float)(1 / 3)
  const float vox = V.h;
  unsigned char* o = obs + (long long)b * 64000;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int vi = points[(long long)b * cap + i];
    const int ix = vi % V.nx, r = vi / V.nx, jy = r % V.ny, kz = r / V.ny;
    const float d0 = __fadd_rn(__fmul_rn((float)ix, vox), -M.m[3]);
    const float d1 = __fadd_rn(__fmul_rn((float)jy, vox), -M.m[7]);
    const float d2 = __fadd_rn(__fmul_rn((float)kz, vox), -M.m[11]);
    float q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      q[c] = __fadd_rn(__fadd_rn(__fmul_rn(M.m[c], d0), __fmul_rn(M.m[4 + c], d1)), __fmul_rn(M.m[8 + c], d2));
    const float fw = floorf(__fadd_rn(__fmul_rn(q[0], third), 20.f));
    const float fe = floorf(__fadd_rn(__fmul_rn(q[1], third), 20.f));
    const float fh = floorf(__fmul_rn(q[2], third));
    if (fw >= 0.f && fw < 40.f && fe >= 0.f && fe < 40.f && fh >= 0.f && fh < 40.f)
      o[((int)fh * 40 + (int)fw) * 40 + (int)fe] = 1;
  }
}

cudaError_t launch_recon_update(const RenderParams& p, const EnvItem* items, int B, int bone, unsigned thr,
                                unsigned* bitmaps, long long words, int* points, int* counts, int cap, int max_lines,
                                cudaStream_t st) {
  const dim3 grid((max_lines + 7) / 8, B);
  recon_update<<<grid, 256, 0, st>>>(p, items, B, bone, thr, bitmaps, words, points, counts, cap);
  return cudaGetLastError();
}

cudaError_t launch_recon_observe(const RenderParams& p, const EnvItem* items, int B, const int* points,
                                 const int* counts, int cap, unsigned char* obs, cudaStream_t st) {
  const dim3 grid(std::max(1, std::min(64, (cap + 255) / 256)), B);
  recon_observe<<<grid, 256, 0, st>>>(p, items, B, points, counts, cap, obs);
  return cudaGetLastError();
}

}  // namespace ussim
