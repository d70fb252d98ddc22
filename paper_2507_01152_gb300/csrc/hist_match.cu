// Histogram matching of CT images to a reference histogram (Sec. 3: the
// learned simulator's input CT slices are matched to the intensity
// histogram of a subset of its training CT images).  Discrete histogram
// specification with exact decisions: FP32 binning, cumulative counts, and
// bin k -> first reference bin m with R[m] n >= S[k] N in 64-bit integers;
// a considered pixel becomes the centre of bin m.
//
// One thread-block cluster of CS CTAs per image (CS = 2, 4 or 8, chosen
// from the batch so that small batches still fill the GPU): each CTA
// histograms its share of the pixels in shared memory; CTA r adds up bin
// segment r over the cluster (distributed shared memory), scans it and maps
// it once the segment totals are exchanged; every CTA then copies the whole
// bin map from its peers and remaps its pixels.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "us_internal.h"

namespace ussim {

namespace cg = cooperative_groups;

constexpr int kMatchThreads = 1024;

__device__ __forceinline__ int hm_bin(float v, float h0, float w, int nb) {
  const float q = floorf(__fdiv_rn(__fsub_rn(v, h0), w));
  return (int)fminf(fmaxf(q, 0.f), (float)(nb - 1));
}

// block-wide inclusive scan of c[0..nb) in place (each thread a contiguous run)
__device__ void hm_scan(int* c, int nb) {
  constexpr int NW = kMatchThreads / 32;
  __shared__ int warp_tot[NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (nb + kMatchThreads - 1) / kMatchThreads;
  const int b0 = min(tid * per, nb), b1 = min(b0 + per, nb);
  int run = 0;
  for (int k = b0; k < b1; ++k) run += c[k];
  // exclusive scan of the runs across the block
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int t = lane < NW ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < NW) warp_tot[lane] = t;   // inclusive over warps
  }
  __syncthreads();
  int acc = incl - run + (warp ? warp_tot[warp - 1] : 0);
  for (int k = b0; k < b1; ++k) {
    acc += c[k];
    c[k] = acc;
  }
  __syncthreads();
}

// image b = cluster index: hu[b][n_pix] (mask[b][n_pix] != 0 considered,
// all if null) -> out[b][n_pix] (if set) and, if slice is set, channel 1
// of the BF16 surrogate input pixels slice[b][n_pix] for the considered
// pixels
__global__ void __launch_bounds__(kMatchThreads) hist_match_kernel(const float* hu, const uint8_t* mask, int n_pix,
                                                                   const long long* R, int nb, float h0, float w,
                                                                   float* out, uint4* slice) {
  extern __shared__ int sm[];
  __shared__ int s_tot;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), r = (int)cl.block_rank(), tid = threadIdx.x;
  int* cnt = sm;        // [nb]: this CTA's counts, then the whole bin map
  int* seg = sm + nb;   // [nb]: this CTA's bin segment (sums, cumulative, map)
  const size_t base = (size_t)(blockIdx.x / cs) * n_pix;
  const int per = (((n_pix + cs - 1) / cs) + 3) & ~3;   // a multiple of 4: vector loads stay aligned
  const int i0 = min(r * per, n_pix), i1 = min(i0 + per, n_pix);
  const int sl = (nb + cs - 1) / cs;
  const int k0 = min(r * sl, nb), k1 = min(k0 + sl, nb);
  const float* x = hu + base;
  const uint8_t* m = mask ? mask + base : nullptr;

  for (int k = tid; k < nb; k += kMatchThreads) cnt[k] = 0;
  __syncthreads();
  // four pixels per load when the image's values (and mask) are 16-byte
  // (4-byte) aligned and n_pix is a multiple of 4
  const bool vec = (n_pix & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0 &&
                   (!m || (reinterpret_cast<uintptr_t>(m) & 3u) == 0);
  if (vec) {
    for (int j = (i0 >> 2) + tid; j < (i1 >> 2); j += kMatchThreads) {
      const float4 v = reinterpret_cast<const float4*>(x)[j];
      const uchar4 mm = m ? reinterpret_cast<const uchar4*>(m)[j] : make_uchar4(1, 1, 1, 1);
      if (mm.x) atomicAdd(&cnt[hm_bin(v.x, h0, w, nb)], 1);
      if (mm.y) atomicAdd(&cnt[hm_bin(v.y, h0, w, nb)], 1);
      if (mm.z) atomicAdd(&cnt[hm_bin(v.z, h0, w, nb)], 1);
      if (mm.w) atomicAdd(&cnt[hm_bin(v.w, h0, w, nb)], 1);
    }
  } else {
    for (int i = i0 + tid; i < i1; i += kMatchThreads)
      if (!m || m[i]) atomicAdd(&cnt[hm_bin(x[i], h0, w, nb)], 1);
  }
  cl.sync();
  // segment r: sums over the cluster, inclusive scan, total
  for (int k = k0 + tid; k < k1; k += kMatchThreads) {
    int t = 0;
    for (int q = 0; q < cs; ++q) t += cl.map_shared_rank(cnt, q)[k];
    seg[k] = t;
  }
  __syncthreads();
  hm_scan(seg + k0, k1 - k0);
  if (tid == 0) s_tot = k1 > k0 ? seg[k1 - 1] : 0;
  cl.sync();
  long long off = 0, n = 0;
  for (int q = 0; q < cs; ++q) {
    const long long t = *cl.map_shared_rank(&s_tot, q);
    if (q < r) off += t;
    n += t;
  }
  const long long N = R[nb - 1];
  if (n > 0)
    for (int k = k0 + tid; k < k1; k += kMatchThreads) {
      const long long want = ((long long)seg[k] + off) * N;
      int lo = 0, hi = nb - 1;   // first m with R[m] n >= want; m = nb - 1 always qualifies
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&R[mid]) * n >= want)
          hi = mid;
        else
          lo = mid + 1;
      }
      seg[k] = lo;
    }
  cl.sync();
  // the whole map from the CTAs' segments
  if (n > 0)
    for (int k = tid; k < nb; k += kMatchThreads) cnt[k] = cl.map_shared_rank(seg, k / sl)[k];
  cl.sync();   // no CTA leaves while a peer still reads its segment
  auto remap = [&](float v, bool sel) -> float {
    return sel ? __fadd_rn(__fmul_rn((float)cnt[hm_bin(v, h0, w, nb)] + 0.5f, w), h0) : v;
  };
  auto to_slice = [&](size_t i, float o) {
    uint4 px = slice[i];
    __nv_bfloat16* c = reinterpret_cast<__nv_bfloat16*>(&px);
    c[1] = __float2bfloat16_rn(fminf(fmaxf(o * 1e-3f, -1.f), 3.f));
    slice[i] = px;
  };
  if (vec && (!out || (reinterpret_cast<uintptr_t>(out + base) & 15u) == 0)) {
    for (int j = (i0 >> 2) + tid; j < (i1 >> 2); j += kMatchThreads) {
      const float4 v = reinterpret_cast<const float4*>(x)[j];
      const uchar4 mm = m ? reinterpret_cast<const uchar4*>(m)[j] : make_uchar4(1, 1, 1, 1);
      const bool s0 = n > 0 && mm.x, s1 = n > 0 && mm.y, s2 = n > 0 && mm.z, s3 = n > 0 && mm.w;
      const float4 o = make_float4(remap(v.x, s0), remap(v.y, s1), remap(v.z, s2), remap(v.w, s3));
      if (out) reinterpret_cast<float4*>(out + base)[j] = o;
      if (slice) {
        const size_t i = base + 4 * (size_t)j;
        if (s0) to_slice(i, o.x);
        if (s1) to_slice(i + 1, o.y);
        if (s2) to_slice(i + 2, o.z);
        if (s3) to_slice(i + 3, o.w);
      }
    }
  } else {
    for (int i = i0 + tid; i < i1; i += kMatchThreads) {
      const bool sel = n > 0 && (!m || m[i]);
      const float o = remap(x[i], sel);
      if (out) out[base + i] = o;
      if (slice && sel) to_slice(base + i, o);
    }
  }
}

cudaError_t launch_hist_match(const float* hu, const uint8_t* mask, int B, int n_pix, const long long* R, int nb,
                              float h0, float w, float* out, void* slice, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(hist_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * sizeof(int) * (size_t)nb));
  if (e != cudaSuccess) return e;
  // CTAs per image: two once the batch has an image per SM (two CTAs of
  // 1024 threads fit an SM), else four or eight (measured: a cluster of two
  // beats one CTA per image even on 512 images)
  int dev = 0, n_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int cs = B >= n_sm ? 2 : (4 * B >= n_sm ? 4 : 8);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)B * cs);
  cfg.blockDim = dim3(kMatchThreads);
  cfg.dynamicSmemBytes = 2 * sizeof(int) * (size_t)nb;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, hist_match_kernel, hu, mask, n_pix, R, nb, h0, w, out,
                            reinterpret_cast<uint4*>(slice));
}

}  // namespace ussim
