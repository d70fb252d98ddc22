// Histogram matching of CT images to a reference histogram (Sec. 3: the
// learned simulator's input CT slices are matched to the intensity
// histogram of a subset of its training CT images).  Discrete histogram
// specification with exact decisions: FP32 binning, cumulative counts, and
// bin k -> first reference bin m with R[m] n >= S[k] N in 64-bit integers;
// a considered pixel becomes the centre of bin m.
//
// One block per image: shared-memory histogram (atomics), block-wide
// inclusive scan, per-bin binary search over the reference, remap.
#include <cuda_bf16.h>

#include "us_internal.h"

namespace ussim {

constexpr int kMatchThreads = 1024;

__device__ __forceinline__ int hm_bin(float v, float h0, float w, int nb) {
  const float q = floorf(__fdiv_rn(__fsub_rn(v, h0), w));
  return (int)fminf(fmaxf(q, 0.f), (float)(nb - 1));
}

// block-wide inclusive scan of c[0..nb) in place (each thread a contiguous run)
__device__ void hm_scan(int* c, int nb) {
  __shared__ int warp_tot[kMatchThreads / 32];
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
    int t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    warp_tot[lane] = t;   // inclusive over warps
  }
  __syncthreads();
  int acc = incl - run + (warp ? warp_tot[warp - 1] : 0);
  for (int k = b0; k < b1; ++k) {
    acc += c[k];
    c[k] = acc;
  }
  __syncthreads();
}

// image b: hu[b][n_pix] (mask[b][n_pix] != 0 considered, all if null) ->
// out[b][n_pix] (if set) and, if slice is set, channel 1 of the BF16
// surrogate input pixels slice[b][n_pix] for the considered pixels
__global__ void __launch_bounds__(kMatchThreads) hist_match_kernel(const float* hu, const uint8_t* mask, int n_pix,
                                                                   const long long* R, int nb, float h0, float w,
                                                                   float* out, uint4* slice) {
  extern __shared__ int cnt[];   // [nb]: counts, cumulative counts, then the bin map
  __shared__ int s_n;
  const int tid = threadIdx.x;
  const size_t base = (size_t)blockIdx.x * n_pix;
  const float* x = hu + base;
  const uint8_t* m = mask ? mask + base : nullptr;
  for (int k = tid; k < nb; k += kMatchThreads) cnt[k] = 0;
  __syncthreads();
  for (int i = tid; i < n_pix; i += kMatchThreads)
    if (!m || m[i]) atomicAdd(&cnt[hm_bin(x[i], h0, w, nb)], 1);
  __syncthreads();
  hm_scan(cnt, nb);
  if (tid == 0) s_n = cnt[nb - 1];
  __syncthreads();
  const long long n = s_n, N = R[nb - 1];
  if (n > 0) {
    for (int k = tid; k < nb; k += kMatchThreads) {
      const long long want = (long long)cnt[k] * N;
      int lo = 0, hi = nb - 1;   // first m with R[m] n >= want; m = nb - 1 always qualifies
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&R[mid]) * n >= want)
          hi = mid;
        else
          lo = mid + 1;
      }
      cnt[k] = lo;
    }
  }
  __syncthreads();
  for (int i = tid; i < n_pix; i += kMatchThreads) {
    const float v = x[i];
    const bool sel = n > 0 && (!m || m[i]);
    float o = v;
    if (sel) o = __fadd_rn(__fmul_rn((float)cnt[hm_bin(v, h0, w, nb)] + 0.5f, w), h0);
    if (out) out[base + i] = o;
    if (slice && sel) {
      uint4 px = slice[base + i];
      __nv_bfloat16* c = reinterpret_cast<__nv_bfloat16*>(&px);
      c[1] = __float2bfloat16_rn(fminf(fmaxf(o * 1e-3f, -1.f), 3.f));
      slice[base + i] = px;
    }
  }
}

cudaError_t launch_hist_match(const float* hu, const uint8_t* mask, int B, int n_pix, const long long* R, int nb,
                              float h0, float w, float* out, void* slice, cudaStream_t st) {
  const size_t smem = sizeof(int) * (size_t)nb;
  cudaError_t e = cudaFuncSetAttribute(hist_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  hist_match_kernel<<<(unsigned)B, kMatchThreads, smem, st>>>(hu, mask, n_pix, R, nb, h0, w, out,
                                                             reinterpret_cast<uint4*>(slice));
  return cudaGetLastError();
}

}  // namespace ussim
