// Fused, persistent, batched render.
//
// One thread-block cluster renders one environment's frame at a time and
// takes the next environment from a global counter (costliest first).  The
// frame's scanlines are split evenly over the cluster's CTAs; each CTA keeps
// its lines' labels, pre-PSF image and log image in shared memory, and the
// stages that need neighbouring lines (incidence angle, lateral PSF, scan
// conversion) read them from the other CTAs through distributed shared
// memory.  Nothing of a frame but the final image touches global memory.
//
// Per environment: (1) label slice of own lines, cluster barrier;
// (2) scanline model + in-place axial PSF per own line, cluster barrier;
// (3) lateral PSF + log compression, cluster barrier; (4) scan conversion
// (curvilinear) or transposed store (linear) with streaming stores.
#include <cooperative_groups.h>

#include "us_internal.h"
#include "us_scanline.cuh"

namespace cg = cooperative_groups;

namespace ussim {

// In-place axial PSF of one line held in shared memory, one warp.  Chunk
// c's filtered values are written back only after chunk c+1 has been
// computed, so every read sees unfiltered data (requires K <= 32).
__device__ __forceinline__ void axial_psf_inplace(float* row, int NS, const float* w, int K, int lane) {
  float prev = 0.f;
  int prev_s = -1;
  for (int c = 0; c < NS; c += 32) {
    const int s = c + lane;
    float acc = 0.f;
    if (s < NS) {
      for (int k = -K; k <= K; ++k) {
        const int ss = s + k;
        if (ss >= 0 && ss < NS) acc = fmaf(__ldg(&w[k + K]), row[ss], acc);
      }
    }
    __syncwarp();
    if (prev_s >= 0 && prev_s < NS) row[prev_s] = prev;
    __syncwarp();
    prev = acc;
    prev_s = s;
  }
  if (prev_s >= 0 && prev_s < NS) row[prev_s] = prev;
  __syncwarp();
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, 1) fused_render(RenderParams p, int sbuf_floats) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int slot[2];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int CS = (int)cl.num_blocks();
  float* sbuf = reinterpret_cast<float*>(smem);   // pre-PSF, then axially filtered lines
  float* ybuf = sbuf + sbuf_floats;                // log image of own lines
  uint8_t* lbuf = reinterpret_cast<uint8_t*>(ybuf + sbuf_floats);  // labels of own lines
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (rank == 0 && threadIdx.x == 0) slot[0] = (int)atomicAdd(p.work, 1u);
  cl.sync();
  int parity = 0;
  int idx = *cl.map_shared_rank(&slot[0], 0);

  while (idx < p.n_items) {
    const EnvItem it = p.items[idx];
    const DevProbe P = p.probes[it.probe];
    const DevVolume V = p.vols[it.vol];
    const DevPair pair = p.pairs[it.pair];
    bool finite;
    const Pose M = load_pose(p.poses, it.b, finite);
    if (!finite && rank == 0 && threadIdx.x == 0) atomicOr(p.err, kErrNonFinitePose);
    const int NL = P.nl, NS = P.ns, NSP = NS | 1;
    const int LPC = (NL + CS - 1) / CS;
    const int lbeg = rank * LPC;
    const int n_own = max(0, min(NL - lbeg, LPC));

    // (1) label slice
    for (int lr = warp; lr < n_own; lr += NW) {
      const int l = lbeg + lr;
      const float2 ln = P.lines[l];
      for (int s = lane; s < NS; s += 32) {
        float x, z;
        beam_point(P, ln, s, x, z);
        const int vi = nearest_voxel(V, to_voxel(M, V.inv_h, x, z));
        const uint8_t lb = vi >= 0 ? __ldg(&V.labels[vi]) : (uint8_t)0;
        lbuf[lr * NS + s] = lb;
        if (p.nn_index) p.nn_index[it.beam_off + (long long)l * NS + s] = vi;
        if (p.label) p.label[it.beam_off + (long long)l * NS + s] = lb;
      }
    }
    cl.sync();

    // (2) scanline model and axial PSF
    auto labf = [&](int line, int s) -> unsigned {
      const int r = line / LPC;
      const int row = line - r * LPC;
      const uint8_t* base = r == rank ? lbuf : cl.map_shared_rank(lbuf, r);
      return base[row * NS + s];
    };
    for (int lr = warp; lr < n_own; lr += NW) {
      float* row = sbuf + lr * NSP;
      scanline_model(p, P, V, pair, M, it.b, lbeg + lr, lane, labf, [&](int s, float v) { row[s] = v; });
      __syncwarp();
      axial_psf_inplace(row, NS, P.w_ax, P.k_ax, lane);
    }
    cl.sync();

    // (3) lateral PSF and log compression
    for (int lr = warp; lr < n_own; lr += NW) {
      const int l = lbeg + lr;
      const int lo = max(l - P.k_lat, 0), hi = min(l + P.k_lat, NL - 1);
      const float* wl = P.w_lat + (P.k_lat - l);
      for (int s = lane; s < NS; s += 32) {
        int r = lo / LPC, row = lo - r * LPC;
        const float* base = r == rank ? sbuf : cl.map_shared_rank(sbuf, r);
        float acc = 0.f;
        for (int ll = lo; ll <= hi; ++ll) {
          acc = fmaf(__ldg(&wl[ll]), base[row * NSP + s], acc);
          if (++row == LPC && ll < hi) {
            row = 0;
            ++r;
            base = r == rank ? sbuf : cl.map_shared_rank(sbuf, r);
          }
        }
        const float y = log_compress(P, acc);
        ybuf[lr * NSP + s] = y;
        if (p.envelope) p.envelope[it.beam_off + (long long)l * NS + s] = acc;
        if (p.logimg) p.logimg[it.beam_off + (long long)l * NS + s] = y;
      }
    }
    if (rank == 0 && threadIdx.x == 0) slot[parity ^ 1] = (int)atomicAdd(p.work, 1u);
    cl.sync();

    // (4) output
    float* out = p.frames + it.frame_off;
    if (P.kind == 0) {
      for (int s = warp; s < NS; s += NW)
        for (int lr = lane; lr < n_own; lr += 32) __stcs(&out[(long long)s * NL + lbeg + lr], ybuf[lr * NSP + s]);
    } else {
      const int W = P.out_w, H = P.out_h;
      auto fan_pixel = [&](float fl, float fs) -> float {
        if (fl < 0.f) return 0.f;
        const int la = min((int)fl, NL - 2), sa = min((int)fs, NS - 2);
        const float a = fl - (float)la, bb = fs - (float)sa;
        const int r0 = la / LPC, row0 = la - r0 * LPC;
        int r1 = r0, row1 = row0 + 1;
        if (row1 == LPC) {
          row1 = 0;
          ++r1;
        }
        const float* b0 = r0 == rank ? ybuf : cl.map_shared_rank(ybuf, r0);
        const float* b1 = r1 == rank ? ybuf : cl.map_shared_rank(ybuf, r1);
        const float y00 = b0[row0 * NSP + sa], y01 = b0[row0 * NSP + sa + 1];
        const float y10 = b1[row1 * NSP + sa], y11 = b1[row1 * NSP + sa + 1];
        const float top = fmaf(a, y10 - y00, y00), bot = fmaf(a, y11 - y01, y01);
        return fmaf(bb, bot - top, top);
      };
      const int nrows = (H - rank + CS - 1) / CS;
      if ((W & 3) == 0) {
        const int n4 = W >> 2;
        const int total = nrows * n4;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
          const int ri = t / n4, c4 = t - ri * n4;
          const long long pix = (long long)(rank + ri * CS) * W + 4 * c4;
          const float4* lut4 = reinterpret_cast<const float4*>(P.lut + pix);
          const float4 f01 = __ldg(lut4), f23 = __ldg(lut4 + 1);
          float4 v;
          v.x = fan_pixel(f01.x, f01.y);
          v.y = fan_pixel(f01.z, f01.w);
          v.z = fan_pixel(f23.x, f23.y);
          v.w = fan_pixel(f23.z, f23.w);
          __stcs(reinterpret_cast<float4*>(out + pix), v);
        }
      } else {
        const int total = nrows * W;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
          const int ri = t / W, c = t - ri * W;
          const long long pix = (long long)(rank + ri * CS) * W + c;
          const float2 f = __ldg(&P.lut[pix]);
          __stcs(&out[pix], fan_pixel(f.x, f.y));
        }
      }
    }
    parity ^= 1;
    idx = *cl.map_shared_rank(&slot[parity], 0);
  }
  cl.sync();  // no CTA may leave while another can still read its shared memory
}

bool fused_shape_fits(FusedShape& s, const std::vector<ProbeHost>& probes) {
  int sbuf = 0, lab = 0;
  for (const ProbeHost& ph : probes) {
    const int NL = ph.desc.n_lines, NS = ph.desc.n_samples;
    const int lpc = (NL + s.cs - 1) / s.cs;
    sbuf = std::max(sbuf, lpc * (NS | 1));
    lab = std::max(lab, lpc * NS);
  }
  sbuf = (sbuf + 3) & ~3;
  s.sbuf_floats = sbuf;
  s.smem = (size_t)sbuf * 8 + (size_t)((lab + 15) & ~15);
  return s.smem <= 227 * 1024;
}

template <int NW>
static cudaError_t prepare(const FusedShape& s, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr) {
  cudaError_t e = cudaFuncSetAttribute(fused_render<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  if (s.cs > 8) {
    e = cudaFuncSetAttribute(fused_render<NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cfg.blockDim = dim3(NW * 32);
  cfg.dynamicSmemBytes = s.smem;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = s.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaSuccess;
}

template <int NW>
static cudaError_t max_clusters_nw(const FusedShape& s, int* clusters) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cudaError_t e = prepare<NW>(s, cfg, attr);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3(s.cs * 1024);
  return cudaOccupancyMaxActiveClusters(clusters, fused_render<NW>, &cfg);
}

cudaError_t fused_max_clusters(const FusedShape& s, int* clusters) {
  switch (s.nw) {
    case 4: return max_clusters_nw<4>(s, clusters);
    case 8: return max_clusters_nw<8>(s, clusters);
    case 16: return max_clusters_nw<16>(s, clusters);
    case 32: return max_clusters_nw<32>(s, clusters);
    default: return cudaErrorInvalidValue;
  }
}

template <int NW>
static cudaError_t launch_nw(const RenderParams& p, const FusedShape& s, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cudaError_t e = prepare<NW>(s, cfg, attr);
  if (e != cudaSuccess) return e;
  const int clusters = std::max(1, std::min(s.clusters, p.n_items));
  cfg.gridDim = dim3(clusters * s.cs);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, fused_render<NW>, p, s.sbuf_floats);
}

cudaError_t launch_fused(const RenderParams& p, const FusedShape& s, cudaStream_t st) {
  switch (s.nw) {
    case 4: return launch_nw<4>(p, s, st);
    case 8: return launch_nw<8>(p, s, st);
    case 16: return launch_nw<16>(p, s, st);
    case 32: return launch_nw<32>(p, s, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- checks

__global__ void max_label_kernel(const uint8_t* labels, long long n, unsigned* out) {
  unsigned m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned)labels[i]);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

cudaError_t max_label(const uint8_t* labels, long long n, unsigned* d_out, cudaStream_t st) {
  max_label_kernel<<<1024, 256, 0, st>>>(labels, n, d_out);
  return cudaGetLastError();
}

}  // namespace ussim
