// Fused, persistent, batched render.
//
// One thread-block cluster renders one environment's frame at a time and
// takes the next environment from a global counter (costliest first).  The
// frame's scanlines are split evenly over the cluster's CTAs; each CTA keeps
// its lines' labels, scatter pattern and reflection impulses (then their
// axially filtered forms), energy and log image in shared memory, and the
// stages that need neighbouring lines (incidence angle, lateral PSF, scan
// conversion) read them from the other CTAs through distributed shared
// memory.  Nothing of a frame but the final image touches global memory.
//
// Per environment: (1) slice: nearest label and impedance of every sample
// of own lines, cluster barrier; (2) scanline model + in-place axial PSF per
// own line, cluster barrier; (3) lateral PSF, image
// I = (P (x) R_imp) + E (P (x) T) (App. B.2) and log compression, cluster
// barrier; (4) scan conversion (curvilinear) or transposed store (linear)
// with streaming stores.  Cross-CTA rows are reached through per-item
// tables of row pointers into the owning CTA's shared memory.
#include <cooperative_groups.h>

#include "us_internal.h"
#include "us_scanline.cuh"

namespace cg = cooperative_groups;

namespace ussim {

// per-item context shared by the CTA (read through shared memory)
struct ItemCtx {
  EnvItem it;
  DevProbe P;
  DevVolume V;
  DevPair pair;
  Pose M;
  int finite;
};

// In-place axial PSF of one line's two padded rows (scatter pattern and
// reflection impulses), one warp: K zeros, NS samples, K zeros, so every
// tap reads in bounds.  Chunk c's results are written back only after chunk
// c+1 has been computed, so every read sees unfiltered data (K <= 32).  Tap
// order matches the plain kernel.
__device__ __forceinline__ void axial_psf_padded(float* pt, float* pr, int NS, const float* w, int K, int lane) {
  float prev_t = 0.f, prev_r = 0.f;
  int prev_s = -1;
  const int taps = 2 * K + 1;
  for (int c = 0; c < NS; c += 32) {
    const int s = c + lane;
    float acc_t = 0.f, acc_r = 0.f;
    if (s < NS) {
      const float* qt = pt + s;
      const float* qr = pr + s;
      for (int k = 0; k < taps; ++k) {
        acc_t = fmaf(w[k], qt[k], acc_t);
        acc_r = fmaf(w[k], qr[k], acc_r);
      }
    }
    __syncwarp();
    if (prev_s >= 0 && prev_s < NS) {
      pt[K + prev_s] = prev_t;
      pr[K + prev_s] = prev_r;
    }
    __syncwarp();
    prev_t = acc_t;
    prev_r = acc_r;
    prev_s = s;
  }
  if (prev_s >= 0 && prev_s < NS) {
    pt[K + prev_s] = prev_t;
    pr[K + prev_s] = prev_r;
  }
  __syncwarp();
}

template <int CS, int NW>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NW * 32, 1) fused_render(RenderParams p, FusedLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ItemCtx cx;
  __shared__ int slot[2];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  float* sbuf = reinterpret_cast<float*>(smem);                   // impedance, then T, then P_ax (x) T
  float* rbuf = reinterpret_cast<float*>(smem + L.off_r);         // R_imp, then P_ax (x) R_imp
  float* ybuf = reinterpret_cast<float*>(smem + L.off_y);         // energy, then log image of own lines
  uint8_t* lbuf = smem + L.off_lab;                               // labels of own lines
  const uint8_t** lab_row = reinterpret_cast<const uint8_t**>(smem + L.off_lrow);  // any line -> its label row
  const float** s_row = reinterpret_cast<const float**>(smem + L.off_srow);        // any line -> its filtered T row
  const float** r_row = reinterpret_cast<const float**>(smem + L.off_rrow);        // any line -> its filtered R row
  const float** y_row = reinterpret_cast<const float**>(smem + L.off_yrow);        // any line -> its log row
  float* wax = reinterpret_cast<float*>(smem + L.off_wax);
  float* wlat = reinterpret_cast<float*>(smem + L.off_wlat);     // zero-padded at both ends
  DevTissue* tis = reinterpret_cast<DevTissue*>(smem + L.off_tis);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int n_items = p.n_items_dev ? *p.n_items_dev : p.n_items;
  if (rank == 0 && tid == 0) slot[0] = (int)atomicAdd(p.work, 1u);
  cl.sync();
  int parity = 0;
  int idx = *cl.map_shared_rank(&slot[0], 0);

  while (idx < n_items) {
    __syncthreads();  // every thread is done with the previous item's context and tables
    if (tid == 0) {
      const EnvItem it = p.items[idx];
      cx.it = it;
      cx.P = p.probes[it.probe];
      cx.V = p.vols[it.vol];
      cx.pair = p.pairs[it.pair];
      bool finite;
      cx.M = load_pose(p.poses, it.b, finite);
      cx.finite = finite;
    }
    __syncthreads();
    const DevProbe& P = cx.P;
    const int NL = P.nl, NS = P.ns, KA = P.k_ax, KL = P.k_lat;
    const int RS = (NS + 2 * KA) | 1;             // padded row stride (odd: no bank conflicts across rows)
    const int LPC = (NL + CS - 1) / CS;
    const int lbeg = rank * LPC;
    const int n_own = max(0, min(NL - lbeg, LPC));
    const int b = cx.it.b;

    for (int t = tid; t < 2 * KA + 1; t += blockDim.x) wax[t] = __ldg(&P.w_ax[t]);
    for (int t = tid; t < 2 * KL + 3; t += blockDim.x) wlat[t] = (t == 0 || t == 2 * KL + 2) ? 0.f : __ldg(&P.w_lat[t - 1]);
    for (int t = tid; t < p.n_labels; t += blockDim.x) tis[t] = P.tissue[t];
    for (int m = tid; m < NL; m += blockDim.x) {
      const int r = m / LPC, row = m - r * LPC;
      lab_row[m] = cl.map_shared_rank(lbuf, r) + row * NS;
      s_row[m] = cl.map_shared_rank(sbuf, r) + row * RS + KA;
      r_row[m] = cl.map_shared_rank(rbuf, r) + row * RS + KA;
      y_row[m] = cl.map_shared_rank(ybuf, r) + row * RS;
    }
    if (!cx.finite && rank == 0 && tid == 0) atomicOr(p.err, kErrNonFinitePose);
    __syncthreads();

    // (1) slice: nearest label and impedance of every sample of own lines
    for (int lr = warp; lr < n_own; lr += NW) {
      const int l = lbeg + lr;
      const float2 ln = P.lines[l];
      float* zrow = sbuf + lr * RS + KA;
      uint8_t* lrow = lbuf + lr * NS;
      for (int s = lane; s < NS; s += 32) {
        float x, z;
        beam_point(P, ln, s, x, z);
        const float3 u = to_voxel(cx.M, cx.V.inv_h, x, z);
        int vi;
        const uint8_t lb = nearest_label(cx.V, u, vi);
        lrow[s] = lb;
        zrow[s] = p.z_mode == 0 ? fmaxf(trilinear_hu(cx.V, u) + 1024.f, 1.f) : tis[lb].z;
        if (p.nn_index) p.nn_index[cx.it.beam_off + (long long)l * NS + s] = vi;
        if (p.label) p.label[cx.it.beam_off + (long long)l * NS + s] = lb;
      }
      for (int q = lane; q < KA; q += 32) {
        sbuf[lr * RS + q] = 0.f;
        sbuf[lr * RS + KA + NS + q] = 0.f;
        rbuf[lr * RS + q] = 0.f;
        rbuf[lr * RS + KA + NS + q] = 0.f;
      }
    }
    cl.sync();

    // (2) scanline model, then the axial PSF in place
    for (int lr = warp; lr < n_own; lr += NW) {
      const int l = lbeg + lr;
      float* row = sbuf + lr * RS + KA;
      float* rrow = rbuf + lr * RS + KA;
      float* erow = ybuf + lr * RS;
      const uint8_t* lrow = lbuf + lr * NS;
      auto labf = [&](int line, int s) -> unsigned { return lab_row[line][s]; };
      auto own = [&](int s) -> unsigned { return lrow[s]; };
      auto zf = [&](int s) -> float { return row[s]; };
      const float2 ln = P.lines[l];
      auto posf = [&](int s) -> float3 {
        float x, z;
        beam_point(P, ln, s, x, z);
        return sample_position(cx.M, x, z);
      };
      scanline_model(p, P, tis, cx.pair, b, l, lane, labf, own, zf,
                     [&](int s, float r, float t, float e) {
                       row[s] = t;
                       rrow[s] = r;
                       erow[s] = e;
                     },
                     posf, cx.it.vol);
      __syncwarp();
      axial_psf_padded(sbuf + lr * RS, rbuf + lr * RS, NS, wax, KA, lane);
    }
    cl.sync();

    // (3) lateral PSF of both filtered rows (two lines per thread), the
    // image with the line's own energy, and log compression (in place of
    // the energy)
    {
      const int nblk = (n_own + 1) >> 1, nch = (NS + 31) >> 5;
      for (int u = warp; u < nblk * nch; u += NW) {
        const int blk = u / nch, ch = u - blk * nch;
        const int s = ch * 32 + lane;
        if (s >= NS) continue;
        const int lr0 = 2 * blk, l0 = lbeg + lr0;
        const int mlo = max(l0 - KL, 0), mhi = min(l0 + 1 + KL, NL - 1);
        float t0 = 0.f, t1 = 0.f, r0 = 0.f, r1 = 0.f;
        for (int m = mlo; m <= mhi; ++m) {
          const float vt = s_row[m][s], vr = r_row[m][s];
          const int q = m - l0 + KL + 1;
          t0 = fmaf(wlat[q], vt, t0);
          t1 = fmaf(wlat[q - 1], vt, t1);
          r0 = fmaf(wlat[q], vr, r0);
          r1 = fmaf(wlat[q - 1], vr, r1);
        }
        const float acc0 = image_value(r0, t0, ybuf[lr0 * RS + s]);
        const float y0 = log_compress(P, acc0);
        ybuf[lr0 * RS + s] = y0;
        if (p.envelope) p.envelope[cx.it.beam_off + (long long)l0 * NS + s] = acc0;
        if (p.logimg) p.logimg[cx.it.beam_off + (long long)l0 * NS + s] = y0;
        if (lr0 + 1 < n_own) {
          const float acc1 = image_value(r1, t1, ybuf[(lr0 + 1) * RS + s]);
          const float y1 = log_compress(P, acc1);
          ybuf[(lr0 + 1) * RS + s] = y1;
          if (p.envelope) p.envelope[cx.it.beam_off + (long long)(l0 + 1) * NS + s] = acc1;
          if (p.logimg) p.logimg[cx.it.beam_off + (long long)(l0 + 1) * NS + s] = y1;
        }
      }
    }
    if (rank == 0 && tid == 0) slot[parity ^ 1] = (int)atomicAdd(p.work, 1u);
    cl.sync();

    // (4) output: scan conversion (curvilinear) or transposed store (linear)
    float* out = p.frames + cx.it.frame_off;
    if (P.kind == 0) {
      for (int s = warp; s < NS; s += NW)
        for (int lr = lane; lr < n_own; lr += 32) __stcs(&out[(long long)s * NL + lbeg + lr], ybuf[lr * RS + s]);
    } else {
      const int W = P.out_w, H = P.out_h;
      auto fan_pixel = [&](float fl, float fs) -> float {
        if (fl < 0.f) return 0.f;
        const int la = min((int)fl, NL - 2), sa = min((int)fs, NS - 2);
        const float a = fl - (float)la, bb = fs - (float)sa;
        const float* r0 = y_row[la];
        const float* r1 = y_row[la + 1];
        const float y00 = r0[sa], y01 = r0[sa + 1];
        const float y10 = r1[sa], y11 = r1[sa + 1];
        const float top = fmaf(a, y10 - y00, y00), bot = fmaf(a, y11 - y01, y01);
        return fmaf(bb, bot - top, top);
      };
      const int nrows = (H - rank + CS - 1) / CS;
      if ((W & 3) == 0) {
        const int n4 = W >> 2;
        const int total = nrows * n4;
        for (int t = tid; t < total; t += blockDim.x) {
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
        for (int t = tid; t < total; t += blockDim.x) {
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

bool fused_shape_fits(FusedShape& s, const std::vector<ProbeHost>& probes, int n_labels) {
  long long sbuf = 0, lab = 0, max_nl = 0;
  for (const ProbeHost& ph : probes) {
    const int NL = ph.desc.n_lines, NS = ph.desc.n_samples;
    const int lpc = (NL + s.cs - 1) / s.cs;
    const int rs = (NS + 2 * ph.k_ax) | 1;
    sbuf = std::max(sbuf, (long long)lpc * rs);
    lab = std::max(lab, (long long)lpc * NS);
    max_nl = std::max(max_nl, (long long)NL);
  }
  auto up = [](long long x, long long a) { return (x + a - 1) / a * a; };
  sbuf = up(sbuf, 4);
  s.sbuf_floats = (int)sbuf;
  long long off = sbuf * 4;
  s.lay.off_r = (int)off;
  off += sbuf * 4;
  s.lay.off_y = (int)off;
  off += sbuf * 4;
  s.lay.off_lab = (int)off;
  off = up(off + lab, 16);
  s.lay.off_lrow = (int)off;
  off += max_nl * 8;
  s.lay.off_srow = (int)off;
  off += max_nl * 8;
  s.lay.off_rrow = (int)off;
  off += max_nl * 8;
  s.lay.off_yrow = (int)off;
  off += max_nl * 8;
  s.lay.off_wax = (int)off;
  off = up(off + 4 * (2 * 32 + 1), 16);
  s.lay.off_wlat = (int)off;
  off = up(off + 4 * (2 * kMaxHalfTaps + 3), 16);
  s.lay.off_tis = (int)off;
  off = up(off + (long long)sizeof(DevTissue) * n_labels, 16);
  s.smem = (size_t)off;
  return s.smem <= 227 * 1024 - 1024;   // static shared memory (item context) takes the rest
}

// (cluster size, warps per CTA) instantiations; the cluster size is part of
// the kernel (__cluster_dims__), so every launch of a given instantiation,
// including a re-parameterised graph node, runs in clusters of that size
#define US_FUSED_SHAPES(X) X(4, 16) X(4, 32) X(8, 8) X(8, 16) X(8, 32) X(16, 8) X(16, 16) X(16, 32)

static const void* fused_fn(int cs, int nw) {
#define US_PICK(C, N) \
  if (cs == C && nw == N) return reinterpret_cast<const void*>(&fused_render<C, N>);
  US_FUSED_SHAPES(US_PICK)
#undef US_PICK
  return nullptr;
}

bool fused_shape_known(int cs, int nw) { return fused_fn(cs, nw) != nullptr; }

cudaError_t fused_prepare(const FusedShape& s) {
  const void* fn = fused_fn(s.cs, s.nw);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  if (s.cs > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t fused_max_clusters(const FusedShape& s, int* clusters) {
  const void* fn = fused_fn(s.cs, s.nw);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s.cs * 1024);
  cfg.blockDim = dim3(s.nw * 32);
  cfg.dynamicSmemBytes = s.smem;
  return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

cudaError_t launch_fused(const RenderParams& p, const FusedShape& s, cudaStream_t st) {
  const void* fn = fused_fn(s.cs, s.nw);
  if (!fn) return cudaErrorInvalidValue;
  const int clusters = std::max(1, p.n_items_dev ? s.clusters : std::min(s.clusters, p.n_items));
  RenderParams pp = p;
  FusedLayout lay = s.lay;
  void* args[2] = {&pp, &lay};
  return cudaLaunchKernel(fn, dim3(clusters * s.cs), dim3(s.nw * 32), args, s.smem, st);
}

// ------------------------------------------------------------- gating
// keep the items whose score exceeds the threshold, in batch order (one
// block, B <= 32 * 1024): out[0 .. *count)
__global__ void gate_compact(const EnvItem* items, int B, const float* score, float thr, EnvItem* out, int* count) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < B; c0 += blockDim.x) {
    const int b = c0 + threadIdx.x;
    const int keep = (b < B && score[b] > thr) ? 1 : 0;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int i = 0; i < w; ++i) before += warp_tot[i];
    if (keep) out[base + before + __popc(m & ((1u << lane) - 1u))] = items[b];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) base += warp_tot[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

cudaError_t launch_gate_compact(const EnvItem* items, int B, const float* score, float thr, EnvItem* out, int* count,
                                cudaStream_t st) {
  gate_compact<<<1, 1024, 0, st>>>(items, B, score, thr, out, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- checks

__global__ void max_label_kernel(const uint8_t* labels, long long n, unsigned* out) {
  unsigned m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned)labels[i]);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// corner records of a volume's HU grid (layout at DevVolume::hu8; the
// records of the y padding, never read, hold the zeros of cells outside)
__global__ void pack_corners_kernel(DevVolume V, uint4* out, long long n) {
  const int px = V.nx + 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long c = t >> 2;
    const int i = (int)(c % px) - 1, jq = (int)((c / px) % V.qy), k = (int)(c / ((long long)px * V.qy)) - 1;
    const int j = jq * 4 + (int)(t & 3) - 1;
    auto at = [&](int a, int b, int c) -> unsigned {
      const bool in = (unsigned)a < (unsigned)V.nx && (unsigned)b < (unsigned)V.ny && (unsigned)c < (unsigned)V.nz;
      return in ? (unsigned)(uint16_t)V.hu[((long long)c * V.ny + b) * V.nx + a] : 0u;
    };
    unsigned w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dj = q & 1, dk = q >> 1;
      w[q] = at(i, j + dj, k + dk) | (at(i + 1, j + dj, k + dk) << 16);
    }
    out[t] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

cudaError_t pack_corners(const DevVolume& V, uint4* out, cudaStream_t st) {
  pack_corners_kernel<<<152 * 8, 256, 0, st>>>(V, out, corner_records(V.nx, V.ny, V.nz));
  return cudaGetLastError();
}

// labels in 4 x 4 x 4 bricks (layout at DevVolume::lab4): one thread per
// 4-voxel row of a brick
__global__ void pack_labels_kernel(DevVolume V, uint32_t* out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t >> 4;
    const int r = (int)(t & 15);
    const int bi = (int)(b % V.bx), bj = (int)((b / V.bx) % V.by), bk = (int)(b / ((long long)V.bx * V.by));
    const int j = bj * 4 + (r & 3), k = bk * 4 + (r >> 2);
    uint32_t w = 0;
    if (j < V.ny && k < V.nz) {
      const uint8_t* row = V.labels + ((long long)k * V.ny + j) * V.nx;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = bi * 4 + q;
        if (i < V.nx) w |= (uint32_t)row[i] << (8 * q);
      }
    }
    out[t] = w;
  }
}

cudaError_t pack_labels(const DevVolume& V, uint8_t* out, cudaStream_t st) {
  pack_labels_kernel<<<152 * 8, 256, 0, st>>>(V, reinterpret_cast<uint32_t*>(out), label_bricks_bytes(V.nx, V.ny, V.nz) / 4);
  return cudaGetLastError();
}

cudaError_t max_label(const uint8_t* labels, long long n, unsigned* d_out, cudaStream_t st) {
  max_label_kernel<<<1024, 256, 0, st>>>(labels, n, d_out);
  return cudaGetLastError();
}

}  // namespace ussim
