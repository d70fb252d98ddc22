// Two-pass batched render without clusters.
//
// Pass A (split_lines): one block per (environment, group of G lines), one
// warp per line.  The block takes the nearest labels of its lines (four
// samples' loads in flight a lane) and of the lines the incidence stencil can
// reach on either side (at most kThetaDMax), the impedance of its own lines,
// runs the scanline model (reflection impulses R_imp, scatter pattern T,
// energy E), applies the axial PSF to R_imp and T, and writes the filtered
// pair (AR, AT) and E to a beam-layout line buffer in global memory.
//
// Pass B (split_image): one block per tile (environment, wedge of GB lines,
// 128-sample chunk).  The block stages the filtered pairs its wedge needs
// (its lines, one more line for the bilinear step, and the lateral PSF's
// reach on both sides) and the energy of its own lines, forms the lateral
// PSF of both, the image
// I = (P (x) R_imp) + E (P (x) T) (App. B.2) and its log in shared memory, and
// scan-converts the output pixels assigned to the wedge: a host-built list,
// per probe, of the pixels whose bilinear footprint lies on the wedge's
// lines (pixels outside the fan go to the wedge of the preceding in-fan
// pixel of their row), so every read is local.
//
// The two grids launch the plan's work units (each environment's own groups
// and tiles, over the costliest-first work list).  Without a unit list,
// blocks are numbered item-major and a block whose group lies past its
// probe's lines, or whose item lies past a device-side item count, exits at
// once.  Per-line arithmetic, tap order and
// bilinear formula are those of the plain and cluster paths, so all three
// produce identical frames.
#include <algorithm>
#include <cstring>

#include "umma.cuh"
#include "us_internal.h"
#include "us_scanline.cuh"

namespace ussim {

// axial PSF of two padded rows (K zeros, NS samples, K zeros each, and one
// more element): the scatter pattern's and the reflection impulses', written
// as (P (x) R_imp, P (x) T) pairs to dst[0 .. NS-1] (the line buffer).
// KC > 0: the half-width is the compile-time KC (== K), the taps sit in
// registers and each lane filters two adjacent samples (s, s + 1) of a
// 64-sample chunk from K + 1 8-byte loads of each row (rows 8-byte aligned
// at even offsets), storing both pairs as one 16-byte store when dst is
// 16-byte aligned; KC = 0: any K, one sample a lane, taps read from shared
// memory.  Same tap order as the plain kernel.  rmask bit i: some
// reflection impulse of samples 32 i .. 32 i + 31 is not zero.  The
// impulses are >= 0, so an output chunk whose window holds none is exactly
// +0, as the full sum of zero taps would be: the warp skips its reflection
// taps there.
template <int KC>
__device__ __forceinline__ void axial_psf_rows(const float* pt, const float* pr, int NS, const float* w, int K,
                                               int lane, unsigned rmask, float2* dst) {
  if constexpr (KC > 0) {
    constexpr int TC = 2 * KC + 1, NV = KC + 1;   // taps; 8-byte loads covering s .. s + 2 KC + 1
    float wr[TC];
#pragma unroll
    for (int k = 0; k < TC; ++k) wr[k] = w[k];
    const bool wide = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;   // warp-uniform
    // two filtered rows from one padded row: output s takes elements
    // s + k, output s + 1 elements s + 1 + k (k = 0 .. 2 KC)
    auto filter2 = [&](const float* q, float& o0, float& o1) {
      float2 v[NV];
#pragma unroll
      for (int m = 0; m < NV; ++m) v[m] = reinterpret_cast<const float2*>(q)[m];
      o0 = 0.f;
      o1 = 0.f;
#pragma unroll
      for (int k = 0; k < TC; ++k) {
        o0 = fmaf(wr[k], (k & 1) ? v[k >> 1].y : v[k >> 1].x, o0);
        o1 = fmaf(wr[k], (k & 1) ? v[(k + 1) >> 1].x : v[k >> 1].y, o1);
      }
    };
    for (int c = 0; c < NS; c += 64) {
      const int s = c + 2 * lane, ci = c >> 5;
      // outputs c .. c + 63 read impulses c - KC .. c + 63 + KC: chunks ci - 1 .. ci + 2
      const bool refl = ((ci == 0 ? rmask << 1 : rmask >> (ci - 1)) & 15u) != 0;   // warp-uniform
      if (s < NS) {
        float t0, t1, r0 = 0.f, r1 = 0.f;
        filter2(pt + s, t0, t1);
        if (refl) filter2(pr + s, r0, r1);
        if (s + 1 < NS && wide) {
          *reinterpret_cast<float4*>(dst + s) = make_float4(r0, t0, r1, t1);
        } else {
          dst[s] = make_float2(r0, t0);
          if (s + 1 < NS) dst[s + 1] = make_float2(r1, t1);
        }
      }
    }
  } else {
    const int taps = 2 * K + 1;
    for (int c = 0; c < NS; c += 32) {
      const int s = c + lane, ci = c >> 5;
      const bool refl = ((ci == 0 ? rmask << 1 : rmask >> (ci - 1)) & 7u) != 0;   // warp-uniform
      if (s < NS) {
        float acc_t = 0.f, acc_r = 0.f;
        const float* qt = pt + s;
        const float* qr = pr + s;
        for (int k = 0; k < taps; ++k) acc_t = fmaf(w[k], qt[k], acc_t);
        if (refl)
          for (int k = 0; k < taps; ++k) acc_r = fmaf(w[k], qr[k], acc_r);
        dst[s] = make_float2(acc_r, acc_t);
      }
    }
  }
}

__device__ __forceinline__ void axial_psf_any(const float* pt, const float* pr, int NS, const float* w, int K,
                                              int lane, unsigned rmask, float2* dst) {
  switch (K) {
    case 1: axial_psf_rows<1>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 2: axial_psf_rows<2>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 3: axial_psf_rows<3>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 4: axial_psf_rows<4>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 5: axial_psf_rows<5>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 6: axial_psf_rows<6>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 7: axial_psf_rows<7>(pt, pr, NS, w, K, lane, rmask, dst); break;
    case 8: axial_psf_rows<8>(pt, pr, NS, w, K, lane, rmask, dst); break;
    default: axial_psf_rows<0>(pt, pr, NS, w, K, lane, rmask, dst); break;
  }
}

// Lateral PSF, image and log compression of rows w0 .. y1-1 of a pass-B
// tile over samples s0 .. s0 + kChunk, kLatLines lines per thread: abuf holds
// the staged filtered pairs (AR, AT) from w0 - K on (zero rows outside the
// frame and past the last needed row), ybuf the energy of rows w0 .. y1-1 and
// receives their log image in place; rows of kRowStride elements, of which
// the first kChunk + 1 are the tile's samples and one more.  Each line's taps
// are summed in increasing line order, for AR and AT alike; then
// I = image_value(P (x) AR, P (x) AT, E).
// KC > 0: K is the compile-time KC and the taps sit in registers; each
// staged row is read once and added into the (up to kLatLines) sums it
// reaches, in the same order.  KC = 0: any K, taps read from shared memory.
constexpr int kLatLines = 3;
template <int KC>
__device__ __forceinline__ void lateral_psf(const RenderParams& p, const DevProbe& P, long long beam_off,
                                            const float2* abuf, float* ybuf, const float* wlat, int NS, int K, int w0,
                                            int w1, int y1, int s0) {
  constexpr int NC = kChunk + 1;   // columns: the tile's samples and one more
  constexpr int LL = kLatLines;
  const int ng = (y1 - w0 + LL - 1) / LL;
  const int taps = 2 * K + 1;
  const int se = min(s0 + kChunk, NS);   // samples this tile exports
  constexpr int TC = 2 * KC + 1;
  float wr[KC > 0 ? TC : 1];
#pragma unroll
  for (int q = 0; q < (KC > 0 ? TC : 0); ++q) wr[q] = wlat[q];
  for (int t = threadIdx.x; t < ng * NC; t += blockDim.x) {
    const int gi = t / NC, c = t - gi * NC, i0 = LL * gi;
    const float2* col = abuf + i0 * kRowStride + c;    // row of line w0 + i0 + j, tap q: i0 + j + q
    float accR[LL], accT[LL];
#pragma unroll
    for (int j = 0; j < LL; ++j) accR[j] = accT[j] = 0.f;
    if constexpr (KC > 0) {
#pragma unroll
      for (int r = 0; r < TC + LL - 1; ++r) {
        const float2 v = col[r * kRowStride];
#pragma unroll
        for (int j = 0; j < LL; ++j)
          if (r - j >= 0 && r - j < TC) {
            accR[j] = fmaf(wr[r - j], v.x, accR[j]);
            accT[j] = fmaf(wr[r - j], v.y, accT[j]);
          }
      }
    } else {
      for (int q = 0; q < taps; ++q) {
        const float w = wlat[q];
        const float2* cp = col + q * kRowStride;
#pragma unroll
        for (int j = 0; j < LL; ++j) {
          const float2 v = cp[j * kRowStride];
          accR[j] = fmaf(w, v.x, accR[j]);
          accT[j] = fmaf(w, v.y, accT[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < LL; ++j) {
      const int i = i0 + j, l = w0 + i;
      if (l >= y1) break;
      float* yp = ybuf + i * kRowStride + c;
      const float I = image_value(accR[j], accT[j], *yp);
      const float y = log_compress(P, I);
      *yp = y;
      const int s = s0 + c;
      if (l < w1 && s < se) {
        if (p.envelope) p.envelope[beam_off + (long long)l * NS + s] = I;
        if (p.logimg) p.logimg[beam_off + (long long)l * NS + s] = y;
      }
    }
  }
}

__device__ __forceinline__ void lateral_psf_any(const RenderParams& p, const DevProbe& P, long long beam_off,
                                                const float2* abuf, float* ybuf, const float* wlat, int NS, int K,
                                                int w0, int w1, int y1, int s0) {
#define US_LAT(k) \
  case k: lateral_psf<k>(p, P, beam_off, abuf, ybuf, wlat, NS, K, w0, w1, y1, s0); break;
  switch (K) {
    US_LAT(2) US_LAT(3) US_LAT(4) US_LAT(5) US_LAT(6) US_LAT(7) US_LAT(8) US_LAT(9) US_LAT(10) US_LAT(11) US_LAT(12)
    default: lateral_psf<0>(p, P, beam_off, abuf, ybuf, wlat, NS, K, w0, w1, y1, s0); break;
  }
#undef US_LAT
}

struct SplitCtx {
  EnvItem it;
  DevProbe P;
  DevVolume V;
  DevPair pair;
  Pose M;
  int finite, valid;
};

// load the item of work unit `blk` (groups per item gpi) into shared memory;
// returns false (for the whole block) if the block has no work
__device__ __forceinline__ bool split_item(const RenderParams& p, const SplitArgs& a, int blk, int G, SplitCtx& cx,
                                           int& group) {
  const int n_items = p.n_items_dev ? *p.n_items_dev : p.n_items;
  int item;
  if (a.units) {
    const int2 u = a.units[blk];
    item = u.x;
    group = u.y;
  } else {
    item = blk / a.gpi_lines;
    group = blk - item * a.gpi_lines;
  }
  if (threadIdx.x == 0) {
    cx.valid = 0;
    if (item < n_items) {
      const EnvItem it = p.items[item];
      const DevProbe P = p.probes[it.probe];
      if (group * G < P.nl) {
        cx.it = it;
        cx.P = P;
        cx.V = p.vols[it.vol];
        cx.pair = p.pairs[it.pair];
        bool finite;
        cx.M = load_pose(p.poses, it.b, finite);
        cx.finite = finite;
        cx.valid = 1;
      }
    }
  }
  __syncthreads();
  return cx.valid != 0;
}

// minimum resident blocks per SM the register budget is cut for (64
// registers a thread): pass A holds two padded rows per line, so its blocks
// fit 4 (8 lines) or 2 (16 lines) to an SM on 512-sample probes
template <int G>
constexpr int lines_min_blocks() {
  return G == 8 ? 4 : (G == 16 ? 2 : 1);
}

// Pass A work unit `blk` = item * gpi_lines + group.  With a.done set,
// the unit then publishes its lines: done[blk] = 1 (release, after every
// thread's stores).
template <int G, bool ANCHORED>
__device__ __forceinline__ void lines_body(const RenderParams& p, const SplitArgs& a, int blk) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SplitCtx cx;
  int group;
  if (!split_item(p, a, blk, G, cx, group)) return;
  const DevProbe& P = cx.P;
  const int NL = P.nl, NS = P.ns, KA = P.k_ax;
  const int RS = lines_row_stride(NS, KA);
  const int g0 = group * G, g1 = min(g0 + G, NL);
  const int L0 = max(g0 - cx.pair.dmax, 0), L1 = min(g1 + cx.pair.dmax, NL);   // labels the stencil can reach
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NW = blockDim.x >> 5;
  float* zbuf = reinterpret_cast<float*>(smem);                      // [G][RS]: impedance, T, then P_ax (x) T
  float* rbuf = reinterpret_cast<float*>(smem + a.off_r);            // [G][RS]: R_imp, then P_ax (x) R_imp
  float* wax = reinterpret_cast<float*>(smem + a.off_wax);
  DevTissue* tis = reinterpret_cast<DevTissue*>(smem + a.off_tis);
  uint8_t* lbuf = smem + a.off_lab;                                   // [L1 - L0][NS]
  for (int t = tid; t < 2 * KA + 1; t += blockDim.x) wax[t] = __ldg(&P.w_ax[t]);
  for (int t = tid; t < p.n_labels; t += blockDim.x) tis[t] = P.tissue[t];
  if (!cx.finite && group == 0 && tid == 0) atomicOr(p.err, kErrNonFinitePose);
  __syncthreads();

  // labels and impedance of own lines g0 .. g1-1 (one line per warp), then
  // the halo lines' labels in 32-sample chunks spread over the warps: a line
  // d lines beyond the group is labelled only below ext[d], the stencil's
  // reach, so the short halo lines do not load a few warps
  // the label passes read the pose, volume and probe fields from register
  // copies: through the shared context they were reloaded for every sample
  // (2% of pass A)
  const Pose Mr = cx.M;
  const DevVolume Vr = cx.V;
  const DevProbe Pr = cx.P;
  auto label_of = [&](float2 ln, int s, float3& u, int& vi) -> uint8_t {
    float x, z;
    beam_point(Pr, ln, s, x, z);
    u = to_voxel(Mr, Vr.inv_h, x, z);
    return nearest_label(Vr, u, vi);
  };
  // Own lines take kLabU samples a lane per step (s, s + 32, ...): every
  // sample's label and corner-record loads are issued before any is used.
  constexpr int kLabU = 4;
  const bool cells = p.z_mode == 0 && cx.V.hu8 != nullptr;
  const bool exports = p.nn_index != nullptr || p.label != nullptr;   // debug exports
  for (int l = g0 + warp; l < g1; l += NW) {
    uint8_t* lrow = lbuf + (l - L0) * NS;
    float* prow = zbuf + (l - g0) * RS;
    const float2 ln = P.lines[l];
    for (int s = lane; s < NS; s += 32 * kLabU) {
      float3 u[kLabU];
      int vi[kLabU];
      uint8_t lb[kLabU];
      float zv[kLabU];
#pragma unroll
      for (int j = 0; j < kLabU; ++j) lb[j] = label_of(ln, s + 32 * j < NS ? s + 32 * j : s, u[j], vi[j]);
      if (cells) {
        HuCell c[kLabU];
#pragma unroll
        for (int j = 0; j < kLabU; ++j) c[j] = hu_cell_fetch(Vr, u[j]);
#pragma unroll
        for (int j = 0; j < kLabU; ++j) zv[j] = fmaxf(hu_cell_value(c[j]) + 1024.f, 1.f);
      } else {
#pragma unroll
        for (int j = 0; j < kLabU; ++j) zv[j] = p.z_mode == 0 ? fmaxf(trilinear_hu(cx.V, u[j]) + 1024.f, 1.f) : tis[lb[j]].z;
      }
#pragma unroll
      for (int j = 0; j < kLabU; ++j) {
        const int sj = s + 32 * j;
        if (sj < NS) {
          lrow[sj] = lb[j];
          prow[KA + sj] = zv[j];
        }
      }
      if (exports) {
#pragma unroll
        for (int j = 0; j < kLabU; ++j) {
          const int sj = s + 32 * j;
          if (sj < NS && p.nn_index) p.nn_index[cx.it.beam_off + (long long)l * NS + sj] = vi[j];
          if (sj < NS && p.label) p.label[cx.it.beam_off + (long long)l * NS + sj] = lb[j];
        }
      }
    }
    float* rrow = rbuf + (l - g0) * RS;
    for (int q = lane; q < KA; q += 32) {
      prow[q] = 0.f;
      prow[KA + NS + q] = 0.f;
      rrow[q] = 0.f;
      rrow[KA + NS + q] = 0.f;
    }
    if (lane == 0) {   // the element past the padded row, read by the two-output filter
      prow[2 * KA + NS] = 0.f;
      rrow[2 * KA + NS] = 0.f;
    }
  }
  {
    // two 32-sample units a warp per step, both loads issued first
    const int nl_left = g0 - L0, nh = nl_left + (L1 - g1), cpl = (NS + 31) >> 5, nu = nh * cpl;
    // t / nh as floor((t + 1/2) / nh) in FP32: (t + 1/2) / nh lies at least
    // 1 / (2 nh) from an integer and below cpl <= 32, far beyond the
    // product's rounding error, so the quotient is exact
    const float inv_nh = 1.f / (float)max(nh, 1);
    for (int t0 = warp; t0 < nu; t0 += 2 * NW) {
      int at[2];
      uint8_t lv[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int t = t0 + j * NW;
        at[j] = -1;
        lv[j] = 0;
        if (t < nu) {
          const int c = __float2int_rz(((float)t + 0.5f) * inv_nh), h = t - c * nh;
          const int l = h < nl_left ? L0 + h : g1 + (h - nl_left);
          const int lim = cx.pair.ext[l < g0 ? g0 - l : l - g1 + 1];
          const int s = (c << 5) + lane;
          if (s < lim) {
            float3 u;
            int vi;
            at[j] = (l - L0) * NS + s;
            lv[j] = label_of(P.lines[l], s, u, vi);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (at[j] >= 0) lbuf[at[j]] = lv[j];
    }
  }
  __syncthreads();

  // scanline model and axial PSF of own lines, one warp per line; the
  // energy goes straight to the line buffer's E plane
  for (int l = g0 + warp; l < g1; l += NW) {
    float* prow = zbuf + (l - g0) * RS;
    float* row = prow + KA;
    float* rrow = rbuf + (l - g0) * RS;
    float* erow = a.ebeam + cx.it.beam_off + (long long)l * NS;
    const uint8_t* lrow = lbuf + (l - L0) * NS;
    auto labf = [&](int line, int s) -> unsigned { return lbuf[(line - L0) * NS + s]; };
    auto own = [&](int s) -> unsigned { return lrow[s]; };
    auto zf = [&](int s) -> float { return row[s]; };
    const float2 ln = P.lines[l];
    auto posf = [&](int s) -> float3 {
      float x, z;
      beam_point(P, ln, s, x, z);
      return sample_position(cx.M, x, z);
    };
    unsigned rmask = 0;   // this lane's 32-sample chunks with a non-zero reflection impulse
    scanline_model<ANCHORED>(p, P, tis, cx.pair, cx.it.b, l, lane, labf, own, zf,
                             [&](int s, float r, float t, float e) {
                               row[s] = t;
                               rrow[KA + s] = r;
                               erow[s] = e;
                               if (r != 0.f) rmask |= 1u << (s >> 5);
                             },
                             posf, cx.it.vol);
    rmask = __reduce_or_sync(kFull, rmask);
    __syncwarp();
    axial_psf_any(prow, rrow, NS, wax, KA, lane, rmask, a.beam + cx.it.beam_off + (long long)l * NS);
  }
  if (a.done) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a.done + blk), "r"(1u) : "memory");
    }
  }
}

template <int G, bool ANCHORED>
__global__ void __launch_bounds__(G * 32, lines_min_blocks<G>()) split_lines(RenderParams p, SplitArgs a) {
  lines_body<G, ANCHORED>(p, a, blockIdx.x);
}

// Pass B tile: GB lines x kChunk samples of one environment.  The block
// stages the filtered lines of its lines (plus one for the bilinear step
// and the lateral PSF's reach) over its samples plus one, forms the log
// image there and writes the pixels whose bilinear base (line, sample)
// falls in the tile.
// Pass B work unit `blk` = item * gpi_image + tile, run by NT threads.
// With a.done set, the unit first waits (bounded) until the pass-A groups
// holding its staged rows have published them.
// One pass-B tile: its environment, lines and samples.
struct TileCtx {
  EnvItem it;
  const DevProbe* P;
  int item, tile, NL, NS, KL;
  int w0, w1, y1;   // wedge lines w0 .. w1-1; log rows w0 .. y1-1
  int s0, sw;       // staged samples s0 .. s0+sw-1
  int r0, nrows;    // staged rows r0 .. r0+nrows-1 (zero outside the frame)
  int a0, a1;       // rows present in the line buffer
};

// the tile of pass-B unit `blk`; false if the unit has no work (past the
// item count or past its probe's tiles).  Every thread reads the same
// addresses (broadcast loads); the result is uniform over the block.
__device__ __forceinline__ bool tile_ctx(const RenderParams& p, const SplitArgs& a, int blk, TileCtx& t) {
  const int n_items = p.n_items_dev ? *p.n_items_dev : p.n_items;
  if (a.units) {
    const int2 u = a.units[a.n_units_a + blk];
    t.item = u.x;
    t.tile = u.y;
  } else {
    t.item = blk / a.gpi_image;
    t.tile = blk - t.item * a.gpi_image;
  }
  if (t.item >= n_items) return false;
  t.it = p.items[t.item];
  t.P = &p.probes[t.it.probe];
  t.NL = t.P->nl;
  t.NS = t.P->ns;
  t.KL = t.P->k_lat;
  const int nchunk = (t.NS + kChunk - 1) / kChunk;
  const int q = t.tile / nchunk, k = t.tile - q * nchunk;
  t.w0 = q * a.GB;
  if (t.w0 >= t.NL) return false;
  t.w1 = min(t.w0 + a.GB, t.NL);
  t.y1 = min(t.w1 + 1, t.NL);
  t.s0 = k * kChunk;
  t.sw = min(kChunk + 1, t.NS - t.s0);
  // zero rows outside the frame, past the last needed row and past the
  // line's end, so that the lateral PSF needs no edge tests (adding w * 0
  // leaves a sum unchanged exactly: the sums never hold -0)
  t.r0 = t.w0 - t.KL;
  t.nrows = (((t.y1 - t.w0) + kLatLines - 1) / kLatLines) * kLatLines + 2 * t.KL;
  t.a0 = max(t.r0, 0);
  t.a1 = min(t.y1 + t.KL, t.NL);
  return true;
}

// Stage a tile into shared memory: the lateral taps (plain stores), the
// (AR, AT) rows and the wedge's energies, as 16-byte cp.async copies where
// the rows are 16-byte aligned (zero-filled past a row's end and for rows
// outside the frame), else plain loads.  Commits one cp.async group in
// every case; the caller waits for it.
__device__ __forceinline__ void tile_stage(const SplitArgs& a, const TileCtx& t, float2* abuf, float* ybuf,
                                           float* wlat, int tid, int NT) {
  for (int i = tid; i < 2 * t.KL + 1; i += NT) wlat[i] = __ldg(&t.P->w_lat[i]);
  const float2* src = a.beam + t.it.beam_off + t.s0;
  const float* esrc = a.ebeam + t.it.beam_off + t.s0;
  const int ne = t.y1 - t.w0, NS = t.NS;
  if ((NS & 3) == 0 && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) &&
      ((reinterpret_cast<uintptr_t>(esrc) & 15u) == 0)) {
    constexpr int PPA = kRowStride / 2;                            // 16-byte pieces per pair row
    for (int i = tid; i < t.nrows * PPA; i += NT) {
      const int r = i / PPA, c = (i - r * PPA) * 2;
      const int line = t.r0 + r;
      const bool present = line >= t.a0 && line < t.a1 && c < t.sw;
      const float2* g = present ? src + (long long)line * NS + c : a.beam;
      umma::cp_async16(abuf + r * kRowStride + c, g, present ? 16u : 0u);
    }
    constexpr int PPE = kRowStride / 4;                            // 16-byte pieces per energy row
    for (int i = tid; i < ne * PPE; i += NT) {
      const int r = i / PPE, c = (i - r * PPE) * 4;
      const bool present = c < t.sw;
      const float* g = present ? esrc + (long long)(t.w0 + r) * NS + c : a.ebeam;
      umma::cp_async16(ybuf + r * kRowStride + c, g, present ? 16u : 0u);
    }
  } else {
    for (int i = tid; i < t.nrows * kRowStride; i += NT) {
      const int r = i / kRowStride, c = i - r * kRowStride;
      const int line = t.r0 + r;
      abuf[i] = line >= t.a0 && line < t.a1 && c < t.sw ? __ldcg(src + (long long)line * NS + c) : make_float2(0.f, 0.f);
    }
    for (int i = tid; i < ne * kRowStride; i += NT) {
      const int r = i / kRowStride, c = i - r * kRowStride;
      ybuf[i] = c < t.sw ? __ldcg(esrc + (long long)(t.w0 + r) * NS + c) : 0.f;
    }
  }
  umma::cp_async_commit();
}

// A staged tile (visible to the block): lateral PSF, log image, then the
// frame's pixels whose bilinear base falls in the tile.
template <int NT>
__device__ __forceinline__ void tile_compute(const RenderParams& p, const TileCtx& t, const float2* abuf, float* ybuf,
                                             const float* wlat, int tid) {
  const DevProbe& P = *t.P;
  const int NL = t.NL, NS = t.NS, w0 = t.w0, w1 = t.w1, s0 = t.s0;
  lateral_psf_any(p, P, t.it.beam_off, abuf, ybuf, wlat, NS, t.KL, w0, w1, t.y1, s0);
  __syncthreads();
  float* out = p.frames + t.it.frame_off;
  const int se = min(s0 + kChunk, NS);
  if (P.kind == 0) {
    // one line a lane (wedges are at most 32 lines), one sample a warp row
    static_assert(NT % 32 == 0, "whole warps");
    const int wl = w1 - w0, j = tid & 31;
    if (j < wl)
      for (int s = tid >> 5; s < se - s0; s += NT >> 5)
        __stcs(&out[(long long)(s0 + s) * NL + w0 + j], ybuf[j * kRowStride + s]);
  } else {
    // kPixU pixels a thread per step, their list entries loaded before any is used
    constexpr int kPixU = 4;
    const int e0 = P.wedge_off[t.tile], e1 = P.wedge_off[t.tile + 1];
    for (int e = e0 + tid; e < e1; e += kPixU * NT) {
      float4 qv[kPixU];
#pragma unroll
      for (int u = 0; u < kPixU; ++u)
        qv[u] = e + u * NT < e1 ? __ldg(&P.wedge[e + u * NT]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kPixU; ++u) {
        if (e + u * NT >= e1) break;
        const int pix = __float_as_int(qv[u].x);
        const float fl = qv[u].y, fs = qv[u].z;
        float v = 0.f;
        if (fl >= 0.f) {
          const int la = min((int)fl, NL - 2), sa = min((int)fs, NS - 2);
          const float al = fl - (float)la, bb = fs - (float)sa;
          const float* r0p = ybuf + (la - w0) * kRowStride + (sa - s0);
          const float* r1p = r0p + kRowStride;
          const float y00 = r0p[0], y01 = r0p[1];
          const float y10 = r1p[0], y11 = r1p[1];
          const float top = fmaf(al, y10 - y00, y00), bot = fmaf(al, y11 - y01, y01);
          v = fmaf(bb, bot - top, top);
        }
        __stcs(&out[pix], v);
      }
    }
  }
}

template <int NT>
__device__ __forceinline__ void image_body(const RenderParams& p, const SplitArgs& a, int blk) {
  extern __shared__ __align__(16) unsigned char smem[];
  TileCtx t;
  if (!tile_ctx(p, a, blk, t)) return;   // uniform over the block
  const int tid = threadIdx.x;
  if (a.done) {
    __shared__ int ready;
    if (tid == 0) {
      ready = 1;
      const int G = a.G;
      for (int g = t.a0 / G; g <= (t.a1 - 1) / G && ready; ++g) {
        const unsigned* f = a.done + (long long)t.item * a.gpi_lines + g;
        const long long t0 = clock64();
        unsigned v;
        for (;;) {
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
          if (v) break;
          if (clock64() - t0 > a.wait_cycles) {
            atomicOr(p.err, kErrStagingTimeout);
            ready = 0;
            break;
          }
          __nanosleep(200);
        }
      }
    }
    __syncthreads();
    if (!ready) return;
  }
  float2* abuf = reinterpret_cast<float2*>(smem);                    // [nrows][kRowStride] (AR, AT)
  float* ybuf = reinterpret_cast<float*>(smem + a.off_y);            // [y1 - w0][kRowStride]: E, then the log image
  float* wlat = reinterpret_cast<float*>(smem + a.off_wlat);
  tile_stage(a, t, abuf, ybuf, wlat, tid, NT);
  umma::cp_async_wait<0>();
  __syncthreads();
  tile_compute<NT>(p, t, abuf, ybuf, wlat, tid);
}

__global__ void __launch_bounds__(kImageThreads, 4) split_image(RenderParams p, SplitArgs a) {
  image_body<kImageThreads>(p, a, blockIdx.x);
}

// Both passes in one persistent grid (one block per resident slot): blocks
// take work units from a counter, all pass-A groups first, then the pass-B
// tiles in environment order; a tile waits only for the groups holding its
// rows, all of which were taken earlier by blocks that are running and wait
// on nothing, so every wait ends.  Pass B's tiles fill pass A's last wave.
template <int G, bool ANCHORED>
__global__ void __launch_bounds__(G * 32, lines_min_blocks<G>()) split_persist(RenderParams p, SplitArgs a) {
  __shared__ int job;
  const int n_items = p.n_items_dev ? *p.n_items_dev : p.n_items;
  const int na = n_items * a.gpi_lines, nb = n_items * a.gpi_image;
  for (;;) {
    if (threadIdx.x == 0) job = (int)atomicAdd(a.work, 1u);
    __syncthreads();
    const int j = job;
    if (j >= na + nb) break;
    if (j < na)
      lines_body<G, ANCHORED>(p, a, j);
    else
      image_body<G * 32>(p, a, j - na);
    __syncthreads();   // shared memory and `job` are reused by the next unit
  }
}

bool split_shape_fits(SplitShape& sh, const std::vector<ProbeHost>& probes, int n_labels) {
  const int G = sh.G;
  if (G != 8 && G != 16 && G != 32) return false;
  auto up = [](long long x, long long a) { return (x + a - 1) / a * a; };
  const size_t lim = 227 * 1024 - 1024;
  // pass A
  long long zb = 0, lab = 0;
  int gl = 0;
  for (const ProbeHost& ph : probes) {
    const int NL = ph.desc.n_lines, NS = ph.desc.n_samples;
    const int rs = lines_row_stride(NS, ph.k_ax);
    zb = std::max(zb, (long long)G * rs * 4);
    lab = std::max(lab, (long long)std::min(NL, G + 2 * kThetaDMax) * NS);
    gl = std::max(gl, (NL + G - 1) / G);
  }
  long long off = up(zb, 16);
  sh.args.off_r = (int)off;
  off = up(off + zb, 16);
  sh.args.off_wax = (int)off;
  off = up(off + 4 * (2 * 32 + 1), 16);
  sh.args.off_tis = (int)off;
  off = up(off + (long long)sizeof(DevTissue) * n_labels, 16);
  sh.args.off_lab = (int)off;
  off = up(off + lab, 16);
  sh.smem_lines = (size_t)off;
  if (sh.smem_lines > lim) return false;
  // pass B: the widest wedge whose staged pair rows (8 bytes a sample) and
  // energy / log rows (kChunk + 1 samples each) fit four blocks per SM,
  // else three, two, one
  for (int per_sm : {4, 3, 2, 1})
  for (int GB : {32, 16, 8}) {
    if (sh.GB_req && GB != sh.GB_req) continue;
    long long ab = 0, yb = 0;
    int gi = 0;
    for (const ProbeHost& ph : probes) {
      const int NL = ph.desc.n_lines, NS = ph.desc.n_samples;
      const int rows = ((std::min(NL, GB + 1) + kLatLines - 1) / kLatLines) * kLatLines + 2 * ph.k_lat;
      ab = std::max(ab, (long long)rows * kRowStride * 8);
      yb = std::max(yb, (long long)std::min(NL, GB + 1) * kRowStride * 4);
      gi = std::max(gi, ((NL + GB - 1) / GB) * ((NS + kChunk - 1) / kChunk));
    }
    long long o = up(ab, 16);
    const int off_y = (int)o;
    o = up(o + yb, 16);
    const int off_wlat = (int)o;
    o = up(o + 4 * (2 * kMaxHalfTaps + 1), 16);
    if ((size_t)o <= std::min(lim, (size_t)(228 * 1024) / per_sm - 1024 - 64)) {
      sh.GB = GB;
      sh.smem_image = (size_t)o;
      sh.args.off_y = off_y;
      sh.args.off_wlat = off_wlat;
      sh.args.G = G;
      sh.args.GB = GB;
      sh.args.gpi_lines = gl;
      sh.args.gpi_image = gi;
      return true;
    }
  }
  return false;
}

// pass 0: split_lines<G>, pass 1: split_image; split_persist<G> takes the
// larger of the two shared-memory sizes
template <int G>
static cudaError_t prepare_g(SplitShape& sh) {
  const int sm = (int)std::max(sh.smem_lines, sh.smem_image);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(split_lines<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sh.smem_lines)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(split_lines<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sh.smem_lines)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(split_image, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem_image)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(split_persist<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(split_persist<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
          cudaSuccess)
    return e;
  int dev = 0, n_sm = 0, b0 = 0, b1 = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, split_persist<G, false>, G * 32, sm)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, split_persist<G, true>, G * 32, sm)) != cudaSuccess)
    return e;
  sh.persist_grid[0] = b0 * n_sm;
  sh.persist_grid[1] = b1 * n_sm;
  return (b0 > 0 && b1 > 0) ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t split_prepare(SplitShape& sh) {
  switch (sh.G) {
    case 8: return prepare_g<8>(sh);
    case 16: return prepare_g<16>(sh);
    case 32: return prepare_g<32>(sh);
    default: return cudaErrorInvalidValue;
  }
}

template <int G>
static cudaError_t launch_g(const RenderParams& p, const SplitShape& sh, const SplitArgs& a, int max_items, int pass,
                            cudaStream_t st) {
  const unsigned grid_a = a.units ? (unsigned)a.n_units_a : (unsigned)(max_items * a.gpi_lines);
  const unsigned grid_b = a.units ? (unsigned)a.n_units_b : (unsigned)(max_items * a.gpi_image);
  if ((pass == 0 && grid_a == 0) || (pass == 1 && grid_b == 0)) return cudaSuccess;
  if (pass == 0 && p.speckle_anchor)
    split_lines<G, true><<<grid_a, G * 32, sh.smem_lines, st>>>(p, a);
  else if (pass == 0)
    split_lines<G, false><<<grid_a, G * 32, sh.smem_lines, st>>>(p, a);
  else if (pass == 1)
    split_image<<<grid_b, kImageThreads, sh.smem_image, st>>>(p, a);
  else {
    // persistent: as many blocks as are resident at once (launched as a
    // cooperative grid, so they all are), no more than there are units
    const int units = max_items * (a.gpi_lines + a.gpi_image);
    const int grid = std::max(1, std::min(units, sh.persist_grid[p.speckle_anchor ? 1 : 0]));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(G * 32);
    cfg.dynamicSmemBytes = std::max(sh.smem_lines, sh.smem_image);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return p.speckle_anchor ? cudaLaunchKernelEx(&cfg, split_persist<G, true>, p, a)
                            : cudaLaunchKernelEx(&cfg, split_persist<G, false>, p, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_pass(const RenderParams& p, const SplitShape& sh, float* beam, long long beam_elems,
                              unsigned* sync, int max_items, int pass, cudaStream_t st, SplitUnits units) {
  SplitArgs a = sh.args;
  set_line_buffer(a, beam, beam_elems);
  if (pass < 2 && units.d) {
    a.units = units.d;
    a.n_units_a = units.n_a;
    a.n_units_b = units.n_b;
  }
  if (pass >= 2) {
    // sync: the unit counter, then one completion flag per pass-A group
    // (pass 3: the caller has zeroed them)
    if (pass == 2) {
      cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(unsigned) * (1 + (size_t)max_items * a.gpi_lines), st);
      if (e != cudaSuccess) return e;
    }
    a.work = sync;
    a.done = sync + 1;
    pass = 2;
  }
  switch (sh.G) {
    case 8: return launch_g<8>(p, sh, a, max_items, pass, st);
    case 16: return launch_g<16>(p, sh, a, max_items, pass, st);
    case 32: return launch_g<32>(p, sh, a, max_items, pass, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_split_wait_selftest(const RenderParams& p, const SplitShape& sh, float* beam, long long beam_elems,
                                       unsigned* sync, int max_items, long long wait_cycles, cudaStream_t st) {
  SplitArgs a = sh.args;
  set_line_buffer(a, beam, beam_elems);
  a.work = sync;
  a.done = sync + 1;
  a.wait_cycles = wait_cycles;
  const unsigned start = (unsigned)(max_items * a.gpi_lines);
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(unsigned) * (1 + (size_t)max_items * a.gpi_lines), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sync, &start, sizeof start, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // `start` lives on this stack frame
  if (e != cudaSuccess) return e;
  switch (sh.G) {
    case 8: return launch_g<8>(p, sh, a, max_items, 2, st);
    case 16: return launch_g<16>(p, sh, a, max_items, 2, st);
    case 32: return launch_g<32>(p, sh, a, max_items, 2, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_split(const RenderParams& p, const SplitShape& sh, float* beam, long long beam_elems, unsigned* sync,
                         int max_items, cudaStream_t st, SplitUnits units) {
  if (sh.persistent) return launch_split_pass(p, sh, beam, beam_elems, sync, max_items, 2, st);
  cudaError_t e = launch_split_pass(p, sh, beam, beam_elems, sync, max_items, 0, st, units);
  return e == cudaSuccess ? launch_split_pass(p, sh, beam, beam_elems, sync, max_items, 1, st, units) : e;
}

// the work units of a list of items (items in launch order) for a shape:
// pass A (item, group) for the probe's groups, pass B (item, tile) for its
// wedges x chunks
void build_split_units(const std::vector<EnvItem>& items, const std::vector<ProbeHost>& probes, int G, int GB,
                       std::vector<int2>& units, int& na, int& nb) {
  units.clear();
  for (int i = 0; i < (int)items.size(); ++i) {
    const int NL = probes[items[i].probe].desc.n_lines;
    for (int g = 0; g * G < NL; ++g) units.push_back(make_int2(i, g));
  }
  na = (int)units.size();
  for (int i = 0; i < (int)items.size(); ++i) {
    const us_probe& d = probes[items[i].probe].desc;
    const int nchunk = (d.n_samples + kChunk - 1) / kChunk, nq = (d.n_lines + GB - 1) / GB;
    for (int t = 0; t < nq * nchunk; ++t) units.push_back(make_int2(i, t));
  }
  nb = (int)units.size() - na;
}

// Pixels of a curvilinear probe's output grid, grouped by pass-B tile
// (wedge of G lines x chunk of kChunk samples), tile = wedge * chunks +
// chunk: a pixel inside the fan belongs to the tile of its bilinear base
// (min(floor(fl), NL - 2), min(floor(fs), NS - 2)); a pixel outside the
// fan to the tile of the preceding inside pixel of its row (tile 0 if
// none).  Within a tile, pixels keep raster order.
void build_wedges(const std::vector<float2>& lut, int W, int H, int NL, int NS, int G, std::vector<float4>& entries,
                  std::vector<int>& off) {
  const int nchunk = (NS + kChunk - 1) / kChunk;
  const int nt = ((NL + G - 1) / G) * nchunk;
  std::vector<std::vector<float4>> per(nt);
  for (int r = 0; r < H; ++r) {
    int t = 0;
    for (int c = 0; c < W; ++c) {
      const float2 f = lut[(size_t)r * W + c];
      if (f.x >= 0.f) t = (std::min((int)f.x, NL - 2) / G) * nchunk + std::min((int)f.y, NS - 2) / kChunk;
      const int pix = r * W + c;
      float4 e;
      std::memcpy(&e.x, &pix, sizeof pix);
      e.y = f.x;
      e.z = f.y;
      e.w = 0.f;
      per[t].push_back(e);
    }
  }
  entries.clear();
  off.assign(nt + 1, 0);
  for (int t = 0; t < nt; ++t) {
    off[t] = (int)entries.size();
    entries.insert(entries.end(), per[t].begin(), per[t].end());
  }
  off[nt] = (int)entries.size();
}

}  // namespace ussim
