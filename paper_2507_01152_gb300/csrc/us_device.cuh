// Device-side data structures and per-sample helpers of the ultrasound
// render (SonoGym App. B.2 image model on the probe's scanline grid).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ussim {

constexpr int kMaxHalfTaps = 48;   // PSF half-width limit (taps <= 97)
constexpr int kThetaDMax = 8;      // lateral reach of the incidence stencil, lines
constexpr int kMaxSpeckleLevels = 3;   // scales of the volume-anchored scatter maps

// error-word bits
constexpr unsigned kErrNonFinitePose = 1u;
constexpr unsigned kErrBadItem = 2u;
constexpr unsigned kErrStagingTimeout = 8u;   // an asynchronous copy into shared memory did not complete

struct DevVolume {
  const uint8_t* labels;
  const int16_t* hu;
  int nx, ny, nz;
  float inv_h;
  float h;   // voxel edge, mm (as given)
  // Corner records of the HU grid, or null: one 16-byte record per cell
  // (i, j, k), the cell based at voxel (i, j, k) for i in [-1, nx-1]
  // (likewise j, k), holding the HU of its 8 corners as int16 in the order
  // c000 c100 c010 c110 c001 c101 c011 c111 (bit 0 of the corner index = x),
  // 0 outside the grid: one 16-byte load per trilinear sample instead of
  // eight gathers.  Records go in quads along y (with J = j + 1, I = i + 1,
  // K = k + 1: record ((K qy + J/4)(nx + 1) + I) 4 + J%4, qy = ceil((ny+1)/4)),
  // so that one 64-byte DRAM fetch holds four cells in y: an image plane
  // whose depth runs along y reads most of them.
  const uint4* hu8;
  int qy;
  // Labels in 4 x 4 x 4 bricks of 64 bytes, or null: voxel (i, j, k) at byte
  // ((k/4 by + j/4) bx + i/4) 64 + (k%4) 16 + (j%4) 4 + i%4, bx = ceil(nx/4),
  // by = ceil(ny/4), 0 in the padding.  A 64-byte fetch then holds a
  // 4 x 4 x 4 neighbourhood that an oblique plane crosses, where a row-major
  // fetch holds 64 voxels of one row.
  const uint8_t* lab4;
  int bx, by;
};

// per (probe, label): attenuation per sample f*alpha*dr (Np), scatter
// statistics, table impedance, and the N1 threshold floor(Phi(mu1) 2^32)
struct DevTissue {
  float att, mu0, sigma0, z;
  unsigned long long t1;
  float mu1;   // density threshold on N1 (anchored maps compare N1 itself)
};

struct DevProbe {
  int kind, nl, ns, out_w, out_h;
  int k_ax, k_lat;
  float dr, r0, e0, log_gain, dtheta, pitch;
  float db_e0;               // 20 log10(e0)
  const float2* lines;       // [nl]: linear (x_l, 0), curvilinear (sin, cos)
  const float* w_ax;         // [2 k_ax + 1]
  const float* w_lat;        // [2 k_lat + 1]
  const float2* lut;         // curvilinear: [out_h * out_w] (fl, fs); fl < 0 outside
  const DevTissue* tissue;   // [n_labels]
  const float* px;           // curvilinear: [out_w] probe-frame x of output pixel columns
  const float* pz;           // curvilinear: [out_h] probe-frame z of output pixel rows
  const float4* wedge;       // curvilinear, two-pass path: (pixel bits, fl, fs, 0) grouped by wedge
  const int* wedge_off;      // [wedges + 1] start of each wedge's pixels
};

// incidence stencil extents for a (volume, probe) pair: axial half window W
// and per-sample lateral reach D[s]
struct DevPair {
  int W;
  const uint8_t* D;
  int dmax;   // max over samples of D: the stencil's lateral reach for this pair
  // ext[d], d = 1..dmax: the stencil reads a line d lines away from the
  // line it serves only at samples below ext[d] (the window's end past the
  // deepest sample s with D[s] >= d)
  int ext[kThetaDMax + 1];
};

// one environment of a batch, in processing order
struct EnvItem {
  int b;            // index in the caller's batch (noise counter, pose)
  int vol, probe;
  int pair;         // vol * n_probes + probe
  long long frame_off, beam_off;
};

struct RenderParams {
  const DevVolume* vols;
  const DevProbe* probes;
  const DevPair* pairs;
  const EnvItem* items;
  int n_items;
  const int* n_items_dev;    // if set, the item count is read here (device-built work lists)
  int n_labels;
  const float* poses;        // [B][12]
  uint2 key;                 // Philox key for this (seed, step)
  int refl_power, transmission, z_mode, speckle;
  int speckle_anchor, speckle_levels;          // volume-anchored scatter maps
  float inv_cell[kMaxSpeckleLevels];           // 1 / (cell edge c 2^k), FP32
  float amp[kMaxSpeckleLevels];                // a_k, sum a_k^2 = 1
  uint2 key_fixed;                             // Philox key of the anchored maps (seed only)
  float* frames;
  float* envelope;           // debug exports, may be null
  float* logimg;
  int* nn_index;
  uint8_t* label;
  unsigned* err;
  unsigned* work;            // work counter (fused path)
};

// ------------------------------------------------------------------ Philox
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 multiplies on counter words 0 and 2, high halves mixed with the
// other words and the round key, key bumped by two Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// uniform in (0,1): odd multiple of 2^-24 from the top 23 bits k = w >> 9,
// (2k + 1) 2^-24, formed exactly as (1 + k 2^-23) - (1 - 2^-24): the float
// with exponent 0 and mantissa k, less a constant; the difference is
// representable, so the subtraction is exact
__device__ __forceinline__ float u01(unsigned w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) - 0.999999940395355224609375f;
}

// ---------------------------------------------------------- index path
// The voxel coordinate of a beam sample is defined in FP32 with a fixed,
// contraction-free order; __fmul_rn / __fadd_rn keep the compiler from
// fusing it into FMAs so that nearest-voxel decisions are reproducible.
__device__ __forceinline__ void beam_point(const DevProbe& P, float2 ln, int s, float& x, float& z) {
  const float sf = (float)s;
  if (P.kind == 0) {
    x = ln.x;
    z = __fmul_rn(sf, P.dr);
  } else {
    const float rho = __fadd_rn(P.r0, __fmul_rn(sf, P.dr));
    x = __fmul_rn(rho, ln.x);
    z = __fadd_rn(__fmul_rn(rho, ln.y), -P.r0);
  }
}

struct Pose {
  float m[12];
};

// volume-frame position (mm) of a probe-frame point (x, 0, z)
__device__ __forceinline__ float3 sample_position(const Pose& M, float x, float z) {
  float3 p;
  p.x = __fadd_rn(__fadd_rn(__fmul_rn(M.m[0], x), __fmul_rn(M.m[2], z)), M.m[3]);
  p.y = __fadd_rn(__fadd_rn(__fmul_rn(M.m[4], x), __fmul_rn(M.m[6], z)), M.m[7]);
  p.z = __fadd_rn(__fadd_rn(__fmul_rn(M.m[8], x), __fmul_rn(M.m[10], z)), M.m[11]);
  return p;
}

__device__ __forceinline__ float3 to_voxel(const Pose& M, float inv_h, float x, float z) {
  const float3 p = sample_position(M, x, z);
  return make_float3(__fmul_rn(p.x, inv_h), __fmul_rn(p.y, inv_h), __fmul_rn(p.z, inv_h));
}

// nearest voxel: floor(u + 1/2) per axis; false outside the grid (NaN -> outside)
__device__ __forceinline__ bool nearest_ijk(const DevVolume& V, float3 u, int& i, int& j, int& k) {
  const float fx = floorf(__fadd_rn(u.x, 0.5f));
  const float fy = floorf(__fadd_rn(u.y, 0.5f));
  const float fz = floorf(__fadd_rn(u.z, 0.5f));
  if (!(fx >= 0.f && fx < (float)V.nx && fy >= 0.f && fy < (float)V.ny && fz >= 0.f && fz < (float)V.nz))
    return false;
  i = (int)fx;
  j = (int)fy;
  k = (int)fz;
  return true;
}

// linear index of the nearest voxel, -1 outside the grid
__device__ __forceinline__ int nearest_voxel(const DevVolume& V, float3 u) {
  int i, j, k;
  return nearest_ijk(V, u, i, j, k) ? (k * V.ny + j) * V.nx + i : -1;
}

// label of voxel (i, j, k) inside the grid
__device__ __forceinline__ uint8_t label_at(const DevVolume& V, int i, int j, int k) {
  if (V.lab4)
    return __ldg(&V.lab4[((((k >> 2) * V.by + (j >> 2)) * V.bx + (i >> 2)) << 6) | ((k & 3) << 4) | ((j & 3) << 2) |
                         (i & 3)]);
  return __ldg(&V.labels[(k * V.ny + j) * V.nx + i]);
}

// label of the nearest voxel (0 outside the grid) and its linear index vi
// (-1 outside)
__device__ __forceinline__ uint8_t nearest_label(const DevVolume& V, float3 u, int& vi) {
  int i, j, k;
  if (!nearest_ijk(V, u, i, j, k)) {
    vi = -1;
    return 0;
  }
  vi = (k * V.ny + j) * V.nx + i;
  return label_at(V, i, j, k);
}

__device__ __forceinline__ float hu_at(const DevVolume& V, int i, int j, int k) {
  return ((unsigned)i < (unsigned)V.nx && (unsigned)j < (unsigned)V.ny && (unsigned)k < (unsigned)V.nz)
             ? (float)__ldg(&V.hu[(k * V.ny + j) * V.nx + i])
             : 0.f;
}

// the trilinear blend of a cell's 8 corner values at fractions (tx, ty, tz),
// in one fixed order
__device__ __forceinline__ float trilinear_blend(float tx, float ty, float tz, float c000, float c100, float c010,
                                                 float c110, float c001, float c101, float c011, float c111) {
  const float a00 = fmaf(tx, c100 - c000, c000), a10 = fmaf(tx, c110 - c010, c010);
  const float a01 = fmaf(tx, c101 - c001, c001), a11 = fmaf(tx, c111 - c011, c011);
  const float b0 = fmaf(ty, a10 - a00, a00), b1 = fmaf(ty, a11 - a01, a01);
  return fmaf(tz, b1 - b0, b0);
}

// Trilinear HU from the corner records in two steps, so that a caller can
// issue the loads of several samples before it blends any: hu_cell_fetch
// loads the sample's record (V.hu8 must be set), hu_cell_value blends it.
// Together they compute exactly what trilinear_hu computes.
struct HuCell {
  uint4 q;
  float tx, ty, tz;
  bool in;   // false: the cell lies outside the grid, the value is 0
};
__device__ __forceinline__ HuCell hu_cell_fetch(const DevVolume& V, float3 u) {
  const float fx = floorf(u.x), fy = floorf(u.y), fz = floorf(u.z);
  HuCell c;
  c.in = fx >= -1.f && fx < (float)V.nx && fy >= -1.f && fy < (float)V.ny && fz >= -1.f && fz < (float)V.nz;
  c.tx = u.x - fx;
  c.ty = u.y - fy;
  c.tz = u.z - fz;
  c.q = make_uint4(0u, 0u, 0u, 0u);
  if (c.in) {
    const int i = (int)fx, j = (int)fy, k = (int)fz;
    c.q = __ldg(&V.hu8[((((k + 1) * V.qy + ((j + 1) >> 2)) * (V.nx + 1) + (i + 1)) << 2) | ((j + 1) & 3)]);
  }
  return c;
}
__device__ __forceinline__ float hu_cell_value(const HuCell& c) {
  if (!c.in) return 0.f;
  // the sign-extended halves of each word are the int16 corner values
  const uint4 q = c.q;
  return trilinear_blend(c.tx, c.ty, c.tz, (float)((int)(q.x << 16) >> 16), (float)((int)q.x >> 16),
                         (float)((int)(q.y << 16) >> 16), (float)((int)q.y >> 16), (float)((int)(q.z << 16) >> 16),
                         (float)((int)q.z >> 16), (float)((int)(q.w << 16) >> 16), (float)((int)q.w >> 16));
}

// trilinear HU; corners outside the grid read 0 (water).  Interior
// footprints (the common case) skip the per-corner bounds checks.
__device__ __forceinline__ float trilinear_hu(const DevVolume& V, float3 u) {
  if (V.hu8) return hu_cell_value(hu_cell_fetch(V, u));
  const float fx = floorf(u.x), fy = floorf(u.y), fz = floorf(u.z);
  if (!(fx >= -1.f && fx < (float)V.nx && fy >= -1.f && fy < (float)V.ny && fz >= -1.f && fz < (float)V.nz))
    return 0.f;
  const int i = (int)fx, j = (int)fy, k = (int)fz;
  const float tx = u.x - fx, ty = u.y - fy, tz = u.z - fz;
  float c000, c100, c010, c110, c001, c101, c011, c111;
  if ((unsigned)i < (unsigned)(V.nx - 1) && (unsigned)j < (unsigned)(V.ny - 1) && (unsigned)k < (unsigned)(V.nz - 1)) {
    const int sy = V.nx, sz = V.nx * V.ny;
    const int16_t* b = V.hu + (k * V.ny + j) * V.nx + i;
    c000 = (float)__ldg(b);
    c100 = (float)__ldg(b + 1);
    c010 = (float)__ldg(b + sy);
    c110 = (float)__ldg(b + sy + 1);
    c001 = (float)__ldg(b + sz);
    c101 = (float)__ldg(b + sz + 1);
    c011 = (float)__ldg(b + sz + sy);
    c111 = (float)__ldg(b + sz + sy + 1);
  } else {
    c000 = hu_at(V, i, j, k);
    c100 = hu_at(V, i + 1, j, k);
    c010 = hu_at(V, i, j + 1, k);
    c110 = hu_at(V, i + 1, j + 1, k);
    c001 = hu_at(V, i, j, k + 1);
    c101 = hu_at(V, i + 1, j, k + 1);
    c011 = hu_at(V, i, j + 1, k + 1);
    c111 = hu_at(V, i + 1, j + 1, k + 1);
  }
  return trilinear_blend(tx, ty, tz, c000, c100, c010, c110, c001, c101, c011, c111);
}

__device__ __forceinline__ float impedance(int z_mode, float hu, const DevTissue& t) {
  return z_mode == 0 ? fmaxf(hu + 1024.f, 1.f) : t.z;
}

// Incidence cosine at a boundary between samples s and s+1 of line l, from
// the label slice: M(l') counts the samples of the window s-W+1..s+W on
// line l' that carry the label below the boundary; the shift of that count
// between lines l-D and l+D gives the boundary's slope.  LabFn(line, s)
// returns the nearest label of a beam sample.  Evaluated by a whole warp
// for one boundary (s, l, W, D, dlat the same in every lane): lane i tests
// window positions i, i + 32, ..., and ballots add up the matches.  Every
// lane returns the cosine.
template <class LabFn>
__device__ __forceinline__ float incidence_cos_warp(LabFn lab, int l, int s, int NL, int NS, int W, int D,
                                                    float dr, float dlat, int lane) {
  const unsigned below = lab(l, s + 1);
  const int lp = min(l + D, NL - 1), lm = max(l - D, 0);
  if (lp <= lm) return 1.f;
  int dM = 0;
  for (int q0 = s - W + 1; q0 <= s + W; q0 += 32) {
    const int q = q0 + lane;
    const int qc = min(max(q, 0), NS - 1);
    const bool in = q <= s + W;
    const unsigned up = __ballot_sync(0xffffffffu, in && lab(lp, qc) == below);
    const unsigned dn = __ballot_sync(0xffffffffu, in && lab(lm, qc) == below);
    dM += __popc(up) - __popc(dn);
  }
  const float t = fabsf((float)dM) * dr / ((float)(lp - lm) * dlat);
  return rsqrtf(fmaf(t, t, 1.f));
}

__device__ __forceinline__ float lateral_spacing(const DevProbe& P, int s) {
  return P.kind == 0 ? P.pitch : fmaf((float)s, P.dr, P.r0) * P.dtheta;
}

// Volume-anchored multi-scale scatter maps at volume-frame position `pos`
// of volume `vol`: (N0, N1).  Scale k: the nearest cell of edge c 2^k
// (cell index floor(pos / (c 2^k) + 1/2), FP32 as for voxels), whose
// Philox words (counter = cell, k << 16 | vol; key = seed) give two
// standard normals as the Box-Muller pair of words 0 and 1 (r cos, r sin);
// N = sum_k a_k N_k.
__device__ __forceinline__ float2 anchored_maps(const RenderParams& p, float3 pos, unsigned vol) {
  float n0 = 0.f, n1 = 0.f;
  for (int k = 0; k < p.speckle_levels; ++k) {
    const float ic = p.inv_cell[k];
    const int cx = (int)floorf(__fadd_rn(__fmul_rn(pos.x, ic), 0.5f));
    const int cy = (int)floorf(__fadd_rn(__fmul_rn(pos.y, ic), 0.5f));
    const int cz = (int)floorf(__fadd_rn(__fmul_rn(pos.z, ic), 0.5f));
    const uint4 w = philox4x32_10(make_uint4((unsigned)cx, (unsigned)cy, (unsigned)cz, ((unsigned)k << 16) | (vol & 0xFFFFu)),
                                  p.key_fixed);
    float sn, cs;
    // angle 2 pi u shifted into [-pi, pi): cos(t) = -cos(t - pi), sin(t) = -sin(t - pi)
    __sincosf(fmaf(6.28318530717958648f, u01(w.y), -3.14159265358979324f), &sn, &cs);
    const float r = sqrtf(-2.f * __logf(u01(w.x)));
    n0 = fmaf(p.amp[k], -r * cs, n0);
    n1 = fmaf(p.amp[k], -r * sn, n1);
  }
  return make_float2(n0, n1);
}

// the image at a beam sample from its blurred reflection impulses
// pr = (P (x) R_imp), its blurred scatter pattern pt = (P (x) T) and its own
// energy e: I = R + B with the backscatter B = E . (P (x) T) (App. B.2).
// Every path forms it here, so they agree bit for bit.
__device__ __forceinline__ float image_value(float pr, float pt, float e) { return fmaf(e, pt, pr); }

// log compression to [0, 1] over the probe's dynamic range:
// 20 log10(I / e0) = (20 log10 2) log2(I) - 20 log10(e0), with the hardware
// base-2 logarithm (about 2^-22 relative error, far below the image's
// quantisation) and the e0 term precomputed on the host
__device__ __forceinline__ float log_compress(const DevProbe& P, float I) {
  const float db = fmaf(6.02059991327962390f, __log2f(fmaxf(I, 1e-30f)), -P.db_e0);
  return __saturatef(fmaf(db, P.log_gain, 1.f));
}

__device__ __forceinline__ Pose load_pose(const float* poses, int b, bool& finite) {
  Pose M;
  finite = true;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    M.m[i] = __ldg(&poses[b * 12 + i]);
    finite = finite && isfinite(M.m[i]);
  }
  return M;
}

}  // namespace ussim
