// The image model along one scanline (SonoGym App. B.2), evaluated by one
// warp: for every sample of the line, the reflection impulse
// R_imp = G |E cos(theta) r|^p, the scatter pattern T and the remaining
// energy E.  The image is I = P (x) R_imp + E . (P (x) T): the PSF blurs the
// impulses and the scatter pattern, and the backscatter B = E . (P (x) T)
// takes the energy at the pixel itself (App. B.2).
#pragma once
#include "us_device.cuh"

namespace ussim {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_inclusive_scan(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// One warp renders line `l` of environment `b`.  Lane i owns the sample
// pair (c + 2i, c + 2i + 1) of each 64-sample chunk c, so one Philox call
// per lane serves both samples (counter = (s >> 1, l, b, 0)).  The energy
// exponent is an exclusive prefix sum along the line: per-lane pair sums,
// a warp inclusive scan, and a carry across chunks.
//   T             -> tissue constants of this probe, indexed by label
//   lab(line, s)  -> nearest label of a beam sample (any line of the env)
//   own(s)        -> nearest label of sample s on line l
//   z_at(s)       -> impedance at sample s < NS of line l
//   store(s, r, t, e) -> receives R_imp, T and E at sample s
//   pos(s)        -> volume-frame position of sample s (anchored scatter maps)
// A lane reads z_at only at its own samples (one chunk ahead) and gets the
// next lane's value by shuffle, so store() may overwrite the storage z_at
// reads from.  `vol` is the environment's volume index.
// ANCHORED = false compiles the volume-anchored branch out (kernels that are
// instantiated per scatter-map kind).
template <bool ANCHORED = true, class LabFn, class OwnFn, class ZFn, class StoreFn, class PosFn>
__device__ __forceinline__ void scanline_model(const RenderParams& p, const DevProbe& P, const DevTissue* T,
                                               const DevPair& pair, int b, int l, int lane, LabFn lab,
                                               OwnFn own, ZFn z_at_in, StoreFn store, PosFn pos, int vol) {
  const int NS = P.ns, NL = P.nl;
  auto z_at = [&](int s) -> float { return s < NS ? z_at_in(s) : 1.f; };

  float z0 = z_at(2 * lane), z1 = z_at(2 * lane + 1);
  float carry = 0.f;
  for (int c = 0; c < NS; c += 64) {
    const int sa = c + 2 * lane, sb = sa + 1;
    const float nz0 = z_at(sa + 64), nz1 = z_at(sb + 64);
    // impedance one sample below sb: the next lane's first sample, or the
    // first sample of the next chunk for the last lane
    float zc = __shfl_down_sync(kFull, z0, 1);
    const float zc_next = __shfl_sync(kFull, nz0, 0);
    if (lane == 31) zc = zc_next;

    const unsigned la = sa < NS ? own(sa) : 0u;
    const unsigned lb = sb < NS ? own(sb) : 0u;
    const unsigned lc = sb + 1 < NS ? own(sb + 1) : lb;
    const bool Ga = sa < NS - 1 && lb != la;
    const bool Gb = sb < NS - 1 && lc != lb;
    // impedances are in [1, 5119]: the fast divide (2 ulp) is exact enough
    const float ra = sa < NS - 1 ? __fdividef(z1 - z0, z1 + z0) : 0.f;
    const float rb = sb < NS - 1 ? __fdividef(zc - z1, zc + z1) : 0.f;

    // boundaries are sparse: the warp takes them one at a time, all lanes
    // on the window of each (lane src's a sample is c + 2 src, b sample + 1)
    float cosa = 1.f, cosb = 1.f;
    {
      const unsigned ma = __ballot_sync(kFull, Ga), mb = __ballot_sync(kFull, Gb);
      for (unsigned k = ma; k; k &= k - 1) {
        const int src = __ffs(k) - 1, s = c + 2 * src;
        const float v = incidence_cos_warp(lab, l, s, NL, NS, pair.W, pair.D[s], P.dr, lateral_spacing(P, s), lane);
        if (lane == src) cosa = v;
      }
      for (unsigned k = mb; k; k &= k - 1) {
        const int src = __ffs(k) - 1, s = c + 2 * src + 1;
        const float v = incidence_cos_warp(lab, l, s, NL, NS, pair.W, pair.D[s], P.dr, lateral_spacing(P, s), lane);
        if (lane == src) cosb = v;
      }
    }

    const DevTissue ta = T[la], tb = T[lb];
    float inc_a = sa < NS ? -ta.att : 0.f;
    float inc_b = sb < NS ? -tb.att : 0.f;
    if (p.transmission) {
      if (Ga) inc_a += __logf(fmaxf(1.f - ra * ra, 1e-30f));
      if (Gb) inc_b += __logf(fmaxf(1.f - rb * rb, 1e-30f));
    }
    const float pair_sum = inc_a + inc_b;
    const float incl = warp_inclusive_scan(pair_sum, lane);
    const float La = carry + (incl - pair_sum);
    const float Lb = La + inc_a;
    carry += __shfl_sync(kFull, incl, 31);
    // hardware exp2 / log2 / sin / cos below: relative errors of order 1e-6
    // on the energy and the speckle, well inside the image's tolerance
    const float Ea = P.e0 * __expf(La), Eb = P.e0 * __expf(Lb);

    float Ra = 0.f, Rb = 0.f;
    if (Ga) {
      const float q = fabsf(cosa * ra);
      Ra = Ea * (p.refl_power == 2 ? q * q : q);
    }
    if (Gb) {
      const float q = fabsf(cosb * rb);
      Rb = Eb * (p.refl_power == 2 ? q * q : q);
    }

    float Ta, Tb;
    if (ANCHORED && p.speckle_anchor) {
      const float2 na = anchored_maps(p, pos(sa), (unsigned)vol), nb = anchored_maps(p, pos(sb), (unsigned)vol);
      Ta = na.y <= ta.mu1 ? fmaf(na.x, ta.sigma0, ta.mu0) : 0.f;
      Tb = nb.y <= tb.mu1 ? fmaf(nb.x, tb.sigma0, tb.mu0) : 0.f;
    } else if (p.speckle) {
      const uint4 w = philox4x32_10(make_uint4((unsigned)sa >> 1, (unsigned)l, (unsigned)b, 0u), p.key);
      const float rad = sqrtf(-2.f * __logf(u01(w.x)));
      // angle 2 pi u shifted into [-pi, pi), where the hardware sine and
      // cosine are accurate: sin(t) = -sin(t - pi), cos(t) = -cos(t - pi)
      float sn, cs;
      __sincosf(fmaf(6.28318530717958648f, u01(w.y), -3.14159265358979324f), &sn, &cs);
      sn = -sn;
      cs = -cs;
      Ta = (unsigned long long)w.z < ta.t1 ? fmaf(rad * cs, ta.sigma0, ta.mu0) : 0.f;
      Tb = (unsigned long long)w.w < tb.t1 ? fmaf(rad * sn, tb.sigma0, tb.mu0) : 0.f;
    } else {
      Ta = ta.mu0;
      Tb = tb.mu0;
    }
    if (sa < NS) store(sa, Ra, Ta, Ea);
    if (sb < NS) store(sb, Rb, Tb, Eb);
    z0 = nz0;
    z1 = nz1;
  }
}

// impedance of a beam sample: Z = max(HU + 1024, 1) from the trilinear HU
// (z_mode 0) or the tissue table (z_mode 1)
__device__ __forceinline__ float sample_impedance(int z_mode, const DevProbe& P, const DevVolume& V, const Pose& M,
                                                  float2 ln, int s, const DevTissue* T, unsigned label) {
  if (z_mode == 0) {
    float x, z;
    beam_point(P, ln, s, x, z);
    return fmaxf(trilinear_hu(V, to_voxel(M, V.inv_h, x, z)) + 1024.f, 1.f);
  }
  return T[label].z;
}

}  // namespace ussim
