// Plain per-environment render: for each environment in turn, one kernel
// per stage (label slice, scanline model, axial PSF, lateral PSF + image
// I = P (x) R_imp + E (P (x) T) + log, scan conversion) through global
// scratch.  This is the simple form the
// fused batched kernel is measured against.
#include "us_internal.h"
#include "us_scanline.cuh"

namespace ussim {

// label slice: nearest label of every beam sample (Fig. 2: slice extraction)
__global__ void plain_slice(RenderParams p, EnvItem it, uint8_t* lab) {
  const DevProbe P = p.probes[it.probe];
  const DevVolume V = p.vols[it.vol];
  const int n = P.nl * P.ns;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  bool finite;
  const Pose M = load_pose(p.poses, it.b, finite);
  if (q == 0 && !finite) atomicOr(p.err, kErrNonFinitePose);
  if (q >= n) return;
  const int l = q / P.ns, s = q - l * P.ns;
  float x, z;
  beam_point(P, P.lines[l], s, x, z);
  int idx;
  const uint8_t lb = nearest_label(V, to_voxel(M, V.inv_h, x, z), idx);
  lab[q] = lb;
  if (p.nn_index) p.nn_index[it.beam_off + q] = idx;
  if (p.label) p.label[it.beam_off + q] = lb;
}

// scanline model, one warp per line: R_imp, T and E of every sample
__global__ void plain_lines(RenderParams p, EnvItem it, const uint8_t* lab, float* R, float* Tp, float* E) {
  const DevProbe P = p.probes[it.probe];
  const DevVolume V = p.vols[it.vol];
  const DevPair pair = p.pairs[it.pair];
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= P.nl) return;
  bool finite;
  const Pose M = load_pose(p.poses, it.b, finite);
  const int NS = P.ns;
  const float2 ln = P.lines[l];
  auto labf = [&](int line, int s) -> unsigned { return lab[line * NS + s]; };
  auto own = [&](int s) -> unsigned { return lab[l * NS + s]; };
  auto zf = [&](int s) -> float { return sample_impedance(p.z_mode, P, V, M, ln, s, P.tissue, lab[l * NS + s]); };
  const size_t row = (size_t)l * NS;
  auto posf = [&](int s) -> float3 {
    float x, z;
    beam_point(P, ln, s, x, z);
    return sample_position(M, x, z);
  };
  scanline_model(p, P, P.tissue, pair, it.b, l, lane, labf, own, zf,
                 [&](int s, float r, float t, float e) {
                   R[row + s] = r;
                   Tp[row + s] = t;
                   E[row + s] = e;
                 },
                 posf, it.vol);
}

// axial PSF of the reflection impulses and of the scatter pattern
__global__ void plain_psf_axial(RenderParams p, EnvItem it, const float* R, const float* Tp, float* AR, float* AT) {
  const DevProbe P = p.probes[it.probe];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.nl * P.ns) return;
  const int l = q / P.ns, s = q - l * P.ns;
  float accR = 0.f, accT = 0.f;
  for (int k = -P.k_ax; k <= P.k_ax; ++k) {
    const int ss = s + k;
    if (ss >= 0 && ss < P.ns) {
      const float w = P.w_ax[k + P.k_ax];
      accR = fmaf(w, R[l * P.ns + ss], accR);
      accT = fmaf(w, Tp[l * P.ns + ss], accT);
    }
  }
  AR[q] = accR;
  AT[q] = accT;
}

// lateral PSF of both, the image I = (P (x) R) + E (P (x) T), log compression
__global__ void plain_psf_lateral_log(RenderParams p, EnvItem it, const float* AR, const float* AT, const float* E,
                                      float* Y) {
  const DevProbe P = p.probes[it.probe];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.nl * P.ns) return;
  const int l = q / P.ns, s = q - l * P.ns;
  float accR = 0.f, accT = 0.f;
  for (int j = -P.k_lat; j <= P.k_lat; ++j) {
    const int ll = l + j;
    if (ll >= 0 && ll < P.nl) {
      const float w = P.w_lat[j + P.k_lat];
      accR = fmaf(w, AR[ll * P.ns + s], accR);
      accT = fmaf(w, AT[ll * P.ns + s], accT);
    }
  }
  const float acc = image_value(accR, accT, E[q]);
  const float y = log_compress(P, acc);
  Y[q] = y;
  if (p.envelope) p.envelope[it.beam_off + q] = acc;
  if (p.logimg) p.logimg[it.beam_off + q] = y;
}

__global__ void plain_scan_convert(RenderParams p, EnvItem it, const float* Y) {
  const DevProbe P = p.probes[it.probe];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.out_w * P.out_h;
  if (q >= n) return;
  float* out = p.frames + it.frame_off;
  if (P.kind == 0) {
    const int s = q / P.nl, l = q - s * P.nl;   // output row = sample, column = line
    out[q] = Y[l * P.ns + s];
    return;
  }
  const float2 f = P.lut[q];
  float v = 0.f;
  if (f.x >= 0.f) {
    const int l0 = min((int)f.x, P.nl - 2), s0 = min((int)f.y, P.ns - 2);
    const float a = f.x - (float)l0, bb = f.y - (float)s0;
    const float y00 = Y[l0 * P.ns + s0], y01 = Y[l0 * P.ns + s0 + 1];
    const float y10 = Y[(l0 + 1) * P.ns + s0], y11 = Y[(l0 + 1) * P.ns + s0 + 1];
    const float top = fmaf(a, y10 - y00, y00), bot = fmaf(a, y11 - y01, y01);
    v = fmaf(bb, bot - top, top);
  }
  out[q] = v;
}

cudaError_t launch_plain_env(const RenderParams& p, const EnvItem& it, const ProbeHost& ph,
                             const PlainScratch& scr, cudaStream_t st) {
  const int n = ph.desc.n_lines * ph.desc.n_samples;
  const int nout = ph.desc.out_w * ph.desc.out_h;
  plain_slice<<<(n + 255) / 256, 256, 0, st>>>(p, it, scr.lab);
  plain_lines<<<(ph.desc.n_lines + 3) / 4, 128, 0, st>>>(p, it, scr.lab, scr.R, scr.T, scr.E);
  plain_psf_axial<<<(n + 255) / 256, 256, 0, st>>>(p, it, scr.R, scr.T, scr.AR, scr.AT);
  plain_psf_lateral_log<<<(n + 255) / 256, 256, 0, st>>>(p, it, scr.AR, scr.AT, scr.E, scr.Y);
  plain_scan_convert<<<(nout + 255) / 256, 256, 0, st>>>(p, it, scr.Y);
  return cudaGetLastError();
}

cudaError_t launch_plain(const RenderParams& p, const EnvItem* items_host, int n_items,
                         const ProbeHost* probes, PlainScratch& scr, cudaStream_t st) {
  for (int i = 0; i < n_items; ++i) {
    const EnvItem& it = items_host[i];
    const ProbeHost& ph = probes[it.probe];
    const int n = ph.desc.n_lines * ph.desc.n_samples;
    const int nout = ph.desc.out_w * ph.desc.out_h;
    plain_slice<<<(n + 255) / 256, 256, 0, st>>>(p, it, scr.lab);
    plain_lines<<<(ph.desc.n_lines + 3) / 4, 128, 0, st>>>(p, it, scr.lab, scr.R, scr.T, scr.E);
    plain_psf_axial<<<(n + 255) / 256, 256, 0, st>>>(p, it, scr.R, scr.T, scr.AR, scr.AT);
    plain_psf_lateral_log<<<(n + 255) / 256, 256, 0, st>>>(p, it, scr.AR, scr.AT, scr.E, scr.Y);
    plain_scan_convert<<<(nout + 255) / 256, 256, 0, st>>>(p, it, scr.Y);
  }
  return cudaGetLastError();
}

}  // namespace ussim
