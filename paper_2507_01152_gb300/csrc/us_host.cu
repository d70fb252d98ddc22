// C ABI of the batched ultrasound render: validation, derived tables,
// per-batch work plans and launches.  See include/ussim.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "us_internal.h"

using namespace ussim;

namespace {

constexpr int kMaxAxialHalf = 32;   // in-place axial filter in the fused kernel
constexpr int kMaxLines = 1024, kMaxSamples = 1024;
constexpr int kMaxMatchBins = 16384;   // histogram matching: bins of the reference (64 KB of shared memory)

us_status graph_launch(us_sim* s, us_plan* pl, const RenderParams& p, cudaStream_t st);
void drop_graph(us_plan& pl);
static cudaError_t two_pass_buffers(us_plan* pl);
static SplitUnits plan_units(us_sim* s, us_plan* pl, cudaStream_t st);

us_status fail(us_sim* s, us_status st, const std::string& msg) {
  if (s) s->last_error = msg;
  return st;
}

us_status cuda_fail(us_sim* s, cudaError_t e, const char* where) {
  if (s) s->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? US_ERR_OOM : US_ERR_CUDA;
}

template <class T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Gaussian taps on a grid of spacing d: exp(-(k d)^2 / (2 sigma^2)),
// |k| <= ceil(3 sigma / d), normalised in FP64, rounded to FP32.
int gaussian_taps(double sigma, double d, std::vector<float>& out) {
  const int K = sigma > 0 ? (int)std::ceil(3.0 * sigma / d) : 0;
  std::vector<double> w(2 * K + 1);
  double sum = 0;
  for (int k = -K; k <= K; ++k) {
    const double x = (double)k * d;
    w[k + K] = K ? std::exp(-x * x / (2.0 * sigma * sigma)) : 1.0;
    sum += w[k + K];
  }
  out.resize(2 * K + 1);
  for (int i = 0; i < 2 * K + 1; ++i) out[i] = (float)(w[i] / sum);
  return K;
}

// N1 density test threshold: P(N1 <= mu1) = Phi(mu1) as a 32-bit fraction
unsigned long long n1_threshold(double mu1) {
  if (std::isinf(mu1)) return mu1 > 0 ? 4294967296ull : 0ull;
  const double phi = 0.5 * std::erfc(-mu1 / std::sqrt(2.0));
  double t = std::floor(phi * 4294967296.0);
  t = std::min(std::max(t, 0.0), 4294967296.0);
  return (unsigned long long)t;
}

std::string validate_probe(const us_probe& p) {
  if (p.kind != 0 && p.kind != 1) return "probe kind must be 0 (linear) or 1 (curvilinear)";
  if (p.n_lines < 2 || p.n_lines > kMaxLines) return "n_lines must be in [2, 1024]";
  if (p.n_samples < 2 || p.n_samples > kMaxSamples) return "n_samples must be in [2, 1024]";
  if (!(p.depth_mm > 0) || !std::isfinite(p.depth_mm)) return "depth_mm must be positive";
  if (!(p.f_mhz > 0) || !(p.e0 > 0) || !(p.dyn_range_db > 0)) return "f_mhz, e0, dyn_range_db must be positive";
  if (!(p.psf_sigma_ax_mm >= 0) || !(p.psf_sigma_lat_mm >= 0)) return "PSF sigmas must be >= 0";
  if (p.kind == 0) {
    if (!(p.pitch_mm > 0)) return "linear probe needs pitch_mm > 0";
    if (p.out_w != p.n_lines || p.out_h != p.n_samples) return "linear probe needs out_w = n_lines, out_h = n_samples";
  } else {
    if (!(p.fan_deg > 0 && p.fan_deg < 180)) return "fan_deg must be in (0, 180)";
    if (!(p.radius_mm > 0)) return "radius_mm must be positive";
    if (p.out_w < 1 || p.out_h < 1 || (long long)p.out_w * p.out_h > (1 << 24)) return "bad output size";
  }
  return "";
}

void derive(ProbeHost& ph) {
  const us_probe& p = ph.desc;
  ph.dr = (double)p.depth_mm / (double)p.n_samples;
  ph.dtheta = p.kind == 1 ? (double)p.fan_deg * M_PI / 180.0 / (double)(p.n_lines - 1) : 0.0;
  ph.dlat_mid = p.kind == 1 ? ((double)p.radius_mm + 0.5 * (double)p.depth_mm) * ph.dtheta : (double)p.pitch_mm;
}

us_status build_probe_tables(us_sim* s, ProbeHost& ph) {
  const us_probe& p = ph.desc;
  const int NL = p.n_lines, NS = p.n_samples;
  // per-line geometry, FP64 rounded once to FP32
  std::vector<float2> lines(NL);
  for (int l = 0; l < NL; ++l) {
    if (p.kind == 0) {
      lines[l] = make_float2((float)(((double)l - 0.5 * (double)(NL - 1)) * (double)p.pitch_mm), 0.f);
    } else {
      const double th = ((double)l - 0.5 * (double)(NL - 1)) * ph.dtheta;
      lines[l] = make_float2((float)std::sin(th), (float)std::cos(th));
    }
  }
  std::vector<float> wax, wlat;
  ph.k_ax = gaussian_taps(p.psf_sigma_ax_mm, ph.dr, wax);
  ph.k_lat = gaussian_taps(p.psf_sigma_lat_mm, ph.dlat_mid, wlat);
  if (ph.k_ax > kMaxAxialHalf) return fail(s, US_ERR_INVALID_ARG, "axial PSF wider than 32 samples each side");
  if (ph.k_lat > kMaxHalfTaps) return fail(s, US_ERR_INVALID_ARG, "lateral PSF wider than 48 lines each side");
  // tissue constants for this probe's frequency and sample spacing
  std::vector<DevTissue> tis(s->table.size());
  for (size_t i = 0; i < s->table.size(); ++i) {
    const us_tissue& t = s->table[i];
    const double alpha_np = (double)t.alpha_db_cm_mhz * std::log(10.0) / 20.0 / 10.0;  // Np/(mm MHz)
    tis[i].att = (float)((double)p.f_mhz * alpha_np * ph.dr);
    tis[i].mu0 = t.mu0;
    tis[i].sigma0 = t.sigma0;
    tis[i].z = t.z_mrayl;
    tis[i].t1 = n1_threshold((double)t.mu1);
    tis[i].mu1 = t.mu1;
  }
  // scan-conversion map (curvilinear): fractional (line, sample) of each
  // output pixel centre over the fan's bounding box, -1 outside the fan;
  // and the probe-frame coordinates of the pixel centres (surrogate input)
  std::vector<float2> lut;
  std::vector<float> px, pz;
  if (p.kind == 1) {
    const int W = p.out_w, H = p.out_h;
    lut.resize((size_t)W * H);
    const double r0 = p.radius_mm, D = p.depth_mm;
    const double half = 0.5 * (double)p.fan_deg * M_PI / 180.0;
    const double xmax = (r0 + D) * std::sin(half), xmin = -xmax;
    const double zmin = r0 * std::cos(half), zmax = r0 + D;
    px.resize(W);
    pz.resize(H);
    for (int c = 0; c < W; ++c) px[c] = (float)(xmin + (c + 0.5) * (xmax - xmin) / W);
    for (int r = 0; r < H; ++r) pz[r] = (float)(zmin + (r + 0.5) * (zmax - zmin) / H - r0);
    for (int r = 0; r < H; ++r)
      for (int c = 0; c < W; ++c) {
        const double x = xmin + (c + 0.5) * (xmax - xmin) / W;
        const double z = zmin + (r + 0.5) * (zmax - zmin) / H;
        const double fl = std::atan2(x, z) / ph.dtheta + 0.5 * (NL - 1);
        const double fs = (std::hypot(x, z) - r0) / ph.dr;
        const bool in = fl >= 0 && fl <= NL - 1 && fs >= 0 && fs <= NS - 1;
        lut[(size_t)r * W + c] = in ? make_float2((float)fl, (float)fs) : make_float2(-1.f, -1.f);
      }
  }
  cudaError_t e;
  if ((e = upload(&ph.d_lines, lines.data(), lines.size())) != cudaSuccess) return cuda_fail(s, e, "upload lines");
  if ((e = upload(&ph.d_wax, wax.data(), wax.size())) != cudaSuccess) return cuda_fail(s, e, "upload taps");
  if ((e = upload(&ph.d_wlat, wlat.data(), wlat.size())) != cudaSuccess) return cuda_fail(s, e, "upload taps");
  if ((e = upload(&ph.d_tissue, tis.data(), tis.size())) != cudaSuccess) return cuda_fail(s, e, "upload tissue");
  if (!lut.empty() && (e = upload(&ph.d_lut, lut.data(), lut.size())) != cudaSuccess) return cuda_fail(s, e, "upload lut");
  ph.lut_host = std::move(lut);
  if (!px.empty() && ((e = upload(&ph.d_px, px.data(), px.size())) != cudaSuccess ||
                      (e = upload(&ph.d_pz, pz.data(), pz.size())) != cudaSuccess))
    return cuda_fail(s, e, "upload pixel grid");
  return US_OK;
}

DevProbe device_probe(const ProbeHost& ph) {
  DevProbe d{};
  const us_probe& p = ph.desc;
  d.kind = p.kind;
  d.nl = p.n_lines;
  d.ns = p.n_samples;
  d.out_w = p.out_w;
  d.out_h = p.out_h;
  d.k_ax = ph.k_ax;
  d.k_lat = ph.k_lat;
  d.dr = (float)ph.dr;
  d.r0 = p.radius_mm;
  d.e0 = p.e0;
  d.log_gain = (float)(1.0 / (double)p.dyn_range_db);
  d.db_e0 = (float)(20.0 * std::log10((double)p.e0));
  d.dtheta = (float)ph.dtheta;
  d.pitch = p.pitch_mm;
  d.lines = ph.d_lines;
  d.w_ax = ph.d_wax;
  d.w_lat = ph.d_wlat;
  d.lut = ph.d_lut;
  d.tissue = ph.d_tissue;
  d.px = ph.d_px;
  d.pz = ph.d_pz;
  d.wedge = ph.d_wedge;
  d.wedge_off = ph.d_wedge_off;
  return d;
}

// incidence stencil extents: axial half window of two voxels, lateral reach
// of one voxel (in lines, at each sample's depth), capped at kThetaDMax
void pair_tables(const us_volume& v, const ProbeHost& ph, int& W, std::vector<uint8_t>& D) {
  const us_probe& p = ph.desc;
  W = (int)std::ceil(2.0 * (double)v.voxel_mm / ph.dr);
  D.resize(p.n_samples);
  for (int s = 0; s < p.n_samples; ++s) {
    const double dlat = p.kind == 0 ? (double)p.pitch_mm : ((double)p.radius_mm + s * ph.dr) * ph.dtheta;
    int d = dlat > 0 ? (int)std::ceil((double)v.voxel_mm / dlat) : 1;
    D[s] = (uint8_t)std::min(std::max(d, 1), kThetaDMax);
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// a batch signature's plan is per stream: renders of the same signature on
// different streams get their own line buffer, synchronisation words, work
// counter and graph, so they may overlap.  b0: the batch is envs b0 ..
// b0 + B - 1 of a larger caller batch (noise counters and poses keep the
// caller's indices)
std::string plan_key(const us_env* envs, int B, cudaStream_t st, int b0) {
  std::string k(reinterpret_cast<const char*>(envs), (size_t)B * sizeof(us_env));
  k.append(reinterpret_cast<const char*>(&st), sizeof st);
  k.append(reinterpret_cast<const char*>(&b0), sizeof b0);
  return k;
}

us_status get_plan(us_sim* s, const us_env* envs, int B, us_plan** out, cudaStream_t st, int b0 = 0) {
  std::string key = plan_key(envs, B, st, b0);
  auto it = s->plans.find(key);
  if (it != s->plans.end()) {
    *out = &it->second;
    return US_OK;
  }
  us_plan pl;
  long long fo = 0, bo = 0;
  const int n_probes = (int)s->probes.size();
  for (int b = 0; b < B; ++b) {
    const us_env& e = envs[b];
    if (e.volume_id < 0 || e.volume_id >= (int)s->vols.size() || e.probe_id < 0 || e.probe_id >= n_probes)
      return fail(s, US_ERR_INVALID_ARG, "env " + std::to_string(b) + " has an out-of-range volume or probe id");
    const us_probe& p = s->probes[e.probe_id].desc;
    EnvItem item;
    item.b = b0 + b;
    item.vol = e.volume_id;
    item.probe = e.probe_id;
    item.pair = e.volume_id * n_probes + e.probe_id;
    item.frame_off = fo;
    item.beam_off = bo;
    pl.items_batch.push_back(item);
    fo += (((long long)p.out_w * p.out_h + 63) / 64) * 64;
    bo += (long long)p.n_lines * p.n_samples;
  }
  pl.frame_floats = fo;
  pl.beam_elems = bo;
  pl.items_sorted = pl.items_batch;
  auto cost = [&](const EnvItem& it) {
    const us_probe& p = s->probes[it.probe].desc;
    return (long long)p.n_lines * p.n_samples + (long long)p.out_w * p.out_h / 4;
  };
  std::stable_sort(pl.items_sorted.begin(), pl.items_sorted.end(),
                   [&](const EnvItem& a, const EnvItem& b) { return cost(a) > cost(b); });
  if (B > 0) {
    cudaError_t e = upload(&pl.d_items, pl.items_sorted.data(), pl.items_sorted.size());
    if (e == cudaSuccess) e = upload(&pl.d_items_batch, pl.items_batch.data(), pl.items_batch.size());
    if (e == cudaSuccess) e = cudaMalloc(&pl.d_work, sizeof(unsigned));
    if (e != cudaSuccess) {
      cudaFree(pl.d_items);
      cudaFree(pl.d_items_batch);
      return cuda_fail(s, e, "upload work list");
    }
  }
  auto ins = s->plans.emplace(std::move(key), std::move(pl));
  *out = &ins.first->second;
  return US_OK;
}

RenderParams base_params(const us_sim* s, const float* poses, uint64_t seed, uint64_t step, float* frames) {
  RenderParams p{};
  p.vols = s->d_vols;
  p.probes = s->d_probes;
  p.pairs = s->d_pairs;
  p.poses = poses;
  p.key = make_uint2((uint32_t)seed ^ (uint32_t)(step * 0x9E3779B9ull), (uint32_t)(seed >> 32));
  p.refl_power = s->opt.refl_power;
  p.transmission = s->opt.transmission;
  p.z_mode = s->opt.z_mode;
  p.speckle = s->opt.speckle;
  p.speckle_anchor = s->opt.speckle && s->opt.speckle_anchor;
  if (p.speckle_anchor) {
    // cell scales c 2^k as FP32 reciprocals (exact powers of two apart) and
    // unit-variance weights a_k ~ 2^(-k/2), computed in FP64
    const int L = s->opt.speckle_levels;
    double norm = 0.0;
    for (int k = 0; k < L; ++k) norm += std::ldexp(1.0, -k);
    const float inv_c0 = (float)(1.0 / (double)s->opt.speckle_cell_mm);
    p.speckle_levels = L;
    for (int k = 0; k < L; ++k) {
      p.inv_cell[k] = inv_c0 * (float)std::ldexp(1.0, -k);
      p.amp[k] = (float)(std::pow(2.0, -0.5 * k) / std::sqrt(norm));
    }
  }
  p.key_fixed = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  p.n_labels = s->n_labels;
  p.frames = frames;
  p.err = s->d_err;
  p.work = s->d_work;
  return p;
}

us_status no_batched(us_sim* s) {
  return fail(s, US_ERR_UNSUPPORTED,
              "no batched launch shape fits this probe set in shared memory; use us_sim_render_plain");
}

us_status check_render_args(us_sim* s, const us_env* envs, int B, const float* poses, float* frames) {
  if (!s) return US_ERR_INVALID_ARG;
  if (B < 0) return fail(s, US_ERR_INVALID_ARG, "B must be >= 0");
  if (B > 0 && (!envs || !poses || !frames)) return fail(s, US_ERR_INVALID_ARG, "NULL envs, poses or frames");
  if (B > 0 && !aligned16(frames)) return fail(s, US_ERR_INVALID_ARG, "frames must be 16-byte aligned");
  if (B > 0 && (reinterpret_cast<uintptr_t>(poses) & 3u)) return fail(s, US_ERR_INVALID_ARG, "poses must be 4-byte aligned");
  return US_OK;
}

us_status do_render(us_sim* s, const us_env* envs, int B, const float* poses, uint64_t seed, uint64_t step,
                    float* frames, float* envelope, float* logimg, int32_t* nn, uint8_t* label, int path,
                    cudaStream_t st, int b0 = 0) {
  us_status r = check_render_args(s, envs, B, poses, frames);
  if (r != US_OK || B == 0) return r;
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, st, b0)) != US_OK) return r;
  RenderParams p = base_params(s, poses, seed, step, frames);
  p.work = pl->d_work;
  p.envelope = envelope;
  p.logimg = logimg;
  p.nn_index = nn;
  p.label = label;
  cudaError_t e;
  if (path == 0) {
    if (!s->batched) return no_batched(s);
    p.items = pl->d_items;
    p.n_items = B;
    const bool two_pass = s->tuning.cluster_size == 1;
    if (two_pass && (e = two_pass_buffers(pl)) != cudaSuccess)
      return cuda_fail(s, e, "two-pass line buffer");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (st && cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusNone;
    if (s->tuning.use_graph && st && cap == cudaStreamCaptureStatusNone) return graph_launch(s, pl, p, st);
    if (two_pass) {
      if ((e = launch_split(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, st, plan_units(s, pl, st))) != cudaSuccess)
        return cuda_fail(s, e, "two-pass render launch");
      return US_OK;
    }
    if ((e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), st)) != cudaSuccess) return cuda_fail(s, e, "reset work counter");
    if ((e = launch_fused(p, s->shape, st)) != cudaSuccess) return cuda_fail(s, e, "fused render launch");
  } else {
    p.n_items = B;
    if ((e = launch_plain(p, pl->items_batch.data(), B, s->probes.data(), s->scratch, st)) != cudaSuccess)
      return cuda_fail(s, e, "plain render launch");
  }
  return US_OK;
}

void free_sim(us_sim* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t& ev : s->copy_ev)
    if (ev) cudaEventDestroy(ev);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (auto& ph : s->probes) {
    cudaFree(ph.d_lines);
    cudaFree(ph.d_wax);
    cudaFree(ph.d_wlat);
    cudaFree(ph.d_lut);
    cudaFree(ph.d_tissue);
    cudaFree(ph.d_px);
    cudaFree(ph.d_pz);
    cudaFree(ph.d_wedge);
    cudaFree(ph.d_wedge_off);
  }
  for (auto* d : s->d_pair_D) cudaFree(d);
  for (auto* d : s->d_hu8) cudaFree(d);
  for (auto* d : s->d_lab4) cudaFree(d);
  cudaFree(s->d_href);
  for (auto& kv : s->plans) {
    drop_graph(kv.second);
    cudaFree(kv.second.d_items);
    cudaFree(kv.second.d_items_batch);
    cudaFree(kv.second.d_items_gated);
    cudaFree(kv.second.d_gated_count);
    cudaFree(kv.second.d_items_audit);
    cudaFree(kv.second.d_audit_count);
    cudaFree(kv.second.d_work);
    cudaFree(kv.second.d_beam);
    cudaFree(kv.second.d_sync);
    cudaFree(kv.second.d_units);
    cudaFree(kv.second.d_slice_hu);
    cudaFree(kv.second.d_slice_fan);
  }
  for (auto& g : s->grids) {
    cudaFree(g.second.d_tabs);
    for (void* b : g.second.bufs) cudaFree(b);
  }
  cudaFree(s->d_vols);
  cudaFree(s->d_probes);
  cudaFree(s->d_pairs);
  cudaFree(s->scratch.lab);
  cudaFree(s->scratch.R);
  cudaFree(s->scratch.T);
  cudaFree(s->scratch.E);
  cudaFree(s->scratch.AR);
  cudaFree(s->scratch.AT);
  cudaFree(s->d_err);
  cudaFree(s->d_work);
  cudaFree(s->d_host_poses);
  cudaFree(s->d_host_frames);
  cudaFree(s->d_poses3d);
  delete s;
}

// two-pass path with G = warps_per_cta lines per block: layouts, wedge
// pixel lists of the curvilinear probes, device probe table
us_status apply_split(us_sim* s, const us_tuning& t) {
  SplitShape sh;
  sh.G = t.warps_per_cta;
  sh.GB_req = t.wedge_lines;
  sh.persistent = t.persistent != 0;
  if (!split_shape_fits(sh, s->probes, s->n_labels))
    return fail(s, US_ERR_UNSUPPORTED, "probe lines per block do not fit in shared memory for the two-pass path");
  cudaError_t e;
  bool changed = false;
  for (ProbeHost& ph : s->probes) {
    if (ph.desc.kind != 1 || ph.wedge_G == sh.GB) continue;
    std::vector<float4> ent;
    std::vector<int> off;
    build_wedges(ph.lut_host, ph.desc.out_w, ph.desc.out_h, ph.desc.n_lines, ph.desc.n_samples, sh.GB, ent, off);
    cudaFree(ph.d_wedge);
    cudaFree(ph.d_wedge_off);
    ph.d_wedge = nullptr;
    ph.d_wedge_off = nullptr;
    ph.wedge_G = 0;
    if ((e = upload(&ph.d_wedge, ent.data(), ent.size())) != cudaSuccess ||
        (e = upload(&ph.d_wedge_off, off.data(), off.size())) != cudaSuccess)
      return cuda_fail(s, e, "wedge tables");
    ph.wedge_G = sh.GB;
    changed = true;
  }
  if (changed) {
    std::vector<DevProbe> dp;
    for (const ProbeHost& ph : s->probes) dp.push_back(device_probe(ph));
    if ((e = cudaMemcpy(s->d_probes, dp.data(), sizeof(DevProbe) * dp.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(s, e, "probe table");
  }
  if ((e = split_prepare(sh)) != cudaSuccess) return cuda_fail(s, e, "kernel attributes");
  s->split = sh;
  s->tuning = t;
  s->batched = true;
  return US_OK;
}

us_status apply_tuning(us_sim* s, const us_tuning& t) {
  const int cs = t.cluster_size, nw = t.warps_per_cta;
  if (t.use_graph & ~1) return fail(s, US_ERR_INVALID_ARG, "use_graph must be 0 or 1");
  if ((t.persistent & ~1) || (t.persistent && cs != 1))
    return fail(s, US_ERR_INVALID_ARG, "persistent must be 0 or 1, and 0 for the cluster path");
  if ((t.wedge_lines != 0 && t.wedge_lines != 8 && t.wedge_lines != 16 && t.wedge_lines != 32) ||
      (t.wedge_lines && cs != 1))
    return fail(s, US_ERR_INVALID_ARG, "wedge_lines must be 0, 8, 16 or 32, and 0 for the cluster path");
  if (cs == 1) {
    if (nw != 8 && nw != 16 && nw != 32) return fail(s, US_ERR_INVALID_ARG, "two-pass path takes 8, 16 or 32 warps");
    return apply_split(s, t);
  }
  if (!fused_shape_known(cs, nw)) return fail(s, US_ERR_INVALID_ARG, "unsupported (cluster_size, warps_per_cta)");
  FusedShape sh;
  sh.cs = cs;
  sh.nw = nw;
  if (!fused_shape_fits(sh, s->probes, s->n_labels))
    return fail(s, US_ERR_UNSUPPORTED, "probe lines per CTA do not fit in shared memory for this cluster size");
  cudaError_t e = fused_prepare(sh);
  if (e != cudaSuccess) return cuda_fail(s, e, "kernel attributes");
  int clusters = 0;
  e = fused_max_clusters(sh, &clusters);
  if (e != cudaSuccess) return cuda_fail(s, e, "occupancy query");
  if (clusters < 1) return fail(s, US_ERR_UNSUPPORTED, "no cluster of this shape fits on the device");
  sh.clusters = clusters;
  s->shape = sh;
  s->tuning = t;
  s->batched = true;
  return US_OK;
}

// the two grids' work units of the plan's items for the current shape,
// rebuilt when the shape changes; empty (every item's full unit range) if
// they cannot be uploaded, or must be rebuilt while st is being captured
static SplitUnits plan_units(us_sim* s, us_plan* pl, cudaStream_t st) {
  if (pl->units_G != s->split.G || pl->units_GB != s->split.GB || !pl->d_units) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (st && cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
      return SplitUnits();
    std::vector<int2> u;
    int na = 0, nb = 0;
    build_split_units(pl->items_sorted, s->probes, s->split.G, s->split.GB, u, na, nb);
    // a captured graph holds the old list's address: capture again
    drop_graph(*pl);
    cudaFree(pl->d_units);
    pl->d_units = nullptr;
    pl->units_G = pl->units_GB = 0;
    if (u.empty() || upload(&pl->d_units, u.data(), u.size()) != cudaSuccess) {
      cudaGetLastError();
      pl->d_units = nullptr;
      return SplitUnits();
    }
    pl->units_G = s->split.G;
    pl->units_GB = s->split.GB;
    pl->units_na = na;
    pl->units_nb = nb;
  }
  SplitUnits su;
  su.d = pl->d_units;
  su.n_a = pl->units_na;
  su.n_b = pl->units_nb;
  return su;
}

// the two-pass path's per-plan buffers: filtered lines and the persistent
// grid's synchronisation words
static cudaError_t two_pass_buffers(us_plan* pl) {
  cudaError_t e = cudaSuccess;
  if (!pl->d_beam && (e = cudaMalloc(&pl->d_beam, kLineBufferBytesPerSample * (size_t)pl->beam_elems)) != cudaSuccess)
    return e;
  if (!pl->d_sync &&
      (e = cudaMalloc(&pl->d_sync, sizeof(unsigned) * split_sync_words((int)pl->items_batch.size()))) != cudaSuccess)
    return e;
  return e;
}

void drop_graph(us_plan& pl) {
  if (pl.gexec) cudaGraphExecDestroy(pl.gexec);
  if (pl.graph) cudaGraphDestroy(pl.graph);
  pl.gexec = nullptr;
  pl.graph = nullptr;
  pl.gnodes.clear();
  pl.gkps.clear();
  pl.g_cs = pl.g_nw = 0;
}

// Capture the render (fused: work-counter reset + kernel; two-pass: both
// kernels, or the synchronisation-word reset + persistent kernel) once per
// batch signature and launch shape; later calls only swap the kernel nodes'
// arguments (the two-pass kernels take the same ones, so node order does
// not matter).
us_status graph_launch(us_sim* s, us_plan* pl, const RenderParams& p, cudaStream_t st) {
  cudaError_t e;
  const bool two_pass = s->tuning.cluster_size == 1;
  RenderParams pp = p;
  FusedLayout lay = s->shape.lay;
  // the kernel arguments of a replay are those launch_split would pass: the
  // persistent grid's counter and flags, or the two grids' work units (a
  // rebuilt unit list drops the graph, so a replay's list is the captured one)
  const SplitUnits su = two_pass && !s->split.persistent ? plan_units(s, pl, st) : SplitUnits();
  SplitArgs sa = s->split.args;
  set_line_buffer(sa, pl->d_beam, pl->beam_elems);
  if (two_pass && s->split.persistent) {
    sa.work = pl->d_sync;
    sa.done = pl->d_sync ? pl->d_sync + 1 : nullptr;
  } else if (su.d) {
    sa.units = su.d;
    sa.n_units_a = su.n_a;
    sa.n_units_b = su.n_b;
  }
  void* fargs[2] = {&pp, &lay};
  void* sargs[2] = {&pp, &sa};
  if (!pl->gexec || pl->g_cs != s->tuning.cluster_size || pl->g_nw != s->tuning.warps_per_cta ||
      pl->g_pers != s->tuning.persistent || pl->g_gb != s->split.GB || pl->g_units != su.d) {
    drop_graph(*pl);
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_fail(s, e, "graph capture");
    cudaError_t e1 = cudaSuccess, e2;
    if (two_pass) {
      e2 = launch_split(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, p.n_items, st, su);
    } else {
      e1 = cudaMemsetAsync(p.work, 0, sizeof(unsigned), st);
      e2 = launch_fused(p, s->shape, st);
    }
    e = cudaStreamEndCapture(st, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(s, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e), "graph capture");
    }
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) cudaGraphGetNodes(g, nodes.data(), &n);
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      cudaKernelNodeParams kp{};
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel &&
          cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess) {
        pl->gnodes.push_back(nd);
        pl->gkps.push_back(kp);
      }
    }
    const size_t want = two_pass && !s->split.persistent ? 2u : 1u;
    if (pl->gnodes.size() != want || (e = cudaGraphInstantiate(&pl->gexec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      pl->gexec = nullptr;
      pl->gnodes.clear();
      pl->gkps.clear();
      return cuda_fail(s, pl->gnodes.empty() ? cudaErrorUnknown : e, "graph instantiate");
    }
    pl->graph = g;
    pl->g_cs = s->tuning.cluster_size;
    pl->g_nw = s->tuning.warps_per_cta;
    pl->g_pers = s->tuning.persistent;
    pl->g_gb = s->split.GB;
    pl->g_units = su.d;
    if ((e = cudaGraphLaunch(pl->gexec, st)) != cudaSuccess) return cuda_fail(s, e, "graph launch");
    return US_OK;
  }
  for (size_t i = 0; i < pl->gnodes.size(); ++i) {
    cudaKernelNodeParams kp = pl->gkps[i];
    kp.kernelParams = two_pass ? sargs : fargs;
    kp.extra = nullptr;
    if ((e = cudaGraphExecKernelNodeSetParams(pl->gexec, pl->gnodes[i], &kp)) != cudaSuccess)
      return cuda_fail(s, e, "graph update");
  }
  if ((e = cudaGraphLaunch(pl->gexec, st)) != cudaSuccess) return cuda_fail(s, e, "graph launch");
  return US_OK;
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

}  // namespace

namespace ussim {
RenderParams sim_render_params(const us_sim* s, const float* poses, uint64_t seed, uint64_t step, float* frames) {
  return base_params(s, poses, seed, step, frames);
}
us_status sim_check_render_args(us_sim* s, const us_env* envs, int B, const float* poses, float* frames) {
  return check_render_args(s, envs, B, poses, frames);
}
}  // namespace ussim

extern "C" {

const char* us_status_string(us_status st) {
  switch (st) {
    case US_OK: return "US_OK";
    case US_ERR_INVALID_ARG: return "US_ERR_INVALID_ARG";
    case US_ERR_CUDA: return "US_ERR_CUDA";
    case US_ERR_OOM: return "US_ERR_OOM";
    case US_ERR_TIMEOUT: return "US_ERR_TIMEOUT";
    case US_ERR_UNSUPPORTED: return "US_ERR_UNSUPPORTED";
    case US_ERR_INTERNAL: return "US_ERR_INTERNAL";
  }
  return "unknown status";
}

const char* us_sim_last_error(const us_sim* s) { return s ? s->last_error.c_str() : "NULL handle"; }

// Read the volumes' contents: every label must index the tissue table, the
// HU grid is copied into corner records and the labels into 4 x 4 x 4
// bricks (each allocated once per volume; a volume whose copy does not fit
// in memory or in 31-bit indices keeps reading the caller's grid, with
// identical results).  Synchronous.
static us_status read_volumes(us_sim* s, cudaStream_t st) {
  cudaError_t e;
  for (size_t i = 0; i < s->vols.size(); ++i) {
    const us_volume& v = s->vols[i];
    unsigned mx = 0;
    if ((e = cudaMemsetAsync(s->d_work, 0, sizeof(unsigned), st)) != cudaSuccess ||
        (e = max_label(v.labels, (long long)v.nx * v.ny * v.nz, s->d_work, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&mx, s->d_work, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(s, e, "label check");
    if ((int)mx >= s->n_labels) return fail(s, US_ERR_INVALID_ARG, "label outside the tissue table");
    const long long n8 = corner_records(v.nx, v.ny, v.nz), n4 = label_bricks_bytes(v.nx, v.ny, v.nz);
    if (!s->d_hu8[i] && s->opt.volume_layout == 0 && n8 < (1ll << 31) && cudaMalloc(&s->d_hu8[i], (size_t)n8 * sizeof(uint4)) != cudaSuccess) {
      cudaGetLastError();
      s->d_hu8[i] = nullptr;
    }
    if (!s->d_lab4[i] && s->opt.volume_layout == 0 && n4 < (1ll << 31) && cudaMalloc(&s->d_lab4[i], (size_t)n4) != cudaSuccess) {
      cudaGetLastError();
      s->d_lab4[i] = nullptr;
    }
    ussim::DevVolume dv = s->dev_vols[i];
    dv.hu8 = nullptr;
    dv.lab4 = nullptr;
    dv.qy = corner_quads_y(v.ny);
    dv.bx = (v.nx + 3) / 4;
    dv.by = (v.ny + 3) / 4;
    if (s->d_hu8[i] && (e = pack_corners(dv, s->d_hu8[i], st)) != cudaSuccess) return cuda_fail(s, e, "corner records");
    if (s->d_lab4[i] && (e = pack_labels(dv, s->d_lab4[i], st)) != cudaSuccess) return cuda_fail(s, e, "label bricks");
    s->dev_vols[i].hu8 = s->d_hu8[i];
    s->dev_vols[i].lab4 = s->d_lab4[i];
    s->dev_vols[i].qy = dv.qy;
    s->dev_vols[i].bx = dv.bx;
    s->dev_vols[i].by = dv.by;
  }
  if ((e = cudaMemcpyAsync(s->d_vols, s->dev_vols.data(), s->dev_vols.size() * sizeof(ussim::DevVolume),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(s, e, "volume descriptors");
  return US_OK;
}

us_status us_sim_refresh_volumes(us_sim* s, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  return read_volumes(s, static_cast<cudaStream_t>(stream));
}

us_status us_sim_create(const us_volume* vols, int32_t n_vols, const us_tissue* table, int32_t n_labels,
                        const us_probe* probes, int32_t n_probes, const us_options* opt, us_sim** out) {
  if (!out) return US_ERR_INVALID_ARG;
  *out = nullptr;
  if (!vols || n_vols < 1 || !table || n_labels < 1 || n_labels > 256 || !probes || n_probes < 1)
    return US_ERR_INVALID_ARG;
  us_sim* s = new (std::nothrow) us_sim();
  if (!s) return US_ERR_OOM;
  s->opt = opt ? *opt : us_options{1, 1, 0, 1, 0, 1, 0.25f, 0};
  if (!(s->opt.refl_power == 1 || s->opt.refl_power == 2) || (s->opt.transmission & ~1) || (s->opt.z_mode & ~1) ||
      (s->opt.speckle & ~1) || (s->opt.speckle_anchor & ~1) || (s->opt.volume_layout & ~1) ||
      (s->opt.speckle_anchor && (s->opt.speckle_levels < 1 || s->opt.speckle_levels > kMaxSpeckleLevels ||
                                 !(s->opt.speckle_cell_mm > 0.f) || !std::isfinite(s->opt.speckle_cell_mm)))) {
    delete s;
    return US_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_vols; ++i) {
    const us_volume& v = vols[i];
    if (!v.labels || !v.hu || v.nx < 1 || v.ny < 1 || v.nz < 1 || !(v.voxel_mm > 0) ||
        (long long)v.nx * v.ny * v.nz >= (1ll << 31)) {
      delete s;
      return US_ERR_INVALID_ARG;
    }
    s->vols.push_back(v);
  }
  for (int i = 0; i < n_labels; ++i) {
    const us_tissue& t = table[i];
    if (!std::isfinite(t.alpha_db_cm_mhz) || !std::isfinite(t.z_mrayl) || !(t.z_mrayl > 0) || !std::isfinite(t.mu0) ||
        !std::isfinite(t.sigma0) || std::isnan(t.mu1)) {
      delete s;
      return US_ERR_INVALID_ARG;
    }
    s->table.push_back(t);
  }
  s->n_labels = n_labels;
  for (int i = 0; i < n_probes; ++i) {
    std::string why = validate_probe(probes[i]);
    if (!why.empty()) {
      delete s;
      return US_ERR_INVALID_ARG;
    }
    ProbeHost ph;
    ph.desc = probes[i];
    derive(ph);
    s->probes.push_back(ph);
  }
  us_status r;
  cudaError_t e;
  for (auto& ph : s->probes)
    if ((r = build_probe_tables(s, ph)) != US_OK) {
      free_sim(s);
      return r;
    }
  std::vector<DevVolume> dv;
  for (const us_volume& v : s->vols)
    dv.push_back(DevVolume{v.labels, v.hu, v.nx, v.ny, v.nz, (float)(1.0 / (double)v.voxel_mm), v.voxel_mm, nullptr,
                                0, nullptr, 0, 0});
  std::vector<DevProbe> dp;
  for (const ProbeHost& ph : s->probes) dp.push_back(device_probe(ph));
  std::vector<DevPair> pairs;
  for (const us_volume& v : s->vols)
    for (const ProbeHost& ph : s->probes) {
      int W;
      std::vector<uint8_t> D;
      pair_tables(v, ph, W, D);
      uint8_t* dD = nullptr;
      if ((e = upload(&dD, D.data(), D.size())) != cudaSuccess) {
        free_sim(s);
        return cuda_fail(nullptr, e, "pairs");
      }
      s->d_pair_D.push_back(dD);
      DevPair pr{W, dD, D.empty() ? 1 : (int)*std::max_element(D.begin(), D.end()), {}};
      for (int d = 0; d <= kThetaDMax; ++d) {
        int deepest = -1;
        for (int q = 0; q < (int)D.size(); ++q)
          if (D[q] >= d) deepest = q;
        pr.ext[d] = deepest < 0 ? 0 : std::min((int)D.size(), deepest + W + 1);
      }
      pairs.push_back(pr);
    }
  size_t max_beam = 0;
  for (const ProbeHost& ph : s->probes) max_beam = std::max(max_beam, (size_t)ph.desc.n_lines * ph.desc.n_samples);
  if ((e = upload(&s->d_vols, dv.data(), dv.size())) != cudaSuccess || (e = upload(&s->d_probes, dp.data(), dp.size())) != cudaSuccess ||
      (e = upload(&s->d_pairs, pairs.data(), pairs.size())) != cudaSuccess ||
      (e = cudaMalloc(&s->scratch.lab, max_beam)) != cudaSuccess ||
      (e = cudaMalloc(&s->scratch.R, max_beam * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->scratch.T, max_beam * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->scratch.E, max_beam * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->scratch.AR, max_beam * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->scratch.AT, max_beam * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_err, sizeof(unsigned))) != cudaSuccess || (e = cudaMalloc(&s->d_work, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMemset(s->d_err, 0, sizeof(unsigned))) != cudaSuccess) {
    us_status st = e == cudaErrorMemoryAllocation ? US_ERR_OOM : US_ERR_CUDA;
    free_sim(s);
    return st;
  }
  s->scratch.Y = s->scratch.R;   // the log image reuses R's storage (R is dead once AR is formed)
  s->dev_vols = dv;
  s->d_hu8.assign(dv.size(), nullptr);
  s->d_lab4.assign(dv.size(), nullptr);
  if ((r = read_volumes(s, nullptr)) != US_OK) {
    free_sim(s);
    return r;
  }
  // default launch shape: the first that fits the probe set, two-pass
  // first; when none fits, the batched entry points report
  // US_ERR_UNSUPPORTED and the plain per-environment path still renders
  {
    static const us_tuning order[] = {{1, 16, 1}, {1, 8, 1}, {1, 32, 1}, {8, 32, 1}, {16, 16, 1}, {16, 8, 1}};
    s->batched = false;
    for (const us_tuning& t : order)
      if (apply_tuning(s, t) == US_OK) break;
    s->last_error.clear();
  }
  *out = s;
  return US_OK;
}

void us_sim_destroy(us_sim* s) { free_sim(s); }

us_status us_sim_frame_layout(const us_sim* s, const us_env* envs, int32_t B, int64_t* offsets) {
  if (!s || B < 0 || !offsets || (B > 0 && !envs)) return US_ERR_INVALID_ARG;
  offsets[0] = 0;
  for (int b = 0; b < B; ++b) {
    if (envs[b].probe_id < 0 || envs[b].probe_id >= (int)s->probes.size() || envs[b].volume_id < 0 ||
        envs[b].volume_id >= (int)s->vols.size())
      return US_ERR_INVALID_ARG;
    const us_probe& p = s->probes[envs[b].probe_id].desc;
    offsets[b + 1] = offsets[b] + (((long long)p.out_w * p.out_h + 63) / 64) * 64;
  }
  return US_OK;
}

us_status us_sim_beam_layout(const us_sim* s, const us_env* envs, int32_t B, int64_t* offsets) {
  if (!s || B < 0 || !offsets || (B > 0 && !envs)) return US_ERR_INVALID_ARG;
  offsets[0] = 0;
  for (int b = 0; b < B; ++b) {
    if (envs[b].probe_id < 0 || envs[b].probe_id >= (int)s->probes.size()) return US_ERR_INVALID_ARG;
    const us_probe& p = s->probes[envs[b].probe_id].desc;
    offsets[b + 1] = offsets[b] + (long long)p.n_lines * p.n_samples;
  }
  return US_OK;
}

us_status us_sim_render(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed, uint64_t step,
                        float* frames, void* stream) {
  return do_render(s, envs, B, poses, seed, step, frames, nullptr, nullptr, nullptr, nullptr, 0,
                   static_cast<cudaStream_t>(stream));
}

us_status us_sim_render_plain(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                              uint64_t step, float* frames, void* stream) {
  return do_render(s, envs, B, poses, seed, step, frames, nullptr, nullptr, nullptr, nullptr, 1,
                   static_cast<cudaStream_t>(stream));
}

us_status us_sim_render_debug(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                              uint64_t step, float* frames, float* envelope, float* logimg, int32_t* nn_index,
                              uint8_t* label, int32_t path, void* stream) {
  if (path != 0 && path != 1) return fail(s, US_ERR_INVALID_ARG, "path must be 0 (fused) or 1 (plain)");
  return do_render(s, envs, B, poses, seed, step, frames, envelope, logimg, nn_index, label, path,
                   static_cast<cudaStream_t>(stream));
}

us_status us_sim_render_host(us_sim* s, const us_env* envs, int32_t B, const float* poses_host, uint64_t seed,
                             uint64_t step, float* frames_host, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (B < 0 || (B > 0 && (!envs || !poses_host || !frames_host))) return fail(s, US_ERR_INVALID_ARG, "bad host buffers");
  if (B == 0) return US_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  us_plan* pl;
  us_status r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream));
  if (r != US_OK) return r;
  for (int i = 0; i < 12 * B; ++i)
    if (!std::isfinite(poses_host[i])) return fail(s, US_ERR_INVALID_ARG, "non-finite pose entry");
  const size_t pose_bytes = (size_t)B * 12 * sizeof(float), frame_bytes = (size_t)pl->frame_floats * sizeof(float);
  cudaError_t e;
  if (pose_bytes > s->host_poses_cap) {
    cudaFree(s->d_host_poses);
    s->d_host_poses = nullptr;
    if ((e = cudaMalloc(&s->d_host_poses, pose_bytes)) != cudaSuccess) return cuda_fail(s, e, "pose staging");
    s->host_poses_cap = pose_bytes;
  }
  if (frame_bytes > s->host_frames_cap) {
    cudaFree(s->d_host_frames);
    s->d_host_frames = nullptr;
    if ((e = cudaMalloc(&s->d_host_frames, frame_bytes)) != cudaSuccess) return cuda_fail(s, e, "frame staging");
    s->host_frames_cap = frame_bytes;
  }
  if ((e = cudaMemcpyAsync(s->d_host_poses, poses_host, pose_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(s, e, "pose copy");
  // A batch of 16 MB of frames or more renders as up to four contiguous
  // sub-batches (env ranges, each keeping its envs' caller indices), and
  // each sub-batch's frames go to the host on a copy stream while the next
  // one renders.  Sub-batch k holds about kSubRatio^k of the frame bytes
  // (normalised; at least 8 MB on average): the copy to host memory runs at
  // about half the render's rate, so each copy still hides behind the next,
  // half-size render, and the one copy left after the last render is short.  A smaller batch renders in one piece: there the sub-batches'
  // extra waves would cost more than the copy overlap gains.
  constexpr size_t kSubBytes = 8u << 20;
  constexpr double kSubRatio = 0.5;
  const int n_sub = (int)std::min<size_t>({(size_t)us_sim::kHostSub, (size_t)B, std::max<size_t>(1, frame_bytes / kSubBytes)});
  if (n_sub == 1) {
    if ((r = do_render(s, envs, B, s->d_host_poses, seed, step, s->d_host_frames, nullptr, nullptr, nullptr, nullptr, 0,
                       st)) != US_OK)
      return r;
    if ((e = cudaMemcpyAsync(frames_host, s->d_host_frames, frame_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(s, e, "frame copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(s, e, "render");
    return US_OK;
  }
  if (!s->copy_stream) {
    // all or nothing: a partial set is released, so the next call retries
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[us_sim::kHostSub] = {};
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int k = 0; k < us_sim::kHostSub && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
      if (cs) cudaStreamDestroy(cs);
      return cuda_fail(s, e, "copy stream");
    }
    s->copy_stream = cs;
    for (int k = 0; k < us_sim::kHostSub; ++k) s->copy_ev[k] = ev[k];
  }
  const std::vector<EnvItem>& items = pl->items_batch;   // caller order, full-batch frame offsets
  auto off_of = [&](int b) -> long long { return b < B ? items[b].frame_off : pl->frame_floats; };
  double wsum = 0, wk = 1;
  for (int k = 0; k < n_sub; ++k, wk *= kSubRatio) wsum += wk;
  int b0 = 0;
  us_status rr = US_OK;
  double cum = 0;
  wk = 1;
  for (int k = 0; k < n_sub && b0 < B; ++k, wk *= kSubRatio) {
    int b1 = b0 + 1;
    cum += wk;
    const long long target = (long long)((double)pl->frame_floats * (cum / wsum));
    while (b1 < B && (k + 1 == n_sub || off_of(b1) < target)) ++b1;
    const long long f0 = off_of(b0), f1 = off_of(b1);
    if ((rr = do_render(s, envs + b0, b1 - b0, s->d_host_poses, seed, step, s->d_host_frames + f0, nullptr, nullptr,
                        nullptr, nullptr, 0, st, b0)) != US_OK)
      break;
    if ((e = cudaEventRecord(s->copy_ev[k], st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s->copy_stream, s->copy_ev[k], 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(frames_host + f0, s->d_host_frames + f0, (size_t)(f1 - f0) * sizeof(float),
                             cudaMemcpyDeviceToHost, s->copy_stream)) != cudaSuccess) {
      rr = cuda_fail(s, e, "frame copy");
      break;
    }
    b0 = b1;
  }
  // both streams drain before the call returns, also after an error
  const cudaError_t e1 = cudaStreamSynchronize(s->copy_stream), e2 = cudaStreamSynchronize(st);
  if (rr != US_OK) return rr;
  if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(s, e1 != cudaSuccess ? e1 : e2, "render");
  return US_OK;
}

us_status us_sim_render_gated(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed, uint64_t step,
                              float* frames, const float* score, float threshold, int32_t* n_rendered, void* stream) {
  us_status r = check_render_args(s, envs, B, poses, frames);
  if (r != US_OK || B == 0) return r;
  if (!score) return fail(s, US_ERR_INVALID_ARG, "NULL score");
  if (B > 32 * 1024) return fail(s, US_ERR_UNSUPPORTED, "gated batches are limited to 32768 envs");
  if (!s->batched) return no_batched(s);
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  cudaError_t e;
  if (!pl->d_items_gated && ((e = cudaMalloc(&pl->d_items_gated, sizeof(EnvItem) * B)) != cudaSuccess ||
                             (e = cudaMalloc(&pl->d_gated_count, sizeof(int))) != cudaSuccess))
    return cuda_fail(s, e, "gated work list");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((e = launch_gate_compact(pl->d_items_batch, B, score, threshold, pl->d_items_gated, pl->d_gated_count, st)) !=
      cudaSuccess)
    return cuda_fail(s, e, "gate");
  RenderParams p = base_params(s, poses, seed, step, frames);
  p.work = pl->d_work;
  p.items = pl->d_items_gated;
  p.n_items = B;
  p.n_items_dev = pl->d_gated_count;
  if (s->tuning.cluster_size == 1) {
    if ((e = two_pass_buffers(pl)) != cudaSuccess)
      return cuda_fail(s, e, "two-pass line buffer");
    if ((e = launch_split(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, st)) != cudaSuccess) return cuda_fail(s, e, "gated render");
  } else if ((e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), st)) != cudaSuccess ||
             (e = launch_fused(p, s->shape, st)) != cudaSuccess) {
    return cuda_fail(s, e, "gated render");
  }
  if (n_rendered && (e = cudaMemcpyAsync(n_rendered, pl->d_gated_count, sizeof(int), cudaMemcpyDeviceToDevice, st)) !=
                        cudaSuccess)
    return cuda_fail(s, e, "gated count");
  return US_OK;
}

us_status us_sim_render_audit(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                              uint64_t step, float* audit_frames, const float* score, float threshold, float fraction,
                              uint8_t* flags, int32_t* n_audited, void* stream) {
  us_status r = check_render_args(s, envs, B, poses, audit_frames);
  if (r != US_OK || B == 0) return r;
  if (!score) return fail(s, US_ERR_INVALID_ARG, "NULL score");
  if (!(fraction >= 0.f && fraction <= 1.f)) return fail(s, US_ERR_INVALID_ARG, "audit fraction must be in [0, 1]");
  if (B > 32 * 1024) return fail(s, US_ERR_UNSUPPORTED, "audited batches are limited to 32768 envs");
  if (!s->batched) return no_batched(s);
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  cudaError_t e;
  if (!pl->d_items_audit && ((e = cudaMalloc(&pl->d_items_audit, sizeof(EnvItem) * B)) != cudaSuccess ||
                             (e = cudaMalloc(&pl->d_audit_count, sizeof(int))) != cudaSuccess))
    return cuda_fail(s, e, "audit work list");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RenderParams p = base_params(s, poses, seed, step, audit_frames);
  p.work = pl->d_work;
  const double t = std::floor((double)fraction * 4294967296.0);
  if ((e = launch_audit_compact(pl->d_items_batch, B, score, threshold, p.key, (unsigned long long)t,
                                pl->d_items_audit, pl->d_audit_count, flags, st)) != cudaSuccess)
    return cuda_fail(s, e, "audit selection");
  p.items = pl->d_items_audit;
  p.n_items = B;
  p.n_items_dev = pl->d_audit_count;
  if (s->tuning.cluster_size == 1) {
    if ((e = two_pass_buffers(pl)) != cudaSuccess) return cuda_fail(s, e, "two-pass line buffer");
    if ((e = launch_split(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, st)) != cudaSuccess)
      return cuda_fail(s, e, "audit render");
  } else if ((e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), st)) != cudaSuccess ||
             (e = launch_fused(p, s->shape, st)) != cudaSuccess) {
    return cuda_fail(s, e, "audit render");
  }
  if (n_audited && (e = cudaMemcpyAsync(n_audited, pl->d_audit_count, sizeof(int), cudaMemcpyDeviceToDevice, st)) !=
                       cudaSuccess)
    return cuda_fail(s, e, "audit count");
  return US_OK;
}

us_status us_sim_sample_slices_grid(us_sim* s, const us_env* envs, int32_t B, const float* poses, int32_t H,
                                    int32_t W, uint16_t* out, void* stream) {
  us_status r = check_render_args(s, envs, B, poses, reinterpret_cast<float*>(out));
  if (r != US_OK || B == 0) return r;
  if (H < 2 || W < 2 || H > 4096 || W > 4096) return fail(s, US_ERR_INVALID_ARG, "grid size must be in [2, 4096]");
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  auto key = std::make_pair((int)H, (int)W);
  auto it = s->grids.find(key);
  cudaError_t e;
  if (it == s->grids.end()) {
    // per probe: pixel centres of an H x W grid over its output field, in
    // FP64, rounded once to FP32 (curvilinear: the fan's bounding box in apex
    // coordinates, shifted by -r0 into the probe frame, and the inside-fan
    // test of the scan conversion; linear: the rectangle of lines 0 .. NL-1
    // and samples 0 .. NS-1, all inside)
    us_sim::GridTabs g;
    std::vector<DevGridTab> tabs;
    for (const ProbeHost& ph : s->probes) {
      const us_probe& p = ph.desc;
      const int NL = p.n_lines, NS = p.n_samples;
      std::vector<float> px(W), pz(H);
      std::vector<uint8_t> mask((size_t)H * W, 1);
      if (p.kind == 1) {
        const double r0 = p.radius_mm, D = p.depth_mm;
        const double half = 0.5 * (double)p.fan_deg * M_PI / 180.0;
        const double xmax = (r0 + D) * std::sin(half), xmin = -xmax;
        const double zmin = r0 * std::cos(half), zmax = r0 + D;
        for (int c = 0; c < W; ++c) px[c] = (float)(xmin + (c + 0.5) * (xmax - xmin) / W);
        for (int q = 0; q < H; ++q) pz[q] = (float)(zmin + (q + 0.5) * (zmax - zmin) / H - r0);
        for (int q = 0; q < H; ++q)
          for (int c = 0; c < W; ++c) {
            const double x = xmin + (c + 0.5) * (xmax - xmin) / W;
            const double z = zmin + (q + 0.5) * (zmax - zmin) / H;
            const double fl = std::atan2(x, z) / ph.dtheta + 0.5 * (NL - 1);
            const double fs = (std::hypot(x, z) - r0) / ph.dr;
            mask[(size_t)q * W + c] = fl >= 0 && fl <= NL - 1 && fs >= 0 && fs <= NS - 1;
          }
      } else {
        for (int c = 0; c < W; ++c)
          px[c] = (float)(((c + 0.5) * NL / W - 0.5 - 0.5 * (NL - 1)) * (double)p.pitch_mm);
        for (int q = 0; q < H; ++q) pz[q] = (float)(((q + 0.5) * NS / H - 0.5) * ph.dr);
      }
      float *dpx = nullptr, *dpz = nullptr;
      uint8_t* dm = nullptr;
      if ((e = upload(&dpx, px.data(), px.size())) == cudaSuccess) g.bufs.push_back(dpx);
      if (e == cudaSuccess && (e = upload(&dpz, pz.data(), pz.size())) == cudaSuccess) g.bufs.push_back(dpz);
      if (e == cudaSuccess && (e = upload(&dm, mask.data(), mask.size())) == cudaSuccess) g.bufs.push_back(dm);
      if (e != cudaSuccess) {
        for (void* b : g.bufs) cudaFree(b);
        return cuda_fail(s, e, "surrogate grid tables");
      }
      tabs.push_back(DevGridTab{dpx, dpz, dm});
    }
    if ((e = upload(&g.d_tabs, tabs.data(), tabs.size())) != cudaSuccess) {
      for (void* b : g.bufs) cudaFree(b);
      return cuda_fail(s, e, "surrogate grid tables");
    }
    it = s->grids.emplace(key, std::move(g)).first;
  }
  RenderParams p = base_params(s, poses, 0, 0, nullptr);
  if ((e = launch_grid_slices(p, pl->d_items_batch, B, H, W, it->second.d_tabs, out,
                              static_cast<cudaStream_t>(stream))) != cudaSuccess)
    return cuda_fail(s, e, "grid slice sampling launch");
  return US_OK;
}

us_status us_sim_resize_frames(us_sim* s, const us_env* envs, int32_t B, const float* src, int32_t H, int32_t W,
                               float* frames, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (B < 0) return fail(s, US_ERR_INVALID_ARG, "B must be >= 0");
  if (B == 0) return US_OK;
  if (!envs || !src || !frames) return fail(s, US_ERR_INVALID_ARG, "NULL envs, src or frames");
  if (!aligned16(frames)) return fail(s, US_ERR_INVALID_ARG, "frames must be 16-byte aligned");
  if (H < 2 || W < 2 || H > 4096 || W > 4096) return fail(s, US_ERR_INVALID_ARG, "grid size must be in [2, 4096]");
  us_plan* pl;
  us_status r;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  int max_out = 0;
  for (const ProbeHost& ph : s->probes) max_out = std::max(max_out, ph.desc.out_w * ph.desc.out_h);
  RenderParams p = base_params(s, nullptr, 0, 0, frames);
  cudaError_t e = launch_resize(p, pl->d_items_batch, B, src, H, W, max_out, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? US_OK : cuda_fail(s, e, "resize launch");
}

us_status us_sim_render_3d(us_sim* s, const us_env* envs, int32_t B, const float* poses, int32_t n_elev,
                           float elev_pitch_mm, uint64_t seed, uint64_t step, float* frames, void* stream) {
  us_status r = check_render_args(s, envs, B, poses, frames);
  if (r != US_OK || B == 0) return r;
  if (n_elev < 1 || n_elev > 64 || !std::isfinite(elev_pitch_mm) || elev_pitch_mm < 0.f)
    return fail(s, US_ERR_INVALID_ARG, "n_elev must be 1..64 and the elevation pitch finite and >= 0");
  if ((long long)B * n_elev > (1ll << 30)) return fail(s, US_ERR_INVALID_ARG, "batch too large");
  const int BE = B * n_elev;
  std::vector<us_env> ex((size_t)BE);
  for (int b = 0; b < B; ++b)
    for (int e = 0; e < n_elev; ++e) ex[(size_t)b * n_elev + e] = envs[b];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  const size_t bytes = sizeof(float) * 12 * (size_t)BE;
  if (bytes > s->poses3d_cap) {
    cudaFree(s->d_poses3d);
    s->d_poses3d = nullptr;
    s->poses3d_cap = 0;
    if ((e = cudaMalloc(&s->d_poses3d, bytes)) != cudaSuccess) return cuda_fail(s, e, "swept poses");
    s->poses3d_cap = bytes;
  }
  if ((e = launch_expand_elevation(poses, B, n_elev, elev_pitch_mm, s->d_poses3d, st)) != cudaSuccess)
    return cuda_fail(s, e, "elevation sweep");
  return do_render(s, ex.data(), BE, s->d_poses3d, seed, step, frames, nullptr, nullptr, nullptr, nullptr, 0, st);
}

us_status us_sim_sweep_poses(const float* poses, int32_t B, int32_t n_elev, float elev_pitch_mm, float* out,
                             void* stream) {
  if (B < 0 || n_elev < 1 || n_elev > 64 || !std::isfinite(elev_pitch_mm) || elev_pitch_mm < 0.f)
    return US_ERR_INVALID_ARG;
  if (B == 0) return US_OK;
  if (!poses || !out || (long long)B * n_elev > (1ll << 30)) return US_ERR_INVALID_ARG;
  return launch_expand_elevation(poses, B, n_elev, elev_pitch_mm, out, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? US_OK
             : US_ERR_CUDA;
}

int64_t us_sim_recon_words(const us_sim* s) {
  if (!s) return -1;
  long long w = 0;
  for (const us_volume& v : s->vols) w = std::max(w, ((long long)v.nx * v.ny * v.nz + 31) / 32);
  return w;
}

us_status us_sim_recon_update(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                              uint64_t step, int32_t bone_label, float p_miss, uint32_t* bitmaps, int32_t* points,
                              int32_t* counts, int32_t cap, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (B < 0 || (B > 0 && (!envs || !poses || !bitmaps || !points || !counts)) || cap < 1 || bone_label < 0 ||
      bone_label > 255 || !(p_miss >= 0.f && p_miss <= 1.f))
    return fail(s, US_ERR_INVALID_ARG, "bad reconstruction arguments");
  if (B == 0) return US_OK;
  us_plan* pl;
  us_status r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream));
  if (r != US_OK) return r;
  RenderParams p = base_params(s, poses, seed, step, nullptr);
  int max_lines = 1;
  for (int b = 0; b < B; ++b) max_lines = std::max(max_lines, s->probes[envs[b].probe_id].desc.n_lines);
  const double t = std::floor((double)p_miss * 4294967296.0);
  const unsigned thr = (unsigned)std::min(t, 4294967295.0);
  cudaError_t e = launch_recon_update(p, pl->d_items_batch, B, bone_label, thr, bitmaps, us_sim_recon_words(s),
                                      points, counts, cap, max_lines, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? US_OK : cuda_fail(s, e, "reconstruction update");
}

us_status us_sim_recon_observe(us_sim* s, const us_env* envs, int32_t B, const float* poses, const int32_t* points,
                               const int32_t* counts, int32_t cap, uint8_t* obs, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (B < 0 || (B > 0 && (!envs || !poses || !points || !counts || !obs)) || cap < 1)
    return fail(s, US_ERR_INVALID_ARG, "bad observation arguments");
  if (B == 0) return US_OK;
  us_plan* pl;
  us_status r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream));
  if (r != US_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(obs, 0, (size_t)B * 64000, st);
  if (e == cudaSuccess)
    e = launch_recon_observe(base_params(s, poses, 0, 0, nullptr), pl->d_items_batch, B, points, counts, cap, obs, st);
  return e == cudaSuccess ? US_OK : cuda_fail(s, e, "reconstruction observation");
}

us_status us_sim_render_timed(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                              uint64_t step, float* frames, float* kernel_ms, int32_t* n_kernels, void* stream) {
  if (!kernel_ms || !n_kernels) return fail(s, US_ERR_INVALID_ARG, "NULL timing outputs");
  *n_kernels = 0;
  us_status r = check_render_args(s, envs, B, poses, frames);
  if (r != US_OK || B == 0) return r;
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  if (!s->batched) return no_batched(s);
  RenderParams p = base_params(s, poses, seed, step, frames);
  p.work = pl->d_work;
  p.items = pl->d_items;
  p.n_items = B;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool two_pass = s->tuning.cluster_size == 1;
  cudaError_t e;
  if (two_pass && (e = two_pass_buffers(pl)) != cudaSuccess)
    return cuda_fail(s, e, "two-pass line buffer");
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(s, e, "events");
  const int nk = two_pass && !s->split.persistent ? 2 : 1;
  if (two_pass && s->split.persistent) {
    // the reset of the synchronisation words sits outside the timed kernel
    e = cudaMemsetAsync(pl->d_sync, 0, sizeof(unsigned) * split_sync_words(B), st);
    cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch_split_pass(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, 3, st);
    cudaEventRecord(ev[1], st);
  } else if (two_pass) {
    cudaEventRecord(ev[0], st);
    e = launch_split_pass(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, 0, st, plan_units(s, pl, st));
    cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = launch_split_pass(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, 1, st, plan_units(s, pl, st));
    cudaEventRecord(ev[2], st);
  } else {
    e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), st);
    cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch_fused(p, s->shape, st);
    cudaEventRecord(ev[1], st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[nk]);
  for (int k = 0; k < nk && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&kernel_ms[k], ev[k], ev[k + 1]);
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(s, e, "timed render");
  *n_kernels = nk;
  return US_OK;
}

us_status us_sim_sample_slices(us_sim* s, const us_env* envs, int32_t B, const float* poses, uint16_t* out,
                               void* stream) {
  us_status r = check_render_args(s, envs, B, poses, reinterpret_cast<float*>(out));
  if (r != US_OK || B == 0) return r;
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  const us_probe& p0 = s->probes[envs[0].probe_id].desc;
  for (int b = 1; b < B; ++b) {
    const us_probe& pb = s->probes[envs[b].probe_id].desc;
    if (pb.out_w != p0.out_w || pb.out_h != p0.out_h)
      return fail(s, US_ERR_INVALID_ARG, "sample_slices needs one output size for the whole batch");
  }
  RenderParams p = base_params(s, poses, 0, 0, nullptr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t npx = (size_t)p0.out_h * p0.out_w;
  cudaError_t e;
  if (s->d_href) {
    // raw HU and inside-fan flags of the batch, then the matching rewrites
    // the HU channel of the in-fan pixels
    if (pl->slice_px < (size_t)B * npx) {
      cudaFree(pl->d_slice_hu);
      cudaFree(pl->d_slice_fan);
      pl->d_slice_hu = nullptr;
      pl->d_slice_fan = nullptr;
      pl->slice_px = 0;
      if ((e = cudaMalloc(&pl->d_slice_hu, sizeof(float) * B * npx)) != cudaSuccess ||
          (e = cudaMalloc(&pl->d_slice_fan, (size_t)B * npx)) != cudaSuccess)
        return cuda_fail(s, e, "slice scratch");
      pl->slice_px = (size_t)B * npx;
    }
    if ((e = launch_slice_input(p, pl->d_items_batch, B, p0.out_h, p0.out_w, out, pl->d_slice_hu, pl->d_slice_fan,
                                st)) != cudaSuccess ||
        (e = launch_hist_match(pl->d_slice_hu, pl->d_slice_fan, B, (int)npx, s->d_href, s->href_nb, s->href_h0,
                               s->href_w, nullptr, out, st)) != cudaSuccess)
      return cuda_fail(s, e, "slice sampling launch");
    return US_OK;
  }
  e = launch_slice_input(p, pl->d_items_batch, B, p0.out_h, p0.out_w, out, nullptr, nullptr, st);
  return e == cudaSuccess ? US_OK : cuda_fail(s, e, "slice sampling launch");
}

us_status us_sim_set_hu_reference(us_sim* s, const int64_t* ref_cum, int32_t n_bins, float h0, float bin_width) {
  if (!s) return US_ERR_INVALID_ARG;
  if (!ref_cum || n_bins == 0) {
    cudaFree(s->d_href);
    s->d_href = nullptr;
    s->href_nb = 0;
    return US_OK;
  }
  if (n_bins < 1 || n_bins > kMaxMatchBins) return fail(s, US_ERR_INVALID_ARG, "n_bins must be in [1, 16384]");
  if (!std::isfinite(h0) || !std::isfinite(bin_width) || !(bin_width > 0.f))
    return fail(s, US_ERR_INVALID_ARG, "h0 and bin_width must be finite, bin_width > 0");
  if (ref_cum[0] < 0 || ref_cum[n_bins - 1] <= 0 || ref_cum[n_bins - 1] >= (1ll << 31))
    return fail(s, US_ERR_INVALID_ARG, "the reference total must be in [1, 2^31)");
  for (int k = 1; k < n_bins; ++k)
    if (ref_cum[k] < ref_cum[k - 1]) return fail(s, US_ERR_INVALID_ARG, "reference cumulative counts must not decrease");
  long long* d = nullptr;
  cudaError_t e;
  if ((e = upload(&d, reinterpret_cast<const long long*>(ref_cum), (size_t)n_bins)) != cudaSuccess)
    return cuda_fail(s, e, "reference histogram");
  cudaFree(s->d_href);
  s->d_href = d;
  s->href_nb = n_bins;
  s->href_h0 = h0;
  s->href_w = bin_width;
  return US_OK;
}

us_status us_sim_hist_match(us_sim* s, const float* hu, const uint8_t* mask, int32_t B, int32_t n_pix, float* out,
                            void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  if (B < 0 || n_pix < 1 || n_pix > (1 << 24)) return fail(s, US_ERR_INVALID_ARG, "B >= 0 and n_pix in [1, 2^24]");
  if (B == 0) return US_OK;
  if (!hu || !out) return fail(s, US_ERR_INVALID_ARG, "NULL image buffer");
  if (!s->d_href) return fail(s, US_ERR_INVALID_ARG, "no reference histogram (us_sim_set_hu_reference)");
  cudaError_t e = launch_hist_match(hu, mask, B, n_pix, s->d_href, s->href_nb, s->href_h0, s->href_w, out, nullptr,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? US_OK : cuda_fail(s, e, "histogram matching launch");
}

us_status us_sim_selftest_tile_wait(us_sim* s, const us_env* envs, int32_t B, const float* poses, float* frames,
                                    int64_t wait_cycles, void* stream) {
  us_status r = check_render_args(s, envs, B, poses, frames);
  if (r != US_OK || B == 0) return r;
  if (wait_cycles < 1 || wait_cycles > 2000000000ll) return fail(s, US_ERR_INVALID_ARG, "wait_cycles out of range");
  if (!s->batched || s->tuning.cluster_size != 1 || !s->tuning.persistent)
    return fail(s, US_ERR_UNSUPPORTED, "the tuning is not the persistent two-pass grid");
  us_plan* pl;
  if ((r = get_plan(s, envs, B, &pl, static_cast<cudaStream_t>(stream))) != US_OK) return r;
  cudaError_t e;
  if ((e = two_pass_buffers(pl)) != cudaSuccess) return cuda_fail(s, e, "two-pass line buffer");
  RenderParams p = base_params(s, poses, 0, 0, frames);
  p.items = pl->d_items;
  p.n_items = B;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((e = launch_split_wait_selftest(p, s->split, pl->d_beam, pl->beam_elems, pl->d_sync, B, wait_cycles, st)) != cudaSuccess)
    return cuda_fail(s, e, "self-test launch");
  return US_OK;
}

us_status us_sim_check(us_sim* s, void* stream) {
  if (!s) return US_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream");
  unsigned w = 0;
  if ((e = cudaMemcpy(&w, s->d_err, sizeof w, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(s, e, "error word");
  if (w) {
    cudaMemset(s->d_err, 0, sizeof w);
    if (w & kErrStagingTimeout)
      return fail(s, US_ERR_TIMEOUT, "a bounded device wait ran out (staging copy or a pass-B tile's lines)");
    if (w & kErrReconOverflow) return fail(s, US_ERR_INVALID_ARG, "a reconstruction point list reached its capacity");
    if (w & kErrNonFinitePose) return fail(s, US_ERR_INVALID_ARG, "a pose had a non-finite entry (rendered as water)");
    return fail(s, US_ERR_INTERNAL, "device consistency check failed");
  }
  return US_OK;
}

us_status us_sim_get_tuning(const us_sim* s, us_tuning* t) {
  if (!s || !t) return US_ERR_INVALID_ARG;
  *t = s->tuning;
  return US_OK;
}

us_status us_sim_set_tuning(us_sim* s, const us_tuning* t) {
  if (!s || !t) return US_ERR_INVALID_ARG;
  return apply_tuning(s, *t);
}

us_status us_sim_autotune(us_sim* s, const us_env* envs, int32_t B, const float* poses, float* frames,
                          const char* cache_path, void* stream) {
  us_status r = check_render_args(s, envs, B, poses, frames);
  if (r != US_OK) return r;
  if (B == 0) return US_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaDeviceProp prop;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || (e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
    return cuda_fail(s, e, "device query");
  // signature: GPU, probe set, batch (env list)
  uint64_t hp = 0;
  for (const ProbeHost& ph : s->probes) hp = fnv1a(&ph.desc, sizeof ph.desc, hp ? hp : 1469598103934665603ull);
  const uint64_t he = fnv1a(envs, sizeof(us_env) * (size_t)B);
  char sig[512];
  std::string gpu(prop.name);
  for (char& c : gpu)
    if (c == ' ') c = '_';
  std::snprintf(sig, sizeof sig, "%s sm%d probes=%016llx envs=%016llx B=%d", gpu.c_str(), prop.multiProcessorCount,
                (unsigned long long)hp, (unsigned long long)he, B);
  const int keep_graph = s->tuning.use_graph;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[768];
      int cs = 0, nw = 0, pg = 0, wl = 0;
      bool found = false;
      while (std::fgets(line, sizeof line, f)) {
        const size_t n = std::strlen(sig);
        int c0 = 0, n0 = 0, p0 = 0, w0 = 0;
        const int got = std::strncmp(line, sig, n) == 0
                            ? std::sscanf(line + n, " cs=%d nw=%d pg=%d wl=%d", &c0, &n0, &p0, &w0)
                            : 0;
        if (got >= 3) {   // lines written before the wedge choice have no wl: the widest wedge
          cs = c0, nw = n0, pg = p0, wl = got == 4 ? w0 : 0;
          found = true;
        }
      }
      std::fclose(f);
      if (found) {
        us_tuning t{cs, nw, keep_graph, pg, wl};
        if (apply_tuning(s, t) == US_OK) return US_OK;
      }
    }
  }
  // (cluster size, warps, persistent, pass-B wedge lines)
  static const int cand[][4] = {
      {8, 32, 0, 0},  {8, 16, 0, 0},  {8, 8, 0, 0},   {16, 32, 0, 0}, {16, 16, 0, 0}, {16, 8, 0, 0},
      {4, 32, 0, 0},  {4, 16, 0, 0},  {1, 32, 0, 32}, {1, 32, 0, 16}, {1, 32, 0, 8},  {1, 16, 0, 32},
      {1, 16, 0, 16}, {1, 16, 0, 8},  {1, 8, 0, 32},  {1, 8, 0, 16},  {1, 8, 0, 8},   {1, 32, 1, 32},
      {1, 32, 1, 16}, {1, 16, 1, 32}, {1, 16, 1, 16}, {1, 8, 1, 32},  {1, 8, 1, 16},  {1, 8, 1, 8}};
  float best = 1e30f;
  int best_cs = 0, best_nw = 0, best_pg = 0, best_wl = 0;
  cudaEvent_t a, b2;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b2)) != cudaSuccess) return cuda_fail(s, e, "events");
  for (const auto& c : cand) {
    us_tuning t{c[0], c[1], 0, c[2], c[3]};
    if (apply_tuning(s, t) != US_OK) continue;
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w)
      ok = do_render(s, envs, B, poses, 0x5EEDull, (uint64_t)w, frames, nullptr, nullptr, nullptr, nullptr, 0, st) == US_OK;
    cudaEventRecord(a, st);
    for (int k = 0; k < 5 && ok; ++k)
      ok = do_render(s, envs, B, poses, 0x5EEDull, (uint64_t)k, frames, nullptr, nullptr, nullptr, nullptr, 0, st) == US_OK;
    cudaEventRecord(b2, st);
    if (!ok || cudaEventSynchronize(b2) != cudaSuccess) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b2);
    if (ms < best) {
      best = ms;
      best_cs = c[0];
      best_nw = c[1];
      best_pg = c[2];
      best_wl = c[3];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b2);
  if (!best_cs) return fail(s, US_ERR_UNSUPPORTED, "no launch shape fits this probe set");
  us_tuning t{best_cs, best_nw, keep_graph, best_pg, best_wl};
  if ((r = apply_tuning(s, t)) != US_OK) return r;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s cs=%d nw=%d pg=%d wl=%d ms=%.4f\n", sig, best_cs, best_nw, best_pg, best_wl, best / 5.0f);
      std::fclose(f);
    }
  }
  return US_OK;
}

}  // extern "C"
