// us_sim_render_plain_static: the plain per-environment render with its
// scratch in a fixed array compiled into the library, for callers that
// must not allocate device memory while they render.
//
// The five plain kernels need, for the environment in flight, the label
// slice (1 byte per beam sample) and five FP32 beam planes (reflection
// impulses, later the log image; scatter pattern; energy; and the two
// axially filtered planes): 21 bytes per sample.  The array below holds that
// for beam grids of up to kStaticBeamSamples samples (256 lines x 512
// samples), 2.625 MiB.  Every GPU that loads this library holds the
// array until the process exits.  All calls share it, and it keeps the
// last call's contents; the kernels overwrite every element they read
// before reading it, so nothing needs clearing.  Two calls whose work
// overlaps on the GPU (different streams, or other processes' contexts do
// not share it) race on the array.
#include <cstdio>
#include <mutex>
#include <string>

#include "us_internal.h"

namespace ussim {

constexpr long long kStaticBeamSamples = 256LL * 512LL;
constexpr size_t kStaticScratchBytes = (size_t)kStaticBeamSamples * kPlainScratchBytesPerSample;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the host-side symbol is only a stand-in, never a device address).
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ussim

using namespace ussim;

extern "C" us_status us_sim_render_plain_static(us_sim* s, const us_env* envs, int32_t B, const float* poses,
                                                uint64_t seed, uint64_t step, float* frames, void* stream) {
  us_status r = sim_check_render_args(s, envs, B, poses, frames);
  if (r != US_OK || B == 0) return r;
  const int n_probes = (int)s->probes.size();
  for (int b = 0; b < B; ++b) {
    const us_env& e = envs[b];
    if (e.volume_id < 0 || e.volume_id >= (int)s->vols.size() || e.probe_id < 0 || e.probe_id >= n_probes) {
      s->last_error = "env " + std::to_string(b) + " has an out-of-range volume or probe id";
      return US_ERR_INVALID_ARG;
    }
    const us_probe& p = s->probes[e.probe_id].desc;
    if ((long long)p.n_lines * p.n_samples > kStaticBeamSamples) {
      s->last_error = "us_sim_render_plain_static: env " + std::to_string(b) + " has " +
                      std::to_string((long long)p.n_lines * p.n_samples) +
                      " beam samples; the static scratch holds at most 131072 (256 x 512)";
      return US_ERR_INVALID_ARG;
    }
  }
  void* base = nullptr;
  cudaError_t e = static_scratch(&base);
  if (e != cudaSuccess) {
    s->last_error = std::string("static scratch lookup: ") + cudaGetErrorString(e);
    return US_ERR_CUDA;
  }
  PlainScratch scr;
  unsigned char* b8 = static_cast<unsigned char*>(base);
  scr.R = reinterpret_cast<float*>(b8);
  scr.T = reinterpret_cast<float*>(b8 + 4 * kStaticBeamSamples);
  scr.E = reinterpret_cast<float*>(b8 + 8 * kStaticBeamSamples);
  scr.AR = reinterpret_cast<float*>(b8 + 12 * kStaticBeamSamples);
  scr.AT = reinterpret_cast<float*>(b8 + 16 * kStaticBeamSamples);
  scr.Y = scr.R;
  scr.lab = b8 + 20 * kStaticBeamSamples;

  // the same parameters as every other render entry point (options,
  // speckle key, volume-anchored map scales), with no debug exports
  RenderParams p = sim_render_params(s, poses, seed, step, frames);
  p.n_items = B;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long frame_off = 0;
  for (int b = 0; b < B; ++b) {
    const us_env& ev = envs[b];
    const ProbeHost& ph = s->probes[ev.probe_id];
    EnvItem it;
    it.b = b;
    it.vol = ev.volume_id;
    it.probe = ev.probe_id;
    it.pair = ev.volume_id * n_probes + ev.probe_id;
    it.frame_off = frame_off;
    it.beam_off = 0;
    frame_off += (((long long)ph.desc.out_w * ph.desc.out_h + 63) / 64) * 64;
    if ((e = launch_plain_env(p, it, ph, scr, st)) != cudaSuccess) {
      s->last_error = std::string("plain render launch: ") + cudaGetErrorString(e);
      return US_ERR_CUDA;
    }
  }
  return US_OK;
}
