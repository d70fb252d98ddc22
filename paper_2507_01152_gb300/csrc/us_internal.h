// Host-side internals of the ussim library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ussim.h"
#include "us_device.cuh"

namespace ussim {

// probe descriptor plus its derived FP64 quantities and device tables
struct ProbeHost {
  us_probe desc;
  double dr, dtheta, dlat_mid;
  int k_ax, k_lat;
  float2* d_lines = nullptr;
  float* d_wax = nullptr;
  float* d_wlat = nullptr;
  float2* d_lut = nullptr;
  DevTissue* d_tissue = nullptr;
  float* d_px = nullptr;
  float* d_pz = nullptr;
  std::vector<float2> lut_host;   // scan-conversion map (curvilinear)
  float4* d_wedge = nullptr;      // two-pass path: pixels grouped by wedge of wedge_G lines
  int* d_wedge_off = nullptr;
  int wedge_G = 0;
};

// global scratch of the plain path (one environment at a time): labels,
// the model's reflection impulses R, scatter pattern T and energy E, their
// axially filtered AR, AT, and the log image Y (Y may share R's storage:
// R is dead once AR is formed)
struct PlainScratch {
  uint8_t* lab = nullptr;
  float* R = nullptr;
  float* T = nullptr;
  float* E = nullptr;
  float* AR = nullptr;
  float* AT = nullptr;
  float* Y = nullptr;
};
// bytes of plain-path scratch per beam sample (lab 1, R/Y, T, E, AR, AT)
constexpr int kPlainScratchBytesPerSample = 1 + 5 * 4;

cudaError_t launch_plain(const RenderParams& p, const EnvItem* items_host, int n_items,
                         const ProbeHost* probes, PlainScratch& scr, cudaStream_t st);
// the same five kernels for one environment, on caller-given scratch
cudaError_t launch_plain_env(const RenderParams& p, const EnvItem& it, const ProbeHost& ph,
                             const PlainScratch& scr, cudaStream_t st);

// launch shape of the fused kernel and its dynamic shared-memory layout
struct FusedLayout {
  int off_r, off_y, off_lab, off_lrow, off_srow, off_rrow, off_yrow, off_wax, off_wlat, off_tis;  // byte offsets
};

struct FusedShape {
  int cs = 8;            // CTAs per cluster (one cluster renders one frame)
  int nw = 32;           // warps per CTA
  int sbuf_floats = 0;   // floats per CTA row buffer (max over probes of lines-per-CTA * row stride)
  FusedLayout lay{};
  size_t smem = 0;       // dynamic shared memory per CTA
  int clusters = 0;      // persistent grid, in clusters
};

// fills sbuf_floats / smem for the probe set; false if it cannot fit
bool fused_shape_fits(FusedShape& s, const std::vector<ProbeHost>& probes, int n_labels);
// is (cs, nw) one of the compiled instantiations?
bool fused_shape_known(int cs, int nw);
// set the kernel's shared-memory / cluster attributes (outside any capture)
cudaError_t fused_prepare(const FusedShape& s);
// occupancy-derived persistent grid (clusters resident at once)
cudaError_t fused_max_clusters(const FusedShape& s, int* clusters);
cudaError_t launch_fused(const RenderParams& p, const FusedShape& s, cudaStream_t st);

// two-pass path: lines per pass-A block G and per pass-B wedge GB (8, 16,
// 32), shared-memory layouts of both passes, blocks per item of each pass
// pass B tiles: GB lines x kChunk samples, kImageThreads threads per block
constexpr int kChunk = 128;
constexpr int kImageThreads = 256;
constexpr int kRowStride = kChunk + 4;   // shared row stride, floats (16-byte rows)
// pass A's padded rows (K zeros, NS samples, K zeros) in floats: one more
// element, which the two-output axial filter reads past an odd row's end,
// rounded up to 16 bytes, so that every row starts 16-byte aligned and every
// even sample offset of it is 8-byte aligned
__host__ __device__ inline int lines_row_stride(int NS, int K) { return (NS + 2 * K + 1 + 3) & ~3; }
struct SplitArgs {
  float2* beam = nullptr;   // axially filtered (AR, AT) pairs, beam layout (per item beam_off)
  float* ebeam = nullptr;   // energy E of every beam sample, same layout
  unsigned* work = nullptr;   // persistent grid: unit counter
  unsigned* done = nullptr;   // persistent grid: per pass-A group, 1 once its lines are written
  long long wait_cycles = 2000000000ll;   // persistent grid: bound of a tile's wait (SM clock cycles, ~1 s)
  int G = 32, GB = 32, gpi_lines = 0, gpi_image = 0;
  // two grids: the launch's work units, pass A's (item, group) then pass B's
  // (item, tile), only those inside each item's probe (null: every item has
  // gpi_lines / gpi_image units, those past its probe exit at once)
  const int2* units = nullptr;
  int n_units_a = 0, n_units_b = 0;
  int off_r = 0, off_wax = 0, off_tis = 0, off_lab = 0;   // pass A byte offsets
  int off_y = 0, off_wlat = 0;                 // pass B byte offsets
};
struct SplitUnits {
  const int2* d = nullptr;   // device: n_a pass-A units, then n_b pass-B units
  int n_a = 0, n_b = 0;
};
struct SplitShape {
  int G = 32;    // pass A lines per block (the tuning's warps_per_cta)
  int GB = 32;   // pass B lines per wedge: the widest whose buffers fit
  int GB_req = 0;   // requested pass B lines per wedge (0: the widest that fits)
  SplitArgs args{};
  size_t smem_lines = 0, smem_image = 0;
  bool persistent = false;        // one persistent grid instead of two
  int persist_grid[2] = {0, 0};   // resident blocks of the persistent grid (beam-keyed, anchored maps)
};
// the line buffer of a batch of beam_elems samples: (AR, AT) pairs, then
// the energy plane, 12 bytes a sample
constexpr size_t kLineBufferBytesPerSample = 12;
inline void set_line_buffer(SplitArgs& a, float* base, long long beam_elems) {
  a.beam = reinterpret_cast<float2*>(base);
  a.ebeam = base + 2 * beam_elems;
}
// words of synchronisation state the persistent two-pass grid needs for a
// batch of B environments (unit counter + a flag per group of >= 8 lines)
inline size_t split_sync_words(int B) { return 1 + (size_t)B * (1024 / 8); }
bool split_shape_fits(SplitShape& sh, const std::vector<ProbeHost>& probes, int n_labels);
cudaError_t split_prepare(SplitShape& sh);
// both passes over the first max_items entries of p.items (fewer if
// p.n_items_dev says so)
cudaError_t launch_split(const RenderParams& p, const SplitShape& sh, float* beam, long long beam_elems, unsigned* sync,
                         int max_items, cudaStream_t st, SplitUnits units = SplitUnits());
// one pass: 0 = lines (pass A), 1 = image (pass B)
// pass 0: pass A, 1: pass B (separate grids); 2: both in the persistent
// grid (resets `sync` first); 3: the persistent grid on a `sync` the
// caller has zeroed
cudaError_t launch_split_pass(const RenderParams& p, const SplitShape& sh, float* beam, long long beam_elems,
                              unsigned* sync, int max_items, int pass, cudaStream_t st,
                              SplitUnits units = SplitUnits());
// the two grids' work units of items (in launch order) for pass-A groups of
// G lines and pass-B tiles of GB lines
void build_split_units(const std::vector<EnvItem>& items, const std::vector<ProbeHost>& probes, int G, int GB,
                       std::vector<int2>& units, int& na, int& nb);
// the persistent grid with its unit counter started past every pass-A group
// and the given wait bound: no group publishes its lines, so every tile's
// wait runs out (self-test of the bounded wait)
cudaError_t launch_split_wait_selftest(const RenderParams& p, const SplitShape& sh, float* beam, long long beam_elems,
                                       unsigned* sync, int max_items, long long wait_cycles, cudaStream_t st);
void build_wedges(const std::vector<float2>& lut, int W, int H, int NL, int NS, int G, std::vector<float4>& entries,
                  std::vector<int>& off);

// items with score > thr, in batch order, and their count (device)
cudaError_t launch_gate_compact(const EnvItem* items, int B, const float* score, float thr, EnvItem* out, int* count,
                                cudaStream_t st);
// items the gate keeps (score <= thr) that the seeded audit selects (Philox
// word below t_audit), in batch order, their count and per-env flags
cudaError_t launch_audit_compact(const EnvItem* items, int B, const float* score, float thr, uint2 key,
                                 unsigned long long t_audit, EnvItem* out, int* count, uint8_t* flags,
                                 cudaStream_t st);

// a probe's H x W surrogate grid over its output field: probe-frame x of
// each column, z of each row (FP64 on the host, rounded once), and the
// inside-fan flag of each pixel
struct DevGridTab {
  const float* px;
  const float* pz;
  const uint8_t* mask;
};
cudaError_t launch_grid_slices(const RenderParams& p, const EnvItem* items_batch, int B, int H, int W,
                               const DevGridTab* tabs, void* out, cudaStream_t st);
// H x W frames -> each env's own output grid (p.frames, frame layout)
cudaError_t launch_resize(const RenderParams& p, const EnvItem* items_batch, int B, const float* src, int H, int W,
                          int max_out, cudaStream_t st);

// surrogate input of a batch on the output pixel grid: [B][H][W][8] BF16
cudaError_t launch_slice_input(const RenderParams& p, const EnvItem* items_batch, int B, int H, int W, void* out,
                               float* hu_raw, uint8_t* in_fan, cudaStream_t st);
// histogram matching of B images of n_pix values to the cumulative reference
// counts R[nb] (device); out (float) and/or slice (BF16 surrogate input,
// channel 1) receive the result
cudaError_t launch_hist_match(const float* hu, const uint8_t* mask, int B, int n_pix, const long long* R, int nb,
                              float h0, float w, float* out, void* slice, cudaStream_t st);

// 3-D probe: B poses -> B * E poses swept along each pose's elevation axis
cudaError_t launch_expand_elevation(const float* poses, int B, int E, float pitch, float* out, cudaStream_t st);

// reconstruction observation (recon.cu)
constexpr unsigned kErrReconOverflow = 16u;   // a reconstruction point list reached its capacity
cudaError_t launch_recon_update(const RenderParams& p, const EnvItem* items, int B, int bone, unsigned thr,
                                unsigned* bitmaps, long long words, int* points, int* counts, int cap, int max_lines,
                                cudaStream_t st);
cudaError_t launch_recon_observe(const RenderParams& p, const EnvItem* items, int B, const int* points,
                                 const int* counts, int cap, unsigned char* obs, cudaStream_t st);

// the render parameters every render entry point starts from (handle's
// tables, options, speckle key of (seed, step), anchored-map scales), and
// the argument checks they share (NULL buffers, 16-byte frames, 4-byte poses)
RenderParams sim_render_params(const us_sim* s, const float* poses, uint64_t seed, uint64_t step, float* frames);
us_status sim_check_render_args(us_sim* s, const us_env* envs, int B, const float* poses, float* frames);

// label check at creation: max label of a volume
cudaError_t max_label(const uint8_t* labels, long long n, unsigned* d_out, cudaStream_t st);
// corner records of V's HU grid into out (corner_records(nx, ny, nz)
// records; V.qy set)
inline int corner_quads_y(int ny) { return (ny + 4) / 4; }
inline long long corner_records(int nx, int ny, int nz) {
  return (long long)(nx + 1) * corner_quads_y(ny) * 4 * (nz + 1);
}
cudaError_t pack_corners(const DevVolume& V, uint4* out, cudaStream_t st);
// V's labels in 4 x 4 x 4 bricks into out (label_bricks_bytes(nx, ny, nz)
// bytes; V.bx, V.by set)
inline long long label_bricks_bytes(int nx, int ny, int nz) {
  return (long long)((nx + 3) / 4) * ((ny + 3) / 4) * ((nz + 3) / 4) * 64;
}
cudaError_t pack_labels(const DevVolume& V, uint8_t* out, cudaStream_t st);

}  // namespace ussim

// a batch signature's precomputed work list and workspace, one per
// (signature, stream)
struct us_plan {
  std::vector<ussim::EnvItem> items_sorted;  // fused order: costliest first
  std::vector<ussim::EnvItem> items_batch;   // caller order
  ussim::EnvItem* d_items = nullptr;         // device copy of items_sorted
  ussim::EnvItem* d_items_batch = nullptr;   // device copy of items_batch
  ussim::EnvItem* d_items_gated = nullptr;   // device-built subset for gated renders
  int* d_gated_count = nullptr;
  unsigned* d_work = nullptr;                // cluster path: this plan's work counter
  ussim::EnvItem* d_items_audit = nullptr;   // device-built subset for the gate's physics audit
  int* d_audit_count = nullptr;
  long long frame_floats = 0, beam_elems = 0;
  float* d_beam = nullptr;                   // two-pass path: filtered lines of the batch
  int g_pers = -1;                           // captured graph's persistent flag
  unsigned* d_sync = nullptr;                // two-pass path: persistent grid's counter and flags
  int2* d_units = nullptr;                   // two grids: work units of items_sorted for units_G / units_GB
  int units_G = 0, units_GB = 0, units_na = 0, units_nb = 0;
  float* d_slice_hu = nullptr;               // slice sampling with histogram matching: raw HU
  uint8_t* d_slice_fan = nullptr;            //   and inside-fan flags of the batch's pixels
  size_t slice_px = 0;
  // captured render (fused: work-counter reset + kernel; two-pass: both
  // kernels), re-parameterised per call
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<cudaGraphNode_t> gnodes;
  std::vector<cudaKernelNodeParams> gkps;
  int g_cs = 0, g_nw = 0, g_gb = 0;   // captured graph's shape (pass B wedge lines)
  const int2* g_units = nullptr;       // the work-unit list the captured graph's kernels read
};

struct us_sim {
  std::vector<us_volume> vols;
  std::vector<ussim::ProbeHost> probes;
  std::vector<us_tissue> table;
  us_options opt{};
  int n_labels = 0;

  ussim::DevVolume* d_vols = nullptr;
  ussim::DevProbe* d_probes = nullptr;
  ussim::DevPair* d_pairs = nullptr;
  std::vector<uint8_t*> d_pair_D;
  std::vector<uint4*> d_hu8;   // corner records per volume (null entries: not built)
  std::vector<uint8_t*> d_lab4;   // bricked labels per volume (null entries: not built)
  long long* d_href = nullptr;  // reference cumulative counts of the HU histogram matching (null: off)
  int href_nb = 0;
  float href_h0 = 0.f, href_w = 1.f;
  std::vector<ussim::DevVolume> dev_vols;

  ussim::PlainScratch scratch;
  unsigned* d_err = nullptr;
  unsigned* d_work = nullptr;

  ussim::FusedShape shape;     // cluster path (also serves gated renders when it is not tuned in)
  ussim::SplitShape split;     // two-pass path (tuning.cluster_size == 1)
  us_tuning tuning{1, 16, 1};
  bool batched = true;         // a batched launch shape fits the probe set

  std::map<std::string, us_plan> plans;

  // surrogate grids of every probe, per grid size (H, W): device tables and
  // the allocations behind them
  struct GridTabs {
    ussim::DevGridTab* d_tabs = nullptr;
    std::vector<void*> bufs;
  };
  std::map<std::pair<int, int>, GridTabs> grids;

  // 3-D probe: swept poses
  float* d_poses3d = nullptr;
  size_t poses3d_cap = 0;

  // staging for us_sim_render_host; its frame copies run on copy_stream,
  // each sub-batch's after copy_ev[k] (created on first use)
  float* d_host_poses = nullptr;
  float* d_host_frames = nullptr;
  size_t host_poses_cap = 0, host_frames_cap = 0;
  static constexpr int kHostSub = 4;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[kHostSub] = {};

  std::string last_error;
};
