/*
 * ussim.h — C ABI of the batched model-based ultrasound render.
 *
 * One call renders one ultrasound frame per environment for a batch of
 * environments, each with its own probe pose, volume and probe type.  The
 * simulation is the convolution-based image model of SonoGym App. B.2
 * (after Salehi et al. 2015), applied to the 2-D label and CT slices that
 * the probe's image plane cuts out of each environment's volumes
 * (Fig. 2 caption; Sec. 4 "Ultrasound simulation"):
 *
 *   E(u) = E0 exp(-f * int_0^y alpha)            remaining energy   (App. B.2)
 *   R_imp(u) = |E cos(theta) (Z(y+dy)-Z(y))/(Z(y+dy)+Z(y))| at boundaries G
 *   T(u) = N0 sigma0 + mu0 if N1 <= mu1 else 0       scatter pattern (App. B.2)
 *   I    = P (x) R_imp + E . (P (x) T),  P a 2-D Gaussian PSF      (App. B.2)
 *          (the backscatter B = E . P (x) T as printed: the pattern is
 *          blurred, then scaled by the energy at the pixel)
 *
 * followed by log compression and, for curvilinear probes, scan conversion
 * to a Cartesian image.  Readings taken where the paper is silent (noise
 * keying, impedance from HU, incidence-angle stencil, transmission loss,
 * log and scan-conversion conventions) are stated beside each switch.
 *
 * Conventions for every entry point:
 *  - Pointers documented as DEVICE point to memory of the current CUDA
 *    device; HOST pointers to ordinary (preferably pinned) host memory.
 *  - Volumes, poses and frames are caller-owned and borrowed: they must stay
 *    valid until the work that uses them has finished on `stream`.  The
 *    library owns only its derived tables, plans and workspace.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream are asynchronous with respect to
 *    the host unless stated otherwise.
 *  - Argument errors are detected on the host before any launch and return
 *    US_ERR_INVALID_ARG with a message in us_sim_last_error().  Errors found
 *    on the device (non-finite pose entries) set a sticky error word that
 *    us_sim_check() reads.  No entry point aborts or traps.
 *  - One handle may be used from one host thread at a time.  Its batched
 *    renders keep their workspace (work lists, line buffer, the persistent
 *    grid's counters, the cluster kernel's work counter, the captured graph)
 *    per batch signature and stream, allocated on first use: renders on
 *    different streams may overlap; two renders of one signature on one
 *    stream are ordered by the stream.  The error word is per handle (its
 *    bits are sticky, so concurrent renders only add to it).
 *    A plan is kept for every (signature, stream) pair seen, until
 *    us_sim_destroy.  us_sim_render_plain and us_sim_render_debug's plain path
 *    share one per-handle scratch, and us_sim_render_host its per-handle staging
 *    buffers: order those calls.  us_sim_render_plain_static shares one
 *    scratch array per process.
 *  - Output is a pure function of (inputs, seed, step): two calls with the
 *    same arguments produce bit-identical frames.
 */
#ifndef USSIM_H
#define USSIM_H

#include <stdint.h>

#if defined(__GNUC__)
#define US_API __attribute__((visibility("default")))
#else
#define US_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  US_OK = 0,
  US_ERR_INVALID_ARG = 1, /* bad argument; nothing was launched */
  US_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  US_ERR_OOM = 3,         /* device or host allocation failed */
  US_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
  US_ERR_UNSUPPORTED = 5, /* valid request this build does not handle */
  US_ERR_INTERNAL = 6     /* device-side consistency check failed */
} us_status;

typedef struct us_sim us_sim; /* opaque */

/* A label map and its CT volume on the same grid (Sec. 4 "Assets": CT
 * volumes with label maps).  DEVICE pointers, layout [nz][ny][nx] with x
 * fastest; voxel (i, j, k) is centred at (i, j, k) * voxel_mm in the
 * volume frame (mm).  Borrowed for the life of the handle.  Samples
 * outside the grid read label 0 and HU 0 (water).  The contents are read
 * at us_sim_create: the labels are range-checked and the HU grid is copied
 * into a library-owned corner layout (16 bytes per cell, (nx+1)(ny+1)(nz+1)
 * cells, unless us_options.volume_layout = 1) that the trilinear
 * interpolation reads.  After changing a
 * volume's contents, call us_sim_refresh_volumes before the next render. */
typedef struct {
  const uint8_t* labels;
  const int16_t* hu;
  int32_t nx, ny, nz;
  float voxel_mm;
} us_volume;

/* Acoustic settings of one tissue class; the table index is the label
 * (App. B.2: attenuation alpha, impedance, scatter mu0 / sigma0 / mu1). */
typedef struct {
  float alpha_db_cm_mhz; /* attenuation, dB/(cm MHz) */
  float z_mrayl;         /* impedance, MRayl (used when z_mode = 1) */
  float mu0, sigma0;     /* scatter mean / std: T~ = N0 sigma0 + mu0 */
  float mu1;             /* density threshold: scatter where N1 <= mu1; -inf = never */
} us_tissue;

/* Probe geometry and imaging settings.
 * kind 0 (linear): line l at lateral offset (l - (NL-1)/2) * pitch_mm,
 *   sample s at depth s * depth_mm / NS; output image NS rows x NL columns
 *   (out_h = n_samples, out_w = n_lines required).
 * kind 1 (curvilinear): apex radius_mm behind the face, line l at angle
 *   (l - (NL-1)/2) * fan/(NL-1), sample s at radius radius_mm + s*depth/NS;
 *   scan-converted to out_h x out_w over the fan's bounding box.
 * PSF: separable Gaussian on the beam grid, sigma in mm, half-width
 * ceil(3 sigma / spacing) taps (at most 48), lateral spacing = pitch (linear)
 * or mid-depth arc length (curvilinear).  Log compression: pixel =
 * clamp((20 log10(I / e0) + dyn_range_db) / dyn_range_db, 0, 1). */
typedef struct {
  int32_t kind;
  int32_t n_lines, n_samples; /* 2 <= NL <= 1024, 2 <= NS <= 1024 */
  float depth_mm;
  float pitch_mm;             /* linear */
  float fan_deg, radius_mm;   /* curvilinear */
  int32_t out_w, out_h;
  float f_mhz, e0, psf_sigma_ax_mm, psf_sigma_lat_mm, dyn_range_db;
} us_probe;

/* Model switches.
 * refl_power 1: R = G E |cos(theta) r| (App. B.2); 2: G E (cos(theta) r)^2,
 *   the intensity reflection coefficient.
 * transmission 1: the energy also loses ln(1 - r^2) at each boundary;
 *   0: attenuation only (App. B.2 as printed).
 * z_mode 0: Z = max(HU + 1024, 1), "proportional to CT intensity" (App. B.2);
 *   1: Z from the tissue table.
 * speckle 1: N0, N1 from Philox-4x32-10 keyed by (env, line, sample, seed,
 *   step); 0: T = mu0 everywhere.
 * speckle_anchor 1 (with speckle 1): N0, N1 are maps fixed over the volume
 *   (App. B.2: sampled over 3-D space once), so the speckle moves with the
 *   tissue: speckle_levels scales (1..3, the multi-scale maps of App. B.2) of
 *   cubic cells of edge speckle_cell_mm * 2^k anchored at the volume origin;
 *   a sample takes its nearest cell at each scale, whose Philox-4x32-10
 *   words (counter = cell x, y, z, k << 16 | volume index; key = seed, no
 *   step) give standard normals; N = sum_k a_k N_k with a_k proportional to
 *   2^(-k/2), unit variance.  T = N0 sigma0 + mu0 where N1 <= mu1.
 *   0: the beam-keyed maps above (speckle_levels, speckle_cell_mm unused).
 * volume_layout 0: the trilinear interpolation reads a library-owned copy
 *   of each HU grid in corner records (the 8 corners of a cell in one 16-byte
 *   record: one load per sample, 16 bytes of device memory per cell);
 *   1: it reads the caller's HU grid (eight loads per sample, no copy).
 *   Both give identical images. */
typedef struct {
  int32_t refl_power, transmission, z_mode, speckle;
  int32_t speckle_anchor, speckle_levels;
  float speckle_cell_mm;
  int32_t volume_layout;
} us_options;

/* One environment of a batch: which volume and which probe it uses. */
typedef struct {
  int32_t volume_id, probe_id;
} us_env;

/* Launch shape of the batched render.
 * cluster_size 4, 8 or 16: persistent cluster kernel, one thread-block
 *   cluster per environment frame (the frame stays in distributed shared
 *   memory); warps_per_cta 8, 16 or 32 (4-CTA clusters: 16 or 32).
 * cluster_size 1: two-pass path without clusters, warps_per_cta (8, 16 or
 *   32) lines per pass-A block; pass B works on tiles of wedge_lines (8, 16
 *   or 32; 0: the widest whose buffers fit four blocks per SM, else three,
 *   two, one) lines x 128 samples.  The axially filtered lines go through a global buffer of
 *   the batch's beam size, allocated on first use per batch signature.
 *   persistent 0: the two passes are two grids; 1: one cooperative grid of
 *   resident blocks takes pass-A groups, then pass-B tiles, from a counter,
 *   and a tile starts as soon as the groups holding its lines are written
 *   (fills the last wave of a small batch).  Same frames as the cluster
 *   kernel either way.
 * Default after us_sim_create: the first of {1, 16, 1, 0, 0}, {1, 8, 1, 0, 0},
 * {1, 32, 1, 0, 0}, {8, 32, 1, 0, 0}, {16, 16, 1, 0, 0}, {16, 8, 1, 0, 0} that fits the
 * probe set.  If none fits, the simulator is still created: the batched
 * entry points then return US_ERR_UNSUPPORTED and us_sim_render_plain
 * renders. */
typedef struct {
  int32_t cluster_size;  /* 1, 4, 8 or 16 */
  int32_t warps_per_cta; /* 8, 16 or 32 */
  int32_t use_graph;     /* 1: replay a captured CUDA graph per batch signature
                            (not on the legacy NULL stream, nor while the
                            caller's stream is itself being captured) */
  int32_t persistent;    /* two-pass path: 0 two grids, 1 one persistent grid;
                            must be 0 for the cluster path */
  int32_t wedge_lines;   /* two-pass path: pass-B tile lines, 0 (widest that
                            fits), 8, 16 or 32; must be 0 for the cluster path */
} us_tuning;

/* Create a simulator (the per-environment assets of Sec. 4 "Ultrasound
 * simulation" and App. B.2: CT volume and label map, tissue acoustic
 * settings, probe geometry).  Copies the descriptors, builds the derived tables
 * (per-line geometry, PSF taps, scan-conversion maps, tissue constants,
 * N1 thresholds) and checks on the device that every label is below
 * n_labels (synchronous).  vols/labels/hu stay borrowed.  opt may be NULL
 * (defaults: refl_power 1, transmission 1, z_mode 0, speckle 1).
 * Errors: US_ERR_INVALID_ARG (bad sizes, NULL pointers, label out of
 * range), US_ERR_OOM, US_ERR_CUDA.  *out is NULL on error. */
US_API us_status us_sim_create(const us_volume* vols, int32_t n_vols, const us_tissue* table,
                        int32_t n_labels, const us_probe* probes, int32_t n_probes,
                        const us_options* opt, us_sim** out);

/* Re-read every volume's contents after the caller changed them: checks
 * the labels against the tissue table and rebuilds the corner layout of
 * the HU grid (App. B.2's image model samples the CT by trilinear
 * interpolation; the layout holds the 8 corners of each cell together).
 * Synchronous on `stream` (NULL = legacy default stream); no render of this
 * handle may run meanwhile.  Errors: US_ERR_INVALID_ARG (a label outside
 * the table; the handle keeps its previous corner layout for volumes not
 * yet re-read), US_ERR_CUDA. */
US_API us_status us_sim_refresh_volumes(us_sim* sim, void* stream);

/* Release every resource of the handle (waits for its work to finish). */
US_API void us_sim_destroy(us_sim* sim);

/* Frame layout for a batch (one H x W image per environment, App. B.2's
 * I in R^(H x W); Sec. 4: the batch of parallel environments): offsets[b] is
 * the first float of frame b in the frame buffer (row-major out_h x out_w),
 * offsets[B] the total size in floats.  Each frame starts on a 256-byte
 * boundary.  offsets: HOST, B+1.  Errors: US_ERR_INVALID_ARG (NULL handle,
 * envs or offsets; B < 0; an id out of range). */
US_API us_status us_sim_frame_layout(const us_sim* sim, const us_env* envs, int32_t B, int64_t* offsets);

/* Beam-grid layout for the debug exports: offsets[b] = first element of
 * env b's [NL][NS] grid.  offsets: HOST, B+1. */
US_API us_status us_sim_beam_layout(const us_sim* sim, const us_env* envs, int32_t B, int64_t* offsets);

/* Render one frame per environment (Fig. 2 caption and Sec. 4 "Ultrasound
 * simulation": probe pose -> image plane -> label / CT slice -> image;
 * App. B.2: the image model above), all environments of the batch in the
 * batched launch shape the handle is tuned to (us_sim_get_tuning): by
 * default the two-pass path (pass A per group of lines: slice, scanline
 * model, axial PSF; pass B per tile: lateral PSF, image, log, scan
 * conversion), in two grids or one persistent grid; or the cluster kernel
 * (one thread-block cluster per frame).  All shapes give the same bits.
 * Replays a captured CUDA graph per batch signature when use_graph is set.
 * envs: HOST [B]; poses: DEVICE float [B][3][4], probe frame (x lateral,
 * y elevation, z along the beam, mm) -> volume frame (mm), 4-byte aligned;
 * frames: DEVICE, laid out by us_sim_frame_layout, 16-byte aligned,
 * caller-owned.  B = 0 is a no-op.  Errors: US_ERR_INVALID_ARG (NULL or
 * misaligned buffers, B < 0, ids out of range), US_ERR_UNSUPPORTED (no
 * batched shape fits the probe set: use us_sim_render_plain), US_ERR_OOM
 * (first use of a batch signature allocates its work list and line
 * buffer), US_ERR_CUDA; non-finite poses render as water and set the error
 * word that us_sim_check reads. */
US_API us_status us_sim_render(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                        uint64_t seed, uint64_t step, float* frames, void* stream);

/* Same result through the plain per-environment form (the same App. B.2
 * model, Sec. 4's batch rendered one environment at a time): for each
 * environment in turn, separate kernels for slicing, the scanline model,
 * the two PSF passes and scan conversion, through per-handle scratch (the
 * comparison baseline).  Arguments and errors as us_sim_render, without
 * US_ERR_UNSUPPORTED. */
US_API us_status us_sim_render_plain(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                              uint64_t seed, uint64_t step, float* frames, void* stream);

/* Render with no device allocation in the call.  The paper has no
 * counterpart; this serves callers that must not allocate device memory
 * while they render (a control loop whose allocations could stall, or a
 * process whose device memory is already fully claimed by its own
 * allocator).  Same frames as us_sim_render_plain (same kernels, frame
 * layout of us_sim_frame_layout), but the per-environment scratch lives in
 * a fixed 2.625 MiB array compiled into the library, which every GPU that
 * loads the library holds until the process exits.  Limit: each env's
 * beam grid must have at most 256 x 512 = 131072 samples (n_lines x
 * n_samples), else US_ERR_INVALID_ARG before any launch.  The call makes
 * no cudaMalloc / cudaFree and no allocating library call.  The first call
 * on a device looks up the array's device address (once per device); make
 * that first call before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU race on it, so serialise them (one
 * stream).  Nothing in it needs clearing; every element is written before
 * it is read. */
US_API us_status us_sim_render_plain_static(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                                            uint64_t seed, uint64_t step, float* frames, void* stream);

/* Render with intermediate exports for testing (the stages of Fig. 2 and
 * App. B.2: the label slice, the image I before and after log compression).
 * path 0 = the tuned batched shape, 1 = plain.  envelope (float), logimg
 * (float), nn_index (int32, -1 outside the volume), label (uint8): DEVICE,
 * laid out by us_sim_beam_layout, [NL][NS] per env; any may be NULL.
 * envelope is I = P (x) R_imp + E (P (x) T) before log compression.
 * Errors as us_sim_render. */
US_API us_status us_sim_render_debug(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                              uint64_t seed, uint64_t step, float* frames, float* envelope,
                              float* logimg, int32_t* nn_index, uint8_t* label, int32_t path,
                              void* stream);

/* Render from HOST poses into HOST frames: copies the poses in and the
 * frames out through library-owned device buffers (grown on demand).
 * Returns after the frames are in host memory (synchronous).  A batch of
 * 16 MB of frames or more renders as two to four contiguous sub-batches
 * of halving size (same frames: each env keeps its batch index), each
 * copied out on a library-owned stream while the next renders; the copies
 * overlap the renders when frames_host is pinned (page-locked) memory. */
US_API us_status us_sim_render_host(us_sim* sim, const us_env* envs, int32_t B, const float* poses_host,
                             uint64_t seed, uint64_t step, float* frames_host, void* stream);

/* Reference histogram of the CT histogram matching (Sec. 3: the learned
 * simulator's input CT slices are matched in intensity histogram to a
 * subset of its training CT images).  ref_cum: HOST int64 [n_bins], the
 * reference's cumulative counts over n_bins bins of width bin_width from h0
 * (bin k(v) = clamp(floor((v - h0) / bin_width), 0, n_bins - 1), FP32),
 * non-decreasing with 0 < ref_cum[n_bins - 1] < 2^31; n_bins in [1, 16384].
 * Copied (synchronous).  ref_cum NULL or n_bins 0 removes the reference.
 * Errors: US_ERR_INVALID_ARG, US_ERR_CUDA. */
US_API us_status us_sim_set_hu_reference(us_sim* sim, const int64_t* ref_cum, int32_t n_bins, float h0,
                                         float bin_width);

/* Histogram matching of B images of n_pix CT values to the reference
 * (discrete histogram specification): per image, S[k] = the number of its
 * considered pixels in bins 0..k, n = S[n_bins - 1], N = the reference
 * total; bin k maps to the first reference bin m with ref_cum[m] * n >=
 * S[k] * N (exact 64-bit integers), and a considered pixel becomes that
 * bin's centre h0 + (m + 0.5) * bin_width (FP32).  hu, out: DEVICE float
 * [B][n_pix] (out may equal hu; values finite); mask: DEVICE uint8
 * [B][n_pix], nonzero = considered, or NULL (all).  Pixels not considered,
 * and images without a considered pixel, are copied unchanged.
 * n_pix in [1, 2^24].  Errors: US_ERR_INVALID_ARG (also: no reference set),
 * US_ERR_CUDA. */
US_API us_status us_sim_hist_match(us_sim* sim, const float* hu, const uint8_t* mask, int32_t B, int32_t n_pix,
                                   float* out, void* stream);

/* Input of the learned surrogate (ussim_surrogate.h) for a batch: the
 * label and CT slices on each env's output pixel grid (Fig. 2: the slices
 * the simulators map to images).  out: DEVICE [B][out_h][out_w][8] BF16,
 * channels (label / 4, clamp(HU / 1000, -1, 3), inside-fan flag, 0 x 5).
 * Curvilinear probes: the scan-conversion grid; linear: the beam grid
 * (row = sample, column = line).  Every env of the batch must have the
 * same output size.  Same voxel-coordinate path as the render.  With a
 * reference histogram set (us_sim_set_hu_reference), the HU channel of each
 * in-fan pixel carries its histogram-matched HU instead (per env slice, see
 * us_sim_hist_match); pixels outside the fan keep the sampled HU.  The raw
 * slices then pass through library-owned buffers (5 bytes per pixel of the
 * batch, allocated on first use per batch signature). */
US_API us_status us_sim_sample_slices(us_sim* sim, const us_env* envs, int32_t B, const float* poses, uint16_t* out,
                                      void* stream);

/* Physics fallback for frames a learned surrogate rendered (App. B.2 has a
 * model-based and a learning-based simulator; here the model-based one
 * judges and replaces the learned one's frames): re-render (into
 * `frames`, same layout as us_sim_render) only the envs whose score[b]
 * exceeds `threshold`, leaving the other frames untouched.  score: DEVICE
 * [B] (e.g. the surrogate's predicted error); the subset is selected on the
 * device, so nothing waits for the host.  n_rendered: DEVICE int32 (may be
 * NULL) receives the number of frames re-rendered.  B <= 32768. */
US_API us_status us_sim_render_gated(us_sim* sim, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                                     uint64_t step, float* frames, const float* score, float threshold,
                                     int32_t* n_rendered, void* stream);

/* The physics audit of the surrogate's error gate (App. B.2's model-based
 * simulator checking its learning-based one; the paper has no gate, this
 * is the library's reading): among the envs the gate keeps (score[b] <=
 * threshold, as us_sim_render_gated), env b is audited when word 0 of
 * Philox-4x32-10 on counter (0, 0, b, 2), key = the render key of
 * (seed, step), is below floor(fraction 2^32): a seeded subset of about
 * that fraction, fresh every step.  The audited envs are rendered by
 * physics into audit_frames (DEVICE, the batch's frame layout; the other
 * frames are left untouched), so that the surrogate frame in the caller's
 * own buffer can be compared with its physics twin.  flags: DEVICE uint8
 * [B] (may be NULL), 1 where audited; n_audited: DEVICE int32 (may be
 * NULL).  fraction in [0, 1]; B <= 32768.  Errors as us_sim_render_gated.
 * Uses its own work list, but the line buffer of the batch signature like
 * every batched render (order it with other renders of the same batch). */
US_API us_status us_sim_render_audit(us_sim* sim, const us_env* envs, int32_t B, const float* poses, uint64_t seed,
                                     uint64_t step, float* audit_frames, const float* score, float threshold,
                                     float fraction, uint8_t* flags, int32_t* n_audited, void* stream);

/* Surrogate input on a common grid for a batch of mixed probes (App. B.2's
 * learned simulator maps the slices to images; one network size serves
 * every probe): each env's label / CT slice sampled on an H x W grid of
 * pixel centres spanning that env's output field, channels as in
 * us_sim_sample_slices.  Curvilinear: the fan's bounding box (the
 * scan-conversion field) at H x W, inside-fan flag from the same test;
 * linear: x = ((c + 1/2) NL / W - 1/2 - (NL - 1) / 2) pitch,
 * z = ((r + 1/2) NS / H - 1/2) depth / NS, flag 1.  Pixel positions are
 * computed in FP64 on the host and rounded once to FP32; the voxel path is
 * the render's.  Probes of any output size may share the batch.  out:
 * DEVICE [B][H][W][8] BF16, 16-byte aligned.  H, W in [2, 4096].  The first
 * call for a grid size builds its tables (synchronous, library-owned).
 * Errors: US_ERR_INVALID_ARG, US_ERR_OOM, US_ERR_CUDA. */
US_API us_status us_sim_sample_slices_grid(us_sim* sim, const us_env* envs, int32_t B, const float* poses, int32_t H,
                                           int32_t W, uint16_t* out, void* stream);

/* Surrogate frames on the common grid back to each env's own output grid:
 * output pixel (r, c) of env b's out_h x out_w frame reads src[b] (DEVICE
 * FP32 [B][H][W], the same field) at fy = (r + 1/2) H / out_h - 1/2,
 * fx = (c + 1/2) W / out_w - 1/2, clamped to the grid, bilinearly;
 * curvilinear pixels outside the fan are 0, as in the physics frame.
 * frames: DEVICE, laid out by us_sim_frame_layout, 16-byte aligned.  H, W
 * in [2, 4096].  Errors: US_ERR_INVALID_ARG, US_ERR_CUDA. */
US_API us_status us_sim_resize_frames(us_sim* sim, const us_env* envs, int32_t B, const float* src, int32_t H,
                                      int32_t W, float* frames, void* stream);

/* Self-test of the persistent two-pass grid's bounded wait (not a render):
 * launches the grid of the current tuning (which must be {1, G, *, 1})
 * for this batch with its unit counter started past every pass-A group,
 * so no group publishes its lines and every pass-B tile's wait runs out
 * after wait_cycles SM clock cycles (1 .. 2e9).  The tiles then return
 * without touching `frames` (DEVICE, the batch's frame layout) and set the
 * error word, so the following us_sim_check returns US_ERR_TIMEOUT; the
 * context stays usable.  Asynchronous on `stream`.  Errors: US_ERR_INVALID_ARG,
 * US_ERR_UNSUPPORTED (another tuning), US_ERR_CUDA. */
US_API us_status us_sim_selftest_tile_wait(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                                           float* frames, int64_t wait_cycles, void* stream);

/* Wait for `stream` and read the sticky device error word: US_OK;
 * US_ERR_INVALID_ARG if a pose had a non-finite entry (that frame renders
 * as water); US_ERR_TIMEOUT if a bounded device wait ran out (that unit's
 * output is missing).  Clears the word. */
US_API us_status us_sim_check(us_sim* sim, void* stream);

/* Read the batched render's launch shape (a property of this build's
 * kernels; the paper batches environments, Sec. 4, without a stated
 * kernel design).  Errors: US_ERR_INVALID_ARG (NULL). */
US_API us_status us_sim_get_tuning(const us_sim* sim, us_tuning* t);
/* Set the batched render's launch shape; invalid shapes are rejected
 * (US_ERR_INVALID_ARG), shapes whose buffers do not fit this probe set in
 * shared memory too (US_ERR_UNSUPPORTED). */
US_API us_status us_sim_set_tuning(us_sim* sim, const us_tuning* t);

/* Time the batched render (the App. B.2 model over Sec. 4's batch of
 * environments) over the candidate launch shapes (cluster and two-pass) on
 * this batch (synchronous, renders into `frames`), keep the fastest, and
 * append it to the text cache at cache_path (may be NULL: no cache).  If
 * cache_path already holds an entry for this GPU, probe set and batch
 * signature it is used without timing.  Arguments as us_sim_render.
 * Errors: as us_sim_render; US_ERR_UNSUPPORTED if no shape fits. */
US_API us_status us_sim_autotune(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                          float* frames, const char* cache_path, void* stream);

/* Volumetric frames of a 3-D probe (Sec. 4, Task 3: H x W x E images; the
 * surgery task's probe is 50 x 37 x 5 at 2 x 2 x 10 mm, App. C): every
 * environment's probe plane is swept over n_elev (1..64) parallel planes at
 * elevation offsets y_e = (e - (n_elev - 1) / 2) * elev_pitch_mm along the
 * pose's own y axis (t' = t + R[:, 1] y_e, in FP32 on the device), and each
 * plane is rendered as a 2-D frame of the expanded batch, entry b * n_elev + e
 * (its own speckle: environment index b * n_elev + e).  frames: device, laid
 * out as us_sim_frame_layout of the expanded env list (env b repeated
 * n_elev times).  poses: device [B][3][4].  Errors as us_sim_render, plus
 * US_ERR_INVALID_ARG for n_elev or the pitch out of range. */
US_API us_status us_sim_render_3d(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                                  int32_t n_elev, float elev_pitch_mm, uint64_t seed, uint64_t step,
                                  float* frames, void* stream);

/* The elevation sweep of us_sim_render_3d on its own: out[b * n_elev + e] =
 * pose b translated by y_e = (e - (n_elev - 1) / 2) * elev_pitch_mm along its
 * own y axis (t' = t + R[:, 1] y_e; FP32, one rounding per product and sum),
 * the rotation unchanged (Sec. 4, Task 3: H x W x E volumetric images).
 * poses: DEVICE [B][3][4]; out: DEVICE [B * n_elev][3][4], caller-owned, not
 * overlapping poses.  n_elev 1..64, pitch finite and >= 0, B >= 0 (0: no-op),
 * else US_ERR_INVALID_ARG; a failed launch gives US_ERR_CUDA. */
US_API us_status us_sim_sweep_poses(const float* poses, int32_t B, int32_t n_elev, float elev_pitch_mm,
                                    float* out, void* stream);

/* Reconstruction observation of the bone-surface task (Sec. 4, Task 2;
 * App. C: 40 x 40 x 40 voxels of 3 mm, 20% missing surface points).
 * Ground-truth surface point: a beam sample s > 0 whose nearest label is
 * bone_label while sample s - 1's is not.  It is kept unless word 0 of
 * Philox-4x32-10 on counter (s, line, env index, 1), key = the render key
 * of (seed, step), is below floor(p_miss 2^32).  The reconstruction of an
 * environment is the set of volume voxels (nearest voxel of a kept point)
 * kept so far, held by the caller as a bitmap over its volume's voxels
 * (us_sim_recon_words() 32-bit words per environment, the largest volume's
 * voxel count / 32 rounded up) plus the list of set voxel indices
 * (capacity `cap` per environment) and its count; zero all three to start.
 * us_sim_recon_update adds one frame per environment (poses device [B][3][4]);
 * a list that reaches its capacity stops growing and is reported by
 * us_sim_check.  us_sim_recon_observe writes obs (device uint8
 * [B][40][40][40], index (h, w, e)): 1 where a reconstructed voxel centre
 * v h, mapped to the probe frame by q = R^T (v h - t) (FP32), has
 * floor(q_x / 3 + 20) = w, floor(q_y / 3 + 20) = e, floor(q_z / 3) = h.
 * Both are asynchronous on `stream`; all buffers are caller-owned device
 * memory.  Errors: US_ERR_INVALID_ARG (NULL buffers, cap < 1, bone label or
 * p_miss out of range, bad ids), US_ERR_CUDA. */
US_API int64_t us_sim_recon_words(const us_sim* sim);
US_API us_status us_sim_recon_update(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                                     uint64_t seed, uint64_t step, int32_t bone_label, float p_miss,
                                     uint32_t* bitmaps, int32_t* points, int32_t* counts, int32_t cap,
                                     void* stream);
US_API us_status us_sim_recon_observe(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                                      const int32_t* points, const int32_t* counts, int32_t cap,
                                      uint8_t* obs, void* stream);

/* The tuned batched render (as us_sim_render, without graph replay) with
 * CUDA events recorded on `stream` around each of its kernels; waits for
 * the render and writes each kernel's duration in ms to kernel_ms[0..n)
 * (host, room for 2): cluster path n = 1 (the persistent kernel), two-pass
 * path with two grids n = 2 (pass A: slice, scanline model, axial PSF; pass
 * B: lateral PSF, log, scan conversion), with one persistent grid n = 1.
 * Errors as us_sim_render. */
US_API us_status us_sim_render_timed(us_sim* sim, const us_env* envs, int32_t B, const float* poses,
                                     uint64_t seed, uint64_t step, float* frames, float* kernel_ms,
                                     int32_t* n_kernels, void* stream);

/* Message of the last error on this handle ("" if none). */
US_API const char* us_sim_last_error(const us_sim* sim);
/* Name of a status code. */
US_API const char* us_status_string(us_status s);

#ifdef __cplusplus
}
#endif

#endif /* USSIM_H */
