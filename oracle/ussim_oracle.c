/*
 * Oracle for the model-based ultrasound render (SonoGym, App. B.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: every table, constant and helper below is written
 * here from the paper's definitions.
 *
 * Plain, slow, literal: one frame at a time, one sample at a time, FP64
 * from the interpolation weights on.  The only FP32 arithmetic is the
 * sample-position / voxel-index path, which is *defined* in FP32 with a
 * fixed, contraction-free operation order so that the nearest-voxel
 * decision is reproducible bit for bit (compile with -ffp-contract=off).
 *
 * Pipeline (Fig. 2 caption and Sec. 4 "Ultrasound simulation"):
 *   probe pose -> image plane -> label/HU slice on the scanline grid ->
 *   image model I = R + B (App. B.2): R = P (x) R_imp (the blurred
 *   reflection impulses), B = E . (P (x) T) (the scatter pattern blurred,
 *   then scaled by the local energy) -> log compression -> scan conversion.
 * The readings taken where the paper is silent are marked READING.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* widest lateral reach of the incidence-angle stencil, in lines */
#define OR_THETA_DMAX 8

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- types */

typedef struct {
  const uint8_t* labels; /* [nz][ny][nx], x fastest */
  const int16_t* hu;     /* same grid */
  int32_t nx, ny, nz;
  float voxel_mm;
  int32_t id;            /* volume index: keys the volume-anchored scatter maps */
} or_volume;

typedef struct {
  float alpha_db_cm_mhz, z_mrayl, mu0, sigma0, mu1;
} or_tissue;

typedef struct {
  int32_t kind; /* 0 linear, 1 curvilinear */
  int32_t n_lines, n_samples;
  float depth_mm, pitch_mm, fan_deg, radius_mm;
  int32_t out_w, out_h;
  float f_mhz, e0, psf_sigma_ax_mm, psf_sigma_lat_mm, dyn_range_db;
} or_probe;

typedef struct {
  int32_t refl_power, transmission, z_mode, speckle;
  int32_t speckle_anchor;   /* 0: maps keyed by (env, line, sample, step); 1: fixed maps over the volume */
  int32_t speckle_levels;   /* anchored maps: number of scales (1..3) */
  float speckle_cell_mm;    /* anchored maps: cell edge of the finest scale */
} or_options;

/* optional per-frame exports; any pointer may be NULL ([NL][NS] unless noted) */
typedef struct {
  double* frame;       /* [out_h][out_w] final image */
  double* envelope;    /* I = P (x) R_imp + E . (P (x) T), before log */
  double* logimg;      /* log-compressed beam image */
  double* S;           /* R_imp + E . T: the image under an identity PSF */
  double* T;           /* scatter pattern T (App. B.2) */
  double* E;           /* remaining energy */
  double* cos_theta;   /* incidence cosine (1 where G = 0) */
  double* hu;          /* interpolated HU */
  int32_t* nn_index;   /* nearest voxel linear index, -1 outside */
  uint8_t* label;      /* nearest label */
  double* n1;          /* anchored scatter maps: the N1 value of each sample */
} or_frame_out;

/* ------------------------------------------------- Philox4x32-10 (SC'11) */
/*
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC 2011): the Philox-4x32 bijection, 10 rounds.  Each round multiplies
 * counter words 0 and 2 by two fixed odd constants (full 64-bit products),
 * then forms the new counter from the high halves XORed with the other two
 * words and the round key, and the low halves.  The two key words are
 * bumped by Weyl constants (golden ratio and sqrt(3)-1, as 32-bit
 * fractions) between rounds.
 */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += OR_PHILOX_W0;
      k1 += OR_PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* READING: the noise maps N0, N1 of App. B.2 are drawn from a counter-based
 * generator keyed by (env, scanline, sample, seed, step) instead of stored
 * 3-D maps.  Counter = (s >> 1, line, env, 0): one call serves the sample
 * pair (2m, 2m+1).  Key = (seed_lo ^ (uint32)(step * 0x9E3779B9), seed_hi). */
void oracle_speckle_words(uint64_t seed, uint64_t step, uint32_t env, uint32_t line,
                          uint32_t sample, uint32_t w[4]) {
  uint32_t ctr[4] = {sample >> 1, line, env, 0u};
  uint32_t key[2];
  key[0] = (uint32_t)seed ^ (uint32_t)(step * 0x9E3779B9ull);
  key[1] = (uint32_t)(seed >> 32);
  oracle_philox4x32_10(ctr, key, w);
}

/* uniform in (0, 1): the top 23 bits as an odd multiple of 2^-24 */
static double or_uniform(uint32_t w) { return (2.0 * (double)(w >> 9) + 1.0) * (1.0 / 16777216.0); }

/* Box-Muller on (u0, u1): even samples take the cosine branch, odd the sine */
double oracle_n0(const uint32_t w[4], uint32_t sample) {
  double u0 = or_uniform(w[0]), u1 = or_uniform(w[1]);
  double rad = sqrt(-2.0 * log(u0));
  return (sample & 1u) ? rad * sin(2.0 * M_PI * u1) : rad * cos(2.0 * M_PI * u1);
}

/* READING: "T = T~ if N1 <= mu1" with N1 standard normal holds with
 * probability Phi(mu1); N1 enters only through that test, so it is drawn as
 * a 32-bit word compared with t1 = floor(Phi(mu1) * 2^32). */
uint64_t oracle_n1_threshold(double mu1) {
  if (isinf(mu1)) return mu1 > 0 ? 4294967296ull : 0ull;
  double phi = 0.5 * erfc(-mu1 / sqrt(2.0));
  double t = floor(phi * 4294967296.0);
  if (t < 0) t = 0;
  if (t > 4294967296.0) t = 4294967296.0;
  return (uint64_t)t;
}

/* ------------------------------------------------------------ geometry */

/* per-probe derived quantities, FP64 */
typedef struct {
  double dr;        /* sample spacing along the beam, mm */
  double dtheta;    /* curvilinear line spacing, rad */
  double dlat_mid;  /* lateral PSF spacing, mm */
  int k_ax, k_lat;  /* PSF half-widths in samples / lines */
} or_derived;

static void or_derive(const or_probe* p, or_derived* d) {
  d->dr = (double)p->depth_mm / (double)p->n_samples;
  d->dtheta = 0.0;
  if (p->kind == 1 && p->n_lines > 1)
    d->dtheta = (double)p->fan_deg * M_PI / 180.0 / (double)(p->n_lines - 1);
  if (p->kind == 1)
    d->dlat_mid = ((double)p->radius_mm + 0.5 * (double)p->depth_mm) * d->dtheta;
  else
    d->dlat_mid = (double)p->pitch_mm;
  d->k_ax = p->psf_sigma_ax_mm > 0 ? (int)ceil(3.0 * (double)p->psf_sigma_ax_mm / d->dr) : 0;
  d->k_lat = (p->psf_sigma_lat_mm > 0 && d->dlat_mid > 0)
                 ? (int)ceil(3.0 * (double)p->psf_sigma_lat_mm / d->dlat_mid) : 0;
}

/* READING (FP32 index path): per-line values computed in FP64, rounded to
 * FP32 once; then, per sample, FP32 products and sums in this order:
 *   linear:      x = x_l,  z = s * dr
 *   curvilinear: rho = r0 + s * dr; x = rho * sin(theta_l); z = rho * cos(theta_l) - r0
 *   p_c = (R_c0 * x + R_c2 * z) + t_c;  u_c = p_c * (1/h)
 * Voxel (i, j, k) is centred at (i, j, k) * h. */
static void or_sample_position(const or_probe* p, const float* M, int l, int s, float pc[3]) {
  float x, z;
  float s_f = (float)s;
  float dr = (float)((double)p->depth_mm / (double)p->n_samples);
  if (p->kind == 0) {
    x = (float)(((double)l - 0.5 * (double)(p->n_lines - 1)) * (double)p->pitch_mm);
    z = s_f * dr;
  } else {
    double dth = p->n_lines > 1 ? (double)p->fan_deg * M_PI / 180.0 / (double)(p->n_lines - 1) : 0.0;
    double th = ((double)l - 0.5 * (double)(p->n_lines - 1)) * dth;
    float sth = (float)sin(th), cth = (float)cos(th);
    float r0 = (float)p->radius_mm;
    float rho = r0 + s_f * dr;
    x = rho * sth;
    float zc = rho * cth;
    z = zc - r0;
  }
  for (int c = 0; c < 3; ++c) {
    float a = M[c * 4 + 0] * x;
    float b = M[c * 4 + 2] * z;
    float q = a + b;
    pc[c] = q + M[c * 4 + 3];
  }
}

static void or_sample_voxel_coords(const or_probe* p, const float* M, float inv_h, int l, int s,
                                   float u[3]) {
  float pc[3];
  or_sample_position(p, M, l, s, pc);
  for (int c = 0; c < 3; ++c) u[c] = pc[c] * inv_h;
}

/* Volume-anchored, multi-scale scatter maps (App. B.2: N0 and N1 are sampled
 * over 3-D space once and stay fixed; multi-scale versions of both are
 * added).  READING: scale k < L is a lattice of cubic cells of edge
 * c 2^k anchored at the volume origin (cell centres at n c 2^k); a sample
 * takes the cell nearest to its volume-frame position, through the same
 * FP32 path as the nearest voxel with 1/(c 2^k) in place of 1/h.  The cell's
 * Philox-4x32-10 words, counter (n_x, n_y, n_z, k << 16 | volume), key =
 * (seed_lo, seed_hi) (no step: the maps are fixed), give two standard
 * normals as the Box-Muller pair of words 0 and 1: Z0 = r cos(theta),
 * Z1 = r sin(theta), r = sqrt(-2 ln u0), theta = 2 pi u1.  N0 = sum_k a_k Z0_k, N1 = sum_k a_k Z1_k, a_k proportional
 * to 2^(-k/2) with sum a_k^2 = 1 (unit variance; coarser scales weigh
 * less).  T = N0 sigma0 + mu0 where N1 <= mu1, else 0. */
static void or_anchored_noise(const float pc[3], const or_options* o, uint32_t vol_id, uint64_t seed,
                              double* n0, double* n1) {
  const int L = o->speckle_levels;
  double norm = 0.0;
  for (int k = 0; k < L; ++k) norm += pow(2.0, -k);
  norm = sqrt(norm);
  const float inv_c0 = (float)(1.0 / (double)o->speckle_cell_mm);
  *n0 = 0.0;
  *n1 = 0.0;
  for (int k = 0; k < L; ++k) {
    const float inv_c = inv_c0 * (float)ldexp(1.0, -k); /* exact: a power of two */
    uint32_t ctr[4], key[2], w[4];
    for (int c = 0; c < 3; ++c) {
      float u = pc[c] * inv_c;
      float f = floorf(u + 0.5f);
      ctr[c] = (uint32_t)(int32_t)f;
    }
    ctr[3] = ((uint32_t)k << 16) | (vol_id & 0xFFFFu);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, w);
    /* the Box-Muller pair of words 0 and 1: r cos(theta), r sin(theta) */
    const double a = pow(2.0, -0.5 * k) / norm;
    const double r = sqrt(-2.0 * log(or_uniform(w[0]))), th = 2.0 * M_PI * or_uniform(w[1]);
    *n0 += a * r * cos(th);
    *n1 += a * r * sin(th);
  }
}

/* exported for the tests: the anchored maps at a volume-frame position */
void oracle_anchored_noise(const float pos[3], int32_t levels, float cell_mm, uint32_t vol_id, uint64_t seed,
                           double out[2]) {
  or_options o = {1, 1, 0, 1, 1, levels, cell_mm};
  or_anchored_noise(pos, &o, vol_id, seed, &out[0], &out[1]);
}

/* nearest voxel: i = floor(u + 0.5) per axis, outside -> -1 */
static int64_t or_nearest(const or_volume* v, const float u[3]) {
  int64_t idx[3];
  const int32_t n[3] = {v->nx, v->ny, v->nz};
  for (int c = 0; c < 3; ++c) {
    float f = floorf(u[c] + 0.5f);
    if (!(f >= 0.0f && f < (float)n[c])) return -1;
    idx[c] = (int64_t)f;
  }
  return (idx[2] * v->ny + idx[1]) * v->nx + idx[0];
}

/* READING: trilinear HU with the fractional offsets t = u - floor(u) (exact
 * in FP32), weights and sum in FP64; voxels outside the grid read HU 0
 * (water).  The paper only says pixels are extracted from the CT volume. */
static double or_trilinear_hu(const or_volume* v, const float u[3]) {
  int64_t i0[3];
  double t[3];
  const int32_t n[3] = {v->nx, v->ny, v->nz};
  for (int c = 0; c < 3; ++c) {
    float f = floorf(u[c]);
    if (!(f >= -1.0f && f < (float)n[c])) return 0.0; /* whole footprint outside */
    i0[c] = (int64_t)f;
    t[c] = (double)(u[c] - f);
  }
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        int64_t i = i0[0] + dx, j = i0[1] + dy, k = i0[2] + dz;
        if (i < 0 || j < 0 || k < 0 || i >= n[0] || j >= n[1] || k >= n[2]) continue;
        double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
        acc += w * (double)v->hu[(k * v->ny + j) * v->nx + i];
      }
  return acc;
}

/* Gaussian PSF taps along one axis: w_k ~ exp(-(k d)^2 / (2 sigma^2)),
 * |k| <= K = ceil(3 sigma / d), normalised to sum 1.  (App. B.2: 2-D
 * Gaussian PSF; READING: separable, sigma in mm on the beam grid.) */
int oracle_psf_taps(double sigma_mm, double spacing_mm, double* taps, int max_taps) {
  int K = sigma_mm > 0 ? (int)ceil(3.0 * sigma_mm / spacing_mm) : 0;
  if (2 * K + 1 > max_taps) return -1;
  double sum = 0.0;
  for (int k = -K; k <= K; ++k) {
    double w = K ? exp(-((double)k * spacing_mm) * ((double)k * spacing_mm) / (2.0 * sigma_mm * sigma_mm)) : 1.0;
    taps[k + K] = w;
    sum += w;
  }
  for (int k = 0; k < 2 * K + 1; ++k) taps[k] /= sum;
  return K;
}

/* ------------------------------------------------------------- render */

static double or_clamp01(double x) { return x < 0 ? 0 : (x > 1 ? 1 : x); }

/* Scan conversion of a curvilinear beam image (READING; the paper's images
 * are linear): output pixel centres on a Cartesian grid in apex coordinates
 * spanning the fan's bounding box; theta = atan2(x, z), rho = hypot(x, z);
 * fractional line / sample indices; outside the fan -> 0; else bilinear. */
void oracle_scan_convert(const or_probe* p, const double* logimg, double* frame) {
  const int NL = p->n_lines, NS = p->n_samples, W = p->out_w, H = p->out_h;
  if (p->kind == 0) {
    for (int s = 0; s < NS; ++s)
      for (int l = 0; l < NL; ++l) frame[(int64_t)s * NL + l] = logimg[(int64_t)l * NS + s];
    return;
  }
  or_derived d;
  or_derive(p, &d);
  double r0 = p->radius_mm, D = p->depth_mm;
  double half = 0.5 * (double)p->fan_deg * M_PI / 180.0;
  double xmax = (r0 + D) * sin(half), xmin = -xmax;
  double zmin = r0 * cos(half), zmax = r0 + D;
  for (int r = 0; r < H; ++r) {
    for (int c = 0; c < W; ++c) {
      double x = xmin + (c + 0.5) * (xmax - xmin) / W;
      double z = zmin + (r + 0.5) * (zmax - zmin) / H;
      double th = atan2(x, z), rho = hypot(x, z);
      double fl = th / d.dtheta + 0.5 * (NL - 1);
      double fs = (rho - r0) / d.dr;
      double v = 0.0;
      if (fl >= 0 && fl <= NL - 1 && fs >= 0 && fs <= NS - 1) {
        int l0 = (int)floor(fl), s0 = (int)floor(fs);
        if (l0 > NL - 2) l0 = NL - 2;
        if (s0 > NS - 2) s0 = NS - 2;
        if (l0 < 0) l0 = 0;
        if (s0 < 0) s0 = 0;
        double a = fl - l0, b = fs - s0;
        int l1 = NL > 1 ? l0 + 1 : l0, s1 = NS > 1 ? s0 + 1 : s0;
        v = (1 - a) * (1 - b) * logimg[(int64_t)l0 * NS + s0] + a * (1 - b) * logimg[(int64_t)l1 * NS + s0] +
            (1 - a) * b * logimg[(int64_t)l0 * NS + s1] + a * b * logimg[(int64_t)l1 * NS + s1];
      }
      frame[(int64_t)r * W + c] = v;
    }
  }
}

/* Render one frame.  Returns 0 on success, -1 on bad arguments, -2 on a
 * label outside the tissue table, -3 on allocation failure. */
int oracle_render_frame(const or_volume* vol, const or_tissue* table, int n_labels, const or_probe* p,
                        const or_options* opt, const float* pose, uint32_t env, uint64_t seed,
                        uint64_t step, or_frame_out* out) {
  const int NL = p->n_lines, NS = p->n_samples;
  if (NL < 1 || NS < 2 || n_labels < 1) return -1;
  or_derived d;
  or_derive(p, &d);
  const int64_t N = (int64_t)NL * NS;
  uint8_t* lab = (uint8_t*)malloc(N);
  double* hu = (double*)malloc(N * sizeof(double));
  double* S = (double*)malloc(N * sizeof(double));
  double* Rm = (double*)malloc(N * sizeof(double));
  double* Tm = (double*)malloc(N * sizeof(double));
  double* Em = (double*)malloc(N * sizeof(double));
  double* tmpR = (double*)malloc(N * sizeof(double));
  double* tmpT = (double*)malloc(N * sizeof(double));
  double* I = (double*)malloc(N * sizeof(double));
  double* Y = (double*)malloc(N * sizeof(double));
  double* wax = (double*)malloc((2 * d.k_ax + 1) * sizeof(double));
  double* wlat = (double*)malloc((2 * d.k_lat + 1) * sizeof(double));
  int rc = 0;
  if (!lab || !hu || !S || !Rm || !Tm || !Em || !tmpR || !tmpT || !I || !Y || !wax || !wlat) { rc = -3; goto done; }

  const float inv_h = (float)(1.0 / (double)vol->voxel_mm);

  /* 1. image plane -> label (nearest) and HU (trilinear) slices */
  for (int l = 0; l < NL; ++l) {
    for (int s = 0; s < NS; ++s) {
      float u[3];
      or_sample_voxel_coords(p, pose, inv_h, l, s, u);
      int64_t idx = or_nearest(vol, u);
      uint8_t lb = idx >= 0 ? vol->labels[idx] : 0;
      if (lb >= n_labels) { rc = -2; goto done; }
      lab[(int64_t)l * NS + s] = lb;
      hu[(int64_t)l * NS + s] = or_trilinear_hu(vol, u);
      if (out && out->nn_index) out->nn_index[(int64_t)l * NS + s] = (int32_t)idx;
      if (out && out->label) out->label[(int64_t)l * NS + s] = lb;
      if (out && out->hu) out->hu[(int64_t)l * NS + s] = hu[(int64_t)l * NS + s];
    }
  }

  /* 2. per-line image model along the beam (+y of the image) */
  for (int l = 0; l < NL; ++l) {
    const uint8_t* L = lab + (int64_t)l * NS;
    double Lsum = 0.0; /* exclusive running sum of the log-energy increments */
    for (int s = 0; s < NS; ++s) {
      const or_tissue* ti = &table[L[s]];
      /* impedance: READING z_mode 0 -> Z = max(HU + 1024, 1) ("proportional to
       * CT intensity", after Kutter et al.); z_mode 1 -> tissue table */
      double Zs, Zn, r = 0.0;
      int G = 0;
      double cth = 1.0;
      if (s < NS - 1) {
        if (opt->z_mode == 0) {
          Zs = fmax(hu[(int64_t)l * NS + s] + 1024.0, 1.0);
          Zn = fmax(hu[(int64_t)l * NS + s + 1] + 1024.0, 1.0);
        } else {
          Zs = table[L[s]].z_mrayl;
          Zn = table[L[s + 1]].z_mrayl;
        }
        r = (Zn - Zs) / (Zn + Zs);
        G = L[s + 1] != L[s];
        if (G) {
          /* READING: incidence angle from the label slice.  m = [label ==
           * L(l, s+1)] (the tissue below the interface); M(l') = sum of m over
           * the axial window s-W+1 .. s+W on line l' (samples clamped), which
           * moves by one per sample of interface shift; tan(theta) = |M(l+D) -
           * M(l-D)| dr / (line distance * dlat).  The window spans two voxels
           * axially (W = ceil(2h/dr)) and one voxel laterally on either side
           * (D = ceil(h/dlat)), so the voxel staircase of the label map is
           * averaged over, capped at D <= OR_THETA_DMAX lines. */
          uint8_t below = L[s + 1];
          double dlat = p->kind == 0 ? (double)p->pitch_mm
                                     : ((double)p->radius_mm + s * d.dr) * d.dtheta;
          int W = (int)ceil(2.0 * (double)vol->voxel_mm / d.dr);
          int D = dlat > 0 ? (int)ceil((double)vol->voxel_mm / dlat) : 1;
          if (D > OR_THETA_DMAX) D = OR_THETA_DMAX;
          if (D < 1) D = 1;
          int lp = l + D < NL - 1 ? l + D : NL - 1;
          int lm = l - D > 0 ? l - D : 0;
          int Mp = 0, Mm = 0;
          for (int q = s - W + 1; q <= s + W; ++q) {
            int qc = q < 0 ? 0 : (q > NS - 1 ? NS - 1 : q);
            Mp += lab[(int64_t)lp * NS + qc] == below;
            Mm += lab[(int64_t)lm * NS + qc] == below;
          }
          double tanth = lp > lm ? fabs((double)(Mp - Mm)) * d.dr / ((double)(lp - lm) * dlat) : 0.0;
          cth = 1.0 / sqrt(1.0 + tanth * tanth);
        }
      }
      /* energy reaching sample s: E0 * exp(sum over v < s of the increments) */
      double E = (double)p->e0 * exp(Lsum);
      double alpha_np = (double)ti->alpha_db_cm_mhz * log(10.0) / 20.0 / 10.0; /* Np/(mm MHz) */
      double inc = -(double)p->f_mhz * alpha_np * d.dr;
      if (opt->transmission && G) inc += log(fmax(1.0 - r * r, 1e-30));
      Lsum += inc;

      /* reflection impulse G * E * |cos(theta) r|^p.  p = 1 is the paper's
       * |E cos(theta) r| (E >= 0); READING p = 2: the intensity reflection
       * coefficient (cos(theta) r)^2, still linear in the incident energy. */
      double Rimp = 0.0;
      if (G) {
        double a = fabs(cth * r);
        Rimp = E * (opt->refl_power == 2 ? a * a : a);
      }
      /* scatter pattern T (App. B.2: T~ = N0 sigma0 + mu0 where N1 <= mu1, else 0) */
      double T;
      if (opt->speckle && opt->speckle_anchor) {
        float pc[3];
        double n0, n1;
        or_sample_position(p, pose, l, s, pc);
        or_anchored_noise(pc, opt, (uint32_t)vol->id, seed, &n0, &n1);
        T = n1 <= (double)ti->mu1 ? n0 * (double)ti->sigma0 + (double)ti->mu0 : 0.0;
        if (out && out->n1) out->n1[(int64_t)l * NS + s] = n1;
      } else if (opt->speckle) {
        uint32_t w[4];
        oracle_speckle_words(seed, step, env, (uint32_t)l, (uint32_t)s, w);
        double n0 = oracle_n0(w, (uint32_t)s);
        uint64_t t1 = oracle_n1_threshold((double)ti->mu1);
        int pass = (uint64_t)w[2 + (s & 1)] < t1;
        T = pass ? n0 * (double)ti->sigma0 + (double)ti->mu0 : 0.0;
      } else {
        T = (double)ti->mu0;
      }
      Rm[(int64_t)l * NS + s] = Rimp;
      Tm[(int64_t)l * NS + s] = T;
      Em[(int64_t)l * NS + s] = E;
      S[(int64_t)l * NS + s] = Rimp + E * T;
      if (out && out->E) out->E[(int64_t)l * NS + s] = E;
      if (out && out->cos_theta) out->cos_theta[(int64_t)l * NS + s] = cth;
    }
  }

  /* 3. PSF: separable Gaussian on the beam grid, zero padded, applied to
   * the reflection impulses and to the scatter pattern separately.
   * Reflection (READING): R = P (x) R_imp, the impulses G |E cos r|^p
   * blurred, so a one-sample interface spreads over the PSF (the printed
   * |E cos r| . P (x) G would leave it one sample thick wherever r is zero
   * off the boundary).  Backscatter, as printed in App. B.2:
   * B(u) = E(u) . (P (x) T)(u): the scatter pattern is blurred first, then
   * scaled by the energy at u itself.  I = R + B. */
  oracle_psf_taps(p->psf_sigma_ax_mm, d.dr, wax, 2 * d.k_ax + 1);
  oracle_psf_taps(p->psf_sigma_lat_mm, d.dlat_mid, wlat, 2 * d.k_lat + 1);
  for (int l = 0; l < NL; ++l)
    for (int s = 0; s < NS; ++s) {
      double accR = 0.0, accT = 0.0;
      for (int k = -d.k_ax; k <= d.k_ax; ++k) {
        int ss = s + k;
        if (ss < 0 || ss >= NS) continue;
        accR += wax[k + d.k_ax] * Rm[(int64_t)l * NS + ss];
        accT += wax[k + d.k_ax] * Tm[(int64_t)l * NS + ss];
      }
      tmpR[(int64_t)l * NS + s] = accR;
      tmpT[(int64_t)l * NS + s] = accT;
    }
  for (int l = 0; l < NL; ++l)
    for (int s = 0; s < NS; ++s) {
      double accR = 0.0, accT = 0.0;
      for (int j = -d.k_lat; j <= d.k_lat; ++j) {
        int ll = l + j;
        if (ll < 0 || ll >= NL) continue;
        accR += wlat[j + d.k_lat] * tmpR[(int64_t)ll * NS + s];
        accT += wlat[j + d.k_lat] * tmpT[(int64_t)ll * NS + s];
      }
      I[(int64_t)l * NS + s] = accR + Em[(int64_t)l * NS + s] * accT;
    }

  /* 4. log compression, READING: 20 log10(I / E0) over a dynamic range DR
   * mapped to [0, 1]; non-positive I floors at 1e-30 */
  for (int64_t i = 0; i < N; ++i) {
    double db = 20.0 * log10(fmax(I[i], 1e-30) / (double)p->e0);
    Y[i] = or_clamp01((db + (double)p->dyn_range_db) / (double)p->dyn_range_db);
  }

  if (out) {
    if (out->S) memcpy(out->S, S, N * sizeof(double));
    if (out->T) memcpy(out->T, Tm, N * sizeof(double));
    if (out->envelope) memcpy(out->envelope, I, N * sizeof(double));
    if (out->logimg) memcpy(out->logimg, Y, N * sizeof(double));
    if (out->frame) oracle_scan_convert(p, Y, out->frame);
  }
done:
  free(lab); free(hu); free(S); free(Rm); free(Tm); free(Em); free(tmpR); free(tmpT); free(I); free(Y);
  free(wax); free(wlat);
  return rc;
}

/* Batch render with one OpenMP thread per frame (the CPU baseline).
 * envs: int32 [B][2] = (volume_id, probe_id); poses float32 [B][12];
 * frames: double, frame b at offsets[b] (elements).  Returns 0 or the first
 * nonzero frame status. */
int oracle_render_batch(const or_volume* vols, int n_vols, const or_tissue* table, int n_labels,
                        const or_probe* probes, int n_probes, const or_options* opt,
                        const int32_t* envs, int B, const float* poses, uint64_t seed, uint64_t step,
                        double* frames, const int64_t* offsets, int n_threads) {
  int status = 0;
  (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int b = 0; b < B; ++b) {
    int v = envs[2 * b], pi = envs[2 * b + 1];
    int rc;
    if (v < 0 || v >= n_vols || pi < 0 || pi >= n_probes) {
      rc = -1;
    } else {
      or_frame_out o;
      memset(&o, 0, sizeof o);
      o.frame = frames + offsets[b];
      rc = oracle_render_frame(&vols[v], table, n_labels, &probes[pi], opt, poses + 12 * b,
                               (uint32_t)b, seed, step, &o);
    }
    if (rc) {
#pragma omp critical
      if (!status) status = rc;
    }
  }
  return status;
}

/* Unique voxels read by a batch: the nearest voxel and the in-grid trilinear
 * corners of every sample.  per_frame[b] gets the count of frame b; the
 * return value is the count over the union of all frames (per volume,
 * summed).  This defines the algorithmic voxel bytes (label 1 B + HU 2 B). */
int64_t oracle_touched_voxels(const or_volume* vols, int n_vols, const or_probe* probes,
                              const int32_t* envs, int B, const float* poses, int64_t* per_frame) {
  int64_t total = 0;
  for (int v = 0; v < n_vols; ++v) {
    int64_t nvox = (int64_t)vols[v].nx * vols[v].ny * vols[v].nz;
    uint8_t* uni = (uint8_t*)calloc((size_t)nvox, 1);
    uint8_t* fr = (uint8_t*)calloc((size_t)nvox, 1);
    if (!uni || !fr) { free(uni); free(fr); return -1; }
    const float inv_h = (float)(1.0 / (double)vols[v].voxel_mm);
    const int32_t n[3] = {vols[v].nx, vols[v].ny, vols[v].nz};
    for (int b = 0; b < B; ++b) {
      if (envs[2 * b] != v) continue;
      const or_probe* p = &probes[envs[2 * b + 1]];
      int64_t cnt = 0;
      memset(fr, 0, (size_t)nvox);
      for (int l = 0; l < p->n_lines; ++l)
        for (int s = 0; s < p->n_samples; ++s) {
          float u[3];
          or_sample_voxel_coords(p, poses + 12 * b, inv_h, l, s, u);
          int64_t idx = or_nearest(&vols[v], u);
          if (idx >= 0 && !fr[idx]) { fr[idx] = 1; ++cnt; }
          if (idx >= 0 && !uni[idx]) { uni[idx] = 1; ++total; }
          int64_t i0[3];
          int ok = 1;
          for (int c = 0; c < 3; ++c) {
            float f = floorf(u[c]);
            if (!(f >= -1.0f && f < (float)n[c])) ok = 0;
            else i0[c] = (int64_t)f;
          }
          if (!ok) continue;
          for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
              for (int dx = 0; dx < 2; ++dx) {
                int64_t i = i0[0] + dx, j = i0[1] + dy, k = i0[2] + dz;
                if (i < 0 || j < 0 || k < 0 || i >= n[0] || j >= n[1] || k >= n[2]) continue;
                int64_t q = (k * n[1] + j) * n[0] + i;
                if (!fr[q]) { fr[q] = 1; ++cnt; }
                if (!uni[q]) { uni[q] = 1; ++total; }
              }
        }
      if (per_frame) per_frame[b] = cnt;
    }
    free(uni);
    free(fr);
  }
  return total;
}

/* the FP32 voxel coordinates of one sample (exported for the index tests) */
void oracle_sample_coords(const or_probe* p, const float* pose, float voxel_mm, int line, int sample,
                          float u[3]) {
  or_sample_voxel_coords(p, pose, (float)(1.0 / (double)voxel_mm), line, sample, u);
}


/* Surrogate input on the output pixel grid (the learned simulator maps the
 * CT / label slice to the image, Sec. 4; App. B.2): per output pixel, the
 * nearest label / 4, clamp(trilinear HU / 1000, -1, 3), and an inside-fan
 * flag.  Curvilinear: pixel centres of the scan-conversion grid, in the
 * probe frame (apex coordinates shifted by -r0), computed in FP64 and
 * rounded to FP32 once; linear: the beam grid (row = sample, column =
 * line).  The voxel coordinate then follows the same FP32 path as the
 * beam samples.  out: [out_h][out_w][3]. */
/* raw = 0: out[H][W][3] = (label / 4, clamp(HU / 1000, -1, 3), mask);
 * raw = 1: out[H][W][3] = (label, HU, mask) (HU unscaled, unclamped) */
static int sample_slice(const or_volume* vol, const or_probe* p, const float* pose, double* out, int raw) {
  const int W = p->out_w, H = p->out_h, NL = p->n_lines, NS = p->n_samples;
  const float inv_h = (float)(1.0 / (double)vol->voxel_mm);
  or_derived d;
  or_derive(p, &d);
  for (int r = 0; r < H; ++r) {
    for (int c = 0; c < W; ++c) {
      float x, z;
      double mask = 1.0;
      if (p->kind == 0) {
        x = (float)(((double)c - 0.5 * (double)(NL - 1)) * (double)p->pitch_mm);
        z = (float)r * (float)((double)p->depth_mm / (double)NS);
      } else {
        double r0 = p->radius_mm, D = p->depth_mm;
        double half = 0.5 * (double)p->fan_deg * M_PI / 180.0;
        double xmax = (r0 + D) * sin(half), xmin = -xmax;
        double zmin = r0 * cos(half), zmax = r0 + D;
        double xa = xmin + (c + 0.5) * (xmax - xmin) / W;
        double za = zmin + (r + 0.5) * (zmax - zmin) / H;
        double fl = atan2(xa, za) / d.dtheta + 0.5 * (NL - 1);
        double fs = (hypot(xa, za) - r0) / d.dr;
        mask = (fl >= 0 && fl <= NL - 1 && fs >= 0 && fs <= NS - 1) ? 1.0 : 0.0;
        x = (float)xa;
        z = (float)(za - r0);
      }
      float u[3];
      for (int k = 0; k < 3; ++k) {
        float a = pose[k * 4 + 0] * x;
        float b = pose[k * 4 + 2] * z;
        float q = a + b;
        float pc = q + pose[k * 4 + 3];
        u[k] = pc * inv_h;
      }
      int64_t idx = or_nearest(vol, u);
      double lab = idx >= 0 ? (double)vol->labels[idx] : 0.0;
      double hu = or_trilinear_hu(vol, u);
      double* o = out + ((int64_t)r * W + c) * 3;
      if (raw) {
        o[0] = lab;
        o[1] = hu;
      } else {
        hu /= 1000.0;
        if (hu < -1.0) hu = -1.0;
        if (hu > 3.0) hu = 3.0;
        o[0] = lab / 4.0;
        o[1] = hu;
      }
      o[2] = mask;
    }
  }
  return 0;
}

int oracle_sample_slice(const or_volume* vol, const or_probe* p, const float* pose, double* out) {
  return sample_slice(vol, p, pose, out, 0);
}

int oracle_sample_slice_raw(const or_volume* vol, const or_probe* p, const float* pose, double* out) {
  return sample_slice(vol, p, pose, out, 1);
}

/* Surrogate input on a common H x W grid over a probe's output field (the
 * learned simulator of App. B.2 run at one size for every probe).  READING:
 * pixel centres of an H x W grid spanning the field, in FP64, rounded once
 * to FP32: curvilinear, the fan's bounding box in apex coordinates (as the
 * scan conversion, at H x W), shifted by -r0 into the probe frame, flag =
 * inside the fan; linear, x = ((c + 1/2) NL / W - 1/2 - (NL - 1) / 2) pitch,
 * z = ((r + 1/2) NS / H - 1/2) dr, flag 1.  The voxel coordinate then
 * follows the render's FP32 path.  out: [H][W][3] = (label / 4,
 * clamp(HU / 1000, -1, 3), flag). */
int oracle_sample_slice_grid(const or_volume* vol, const or_probe* p, const float* pose, int H, int W, double* out) {
  const int NL = p->n_lines, NS = p->n_samples;
  const float inv_h = (float)(1.0 / (double)vol->voxel_mm);
  or_derived d;
  or_derive(p, &d);
  for (int r = 0; r < H; ++r) {
    for (int c = 0; c < W; ++c) {
      float x, z;
      double flag = 1.0;
      if (p->kind == 0) {
        x = (float)(((c + 0.5) * NL / W - 0.5 - 0.5 * (NL - 1)) * (double)p->pitch_mm);
        z = (float)(((r + 0.5) * NS / H - 0.5) * d.dr);
      } else {
        double r0 = p->radius_mm, D = p->depth_mm;
        double half = 0.5 * (double)p->fan_deg * M_PI / 180.0;
        double xmax = (r0 + D) * sin(half), xmin = -xmax;
        double zmin = r0 * cos(half), zmax = r0 + D;
        double xa = xmin + (c + 0.5) * (xmax - xmin) / W;
        double za = zmin + (r + 0.5) * (zmax - zmin) / H;
        double fl = atan2(xa, za) / d.dtheta + 0.5 * (NL - 1);
        double fs = (hypot(xa, za) - r0) / d.dr;
        flag = (fl >= 0 && fl <= NL - 1 && fs >= 0 && fs <= NS - 1) ? 1.0 : 0.0;
        x = (float)xa;
        z = (float)(za - r0);
      }
      float u[3];
      for (int k = 0; k < 3; ++k) {
        float a = pose[k * 4 + 0] * x;
        float b = pose[k * 4 + 2] * z;
        float q = a + b;
        float pc = q + pose[k * 4 + 3];
        u[k] = pc * inv_h;
      }
      int64_t idx = or_nearest(vol, u);
      double hu = or_trilinear_hu(vol, u) / 1000.0;
      if (hu < -1.0) hu = -1.0;
      if (hu > 3.0) hu = 3.0;
      double* o = out + ((int64_t)r * W + c) * 3;
      o[0] = (idx >= 0 ? (double)vol->labels[idx] : 0.0) / 4.0;
      o[1] = hu;
      o[2] = flag;
    }
  }
  return 0;
}

/* ------------------------------------------- reconstruction observation */
/*
 * Task 2 of Sec. 4 with App. C: the bone surface segmented from each frame
 * (simulated from the ground truth with a missing probability per point)
 * updates a 3-D reconstruction with the probe's pose; the observation is
 * that reconstruction transformed to the current probe frame and voxelized
 * to H x W x E = 40 x 40 x 40 voxels of 3 mm.
 * READING: a ground-truth surface point is a beam sample s whose nearest
 * label is the bone label while sample s-1's is not (the boundary G of
 * App. B.2 with bone below); it is kept unless its Philox-4x32-10 word 0,
 * counter (s, line, env, 1), key = the render key of (seed, step), falls
 * below floor(p_miss 2^32).  The reconstruction is the set of volume voxels
 * (the point's nearest voxel) ever kept.  Observation voxel (h, w, e) holds
 * 1 iff some reconstructed voxel centre v h, mapped to the probe frame by
 * q = R^T (v h - t) (FP32: differences, then per column the three products
 * summed in row order), has floor(q_x / 3 + 20) = w, floor(q_y / 3 + 20) = e,
 * floor(q_z / 3) = h.
 */
uint32_t oracle_recon_keep_threshold(double p_miss) {
  double t = floor(p_miss * 4294967296.0);
  if (t < 0) t = 0;
  if (t > 4294967295.0) t = 4294967295.0;
  return (uint32_t)t;
}

/* add this frame's kept surface points to `recon` (one byte per voxel of the
 * volume); returns the number of ground-truth points, *kept those kept */
int64_t oracle_recon_update(const or_volume* vol, const or_probe* p, const float* pose, uint32_t env, uint64_t seed,
                            uint64_t step, int32_t bone_label, double p_miss, uint8_t* recon, int64_t* kept) {
  const int NL = p->n_lines, NS = p->n_samples;
  const float inv_h = (float)(1.0 / (double)vol->voxel_mm);
  const uint32_t thr = oracle_recon_keep_threshold(p_miss);
  uint32_t key[2];
  key[0] = (uint32_t)seed ^ (uint32_t)(step * 0x9E3779B9ull);
  key[1] = (uint32_t)(seed >> 32);
  int64_t n = 0, k = 0;
  for (int l = 0; l < NL; ++l) {
    int prev_lab = -1;
    for (int s = 0; s < NS; ++s) {
      float u[3];
      or_sample_voxel_coords(p, pose, inv_h, l, s, u);
      int64_t idx = or_nearest(vol, u);
      int lab = idx >= 0 ? vol->labels[idx] : 0;
      if (s > 0 && lab == bone_label && prev_lab != bone_label) {
        ++n;
        uint32_t ctr[4] = {(uint32_t)s, (uint32_t)l, env, 1u}, w[4];
        oracle_philox4x32_10(ctr, key, w);
        if (w[0] >= thr) {
          recon[idx] = 1;
          ++k;
        }
      }
      prev_lab = lab;
    }
  }
  if (kept) *kept = k;
  return n;
}

/* voxelize the reconstruction in the probe frame of `pose`: obs [40][40][40]
 * (h, w, e), 1 where a reconstructed voxel lands */
void oracle_recon_observe(const or_volume* vol, const uint8_t* recon, const float* pose, uint8_t* obs) {
  memset(obs, 0, 40 * 40 * 40);
  const float h = vol->voxel_mm, third = (float)(1.0 / 3.0);
  for (int64_t kz = 0; kz < vol->nz; ++kz)
    for (int64_t jy = 0; jy < vol->ny; ++jy)
      for (int64_t ix = 0; ix < vol->nx; ++ix) {
        if (!recon[(kz * vol->ny + jy) * vol->nx + ix]) continue;
        float d[3];
        d[0] = (float)ix * h - pose[3];
        d[1] = (float)jy * h - pose[7];
        d[2] = (float)kz * h - pose[11];
        float q[3];
        for (int c = 0; c < 3; ++c) {
          float a = pose[0 * 4 + c] * d[0];
          float b = pose[1 * 4 + c] * d[1];
          float e = pose[2 * 4 + c] * d[2];
          float ab = a + b;
          q[c] = ab + e;
        }
        float fw = floorf(q[0] * third + 20.0f), fe = floorf(q[1] * third + 20.0f), fh = floorf(q[2] * third);
        if (fw >= 0 && fw < 40 && fe >= 0 && fe < 40 && fh >= 0 && fh < 40)
          obs[((int)fh * 40 + (int)fw) * 40 + (int)fe] = 1;
      }
}
