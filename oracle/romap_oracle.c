/*
 * romap_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU implementation of the per-object NeRF
 * training step of RO-MAP (Han, Liu, Ding, Yang, "RO-MAP: Real-Time
 * Multi-Object Mapping with Neural Radiance Fields", RA-L 2023), written from
 * the paper's Sec. V (Eq. 6-11) and the hash encoding it cites (Mueller et
 * al., "Instant Neural Graphics Primitives", 2022).  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this library; the
 * product path (the CUDA library) never does, and the two share no code.
 *
 * Precision.  Everything is FP64 except the sampler stage (world->object
 * transform, slab test, stratified sample positions, occupancy cell and hash
 * corner selection), which is written in FP32 with one fixed operation order
 * and no fused multiply-add (compiled with -ffp-contract=off), so that sample
 * positions and hash indices are reproducible bit for bit by an independent
 * FP32 implementation.  The FP32 outputs of that stage are promoted to FP64
 * before the encoding's interpolation weights are formed.
 *
 * Readings of the paper where it is silent (numbered R-1 .. R-16; each one is
 * cited where it is used):
 *  R-1  Random numbers: Philox4x32-10 (Salmon et al., SC'11).  key = (seed
 *       low 32 bits, seed high 32 bits); counter = (a, b, purpose, c) as
 *       documented per use below.  u01(x) = (x >> 8) * 2^-24.
 *  R-2  Slab test (Sec. V-B "intersects with the 3D bounding box"): IEEE
 *       1/d, fminf/fmaxf (NaN-ignoring), t_near = max(t0, 0), hit iff
 *       t_far > t_near.
 *  R-3  Stratified samples: t_i = t_near + (i + u_i) * (t_far - t_near)/N,
 *       delta_i = t_{i+1} - t_i, delta_{N-1} = t_far - t_{N-1}, x = o + t d.
 *  R-4  Level resolutions: N_l = floor(N_min * b^l + 1e-6) in FP64.
 *  R-5  Corner selection, dense/hashed index (Mueller et al. Sec. 3).
 *  R-6  Trilinear weights, level-major feature order, U(-1e-4,1e-4) init.
 *  R-7  Object frame: x_o = R_z(yaw)^T (x_w - t), d_o normalised.
 *  R-8  Occupancy culling: culled sample has sigma := 0, keeps its delta.
 *  R-9  Losses (Eq. 7-11): squared L2 over RGB, all terms divided by the
 *       batch size B; every ray composites over its own background colour.
 *  R-10 Compositing adjoint by explicit suffix sums.
 *  R-11 MLP: density (L*F)->H->16 ReLU; colour (15 + dir)->H->H->3, ReLU,
 *       sigmoid; no biases.
 *  R-11' The paper's model (Sec. V: hash encoding and a single-layer MLP,
 *       positions only): (L*F)->H->16 with sigma from output 0 and the
 *       colour sigmoid(outputs 1..3); the colour-net layers are unused.
 *  R-13 sigma = exp(clamp(o_0, -15, 15)); zero gradient outside the clamp.
 *  R-14 Adam (Kingma & Ba) with bias correction, step counter from 1.
 *  R-17 Occupancy update (not in the paper): density at the 64^3 cell
 *       centres, d = max(decay d, sigma), bit = d > threshold.
 *  R-19 Mesh extraction (Table 3, 64^3 marching cubes): 64^3 cubes over the
 *       object box, densities at the 65^3 lattice vertices, one vertex per
 *       lattice edge crossing the iso-level, linear interpolation.
 *  R-18 Data-update rule (Eq. 5): the angle between the object-to-camera
 *       vectors of the last used and the current image; update when it
 *       exceeds the threshold, and always for the first image.
 * Storage (not the method): each level's entries start at a multiple of 8.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_MAX_LEVELS 32
#define OC_MAX_LF 64
#define OC_MAX_H 128

/* Philox purposes (counter word 2), reading R-1. */
#define OC_PURPOSE_RAY 1u
#define OC_PURPOSE_BG 2u
#define OC_PURPOSE_JITTER 3u
#define OC_PURPOSE_INIT_HASH 4u
#define OC_PURPOSE_INIT_MLP 5u

/* Ray classes (Sec. V-B): object rays R_o, background rays R_b, occluders. */
#define OC_CLS_OBJECT 0
#define OC_CLS_BACKGROUND 1
#define OC_CLS_OCCLUDER 2

typedef struct oc_config {
  int32_t L;              /* levels */
  int32_t F;              /* features per level */
  uint32_t T;             /* max entries per level (hash table size) */
  int32_t res[OC_MAX_LEVELS]; /* N_l, from oc_level_resolutions */
  int32_t n_samples;      /* N samples per ray (Sec. V-B) */
  int32_t rays_per_step;  /* rays drawn per step */
  int32_t hidden;         /* MLP width (64 in the paper) */
  int32_t geo;            /* geometry features passed to the colour net (15) */
  int32_t dir_dims;       /* 0 or 3 view-direction inputs */
  int32_t bg_random;      /* 1: per-ray random background each step (Eq. 9) */
  double bg_const[3];     /* background when bg_random == 0 */
  double lambda1, lambda2;/* Eq. 11 */
  double lr, beta1, beta2, eps; /* Adam */
  int32_t single_net;     /* 1: the paper's model (R-11'): colour logits = density-net outputs 1..3 */
  int32_t hidden_layers;  /* single-network model: hidden layers of width H (1..3, Table 4); 0 reads as 1 */
} oc_config;

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror, Shaw,   */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.      */
/* ------------------------------------------------------------------ */
void oc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0; k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t philox_word(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                            const uint32_t key[2], int word) {
  uint32_t ctr[4] = {c0, c1, c2, c3}, out[4];
  oc_philox4x32_10(ctr, key, out);
  return out[word];
}

/* u01 in [0, 1): 24 random bits scaled by 2^-24 (exact in FP32). */
float oc_u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

/* ------------------------------------------------------------------ */
/* Grid layout (R-4, R-5).                                             */
/* ------------------------------------------------------------------ */
int oc_level_resolutions(int32_t L, double n_min, double growth, double n_max, int32_t* res) {
  if (L < 1 || L > OC_MAX_LEVELS) return -1;
  double b = growth;
  if (!(b > 0.0)) b = (L > 1) ? exp((log(n_max) - log(n_min)) / (double)(L - 1)) : 1.0;
  for (int l = 0; l < L; ++l) res[l] = (int32_t)floor(n_min * pow(b, (double)l) + 1e-6);
  return 0;
}

static uint64_t level_dense_count(const oc_config* c, int l) {
  uint64_t n = (uint64_t)c->res[l] + 1u;
  return n * n * n;
}
int oc_level_is_dense(const oc_config* c, int l) { return level_dense_count(c, l) <= (uint64_t)c->T; }
uint64_t oc_level_size(const oc_config* c, int l) {
  return oc_level_is_dense(c, l) ? level_dense_count(c, l) : (uint64_t)c->T;
}
/* Storage layout (not part of the method): each level's entries start at a multiple of 8 entries, so a level of
 * (N+1)^3 dense entries is followed by up to 7 unused entries. */
uint64_t oc_level_offset(const oc_config* c, int l) {
  uint64_t off = 0;
  for (int i = 0; i < l; ++i) off += (oc_level_size(c, i) + 7u) / 8u * 8u;
  return off;
}
uint64_t oc_hash_param_count(const oc_config* c) {
  return oc_level_offset(c, c->L) * (uint64_t)c->F;
}
/* MLP layers (R-11), row-major [out][in]:
 *   0: density 1  H x (L*F)      1: density 2  (1+geo) x H
 *   2: colour 1   H x (geo+dir)  3: colour 2   H x H        4: colour 3  3 x H
 * and, for the single-network model with K > 1 hidden layers (Table 4), K - 1 more H x H layers 5, 6 between
 * the first hidden layer and layer 1 (the colour-net layers 2..4 stay in the layout, unused). */
int oc_extra_layers(const oc_config* c) {
  return (c->single_net && c->hidden_layers > 1) ? c->hidden_layers - 1 : 0;
}
static void mlp_shape(const oc_config* c, int layer, int* out, int* in) {
  int H = c->hidden, LF = c->L * c->F;
  switch (layer) {
    case 0: *out = H; *in = LF; break;
    case 1: *out = 1 + c->geo; *in = H; break;
    case 2: *out = H; *in = c->geo + c->dir_dims; break;
    case 4: *out = 3; *in = H; break;
    default: *out = H; *in = H; break;  /* 3, 5, 6 */
  }
}
uint64_t oc_mlp_layer_offset(const oc_config* c, int layer) {
  uint64_t off = 0;
  for (int i = 0; i < layer; ++i) { int o, n; mlp_shape(c, i, &o, &n); off += (uint64_t)o * n; }
  return off;
}
uint64_t oc_mlp_param_count(const oc_config* c) { return oc_mlp_layer_offset(c, 5 + oc_extra_layers(c)); }
uint64_t oc_param_count(const oc_config* c) { return oc_hash_param_count(c) + oc_mlp_param_count(c); }

/* Index of grid vertex (cx, cy, cz) on level l (R-5). */
uint32_t oc_grid_index(const oc_config* c, int l, uint32_t cx, uint32_t cy, uint32_t cz) {
  if (oc_level_is_dense(c, l)) {
    uint32_t n = (uint32_t)c->res[l] + 1u;
    return cx + cy * n + cz * n * n;
  }
  uint32_t h = (cx * 1u) ^ (cy * 2654435761u) ^ (cz * 805459861u);
  return h % c->T;
}

/* ------------------------------------------------------------------ */
/* Parameter initialisation (R-6, R-13), FP32 formula then promoted.  */
/* ------------------------------------------------------------------ */
void oc_init_params(const oc_config* c, uint64_t seed, double* params) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint64_t nh = oc_hash_param_count(c);
  for (uint64_t k = 0; k < nh; ++k) {
    uint32_t x = philox_word((uint32_t)(k >> 2), 0u, OC_PURPOSE_INIT_HASH, 0u, key, (int)(k & 3u));
    float u = oc_u01(x);
    float v = (2.0f * u - 1.0f) * 1e-4f;
    params[k] = (double)v;
  }
  for (int layer = 0; layer < 5 + oc_extra_layers(c); ++layer) {
    int o, n;
    mlp_shape(c, layer, &o, &n);
    float limit = (float)sqrt(6.0 / (double)(o + n)); /* Glorot-uniform */
    double* w = params + nh + oc_mlp_layer_offset(c, layer);
    for (uint64_t k = 0; k < (uint64_t)o * n; ++k) {
      uint32_t x = philox_word((uint32_t)(k >> 2), (uint32_t)layer, OC_PURPOSE_INIT_MLP, 0u, key, (int)(k & 3u));
      float u = oc_u01(x);
      float v = (2.0f * u - 1.0f) * limit;
      w[k] = (double)v;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Sampler stage, FP32 (R-2, R-3, R-7, R-8).                           */
/* ------------------------------------------------------------------ */
/* World -> object frame: the object pose is a translation t and a yaw about
 * world z (Sec. IV-B, Eq. 1); rays are generated in the object frame
 * (Sec. V-B).  cos/sin are evaluated in FP64 and rounded to FP32 once. */
void oc_world_to_object(int64_t n, const float* o_w, const float* d_w, const float t[3],
                        double yaw, float* o_o, float* d_o) {
  float cz = (float)cos(yaw), sz = (float)sin(yaw);
  for (int64_t r = 0; r < n; ++r) {
    float px = o_w[3 * r + 0] - t[0];
    float py = o_w[3 * r + 1] - t[1];
    float pz = o_w[3 * r + 2] - t[2];
    o_o[3 * r + 0] = cz * px + sz * py;
    o_o[3 * r + 1] = cz * py - sz * px;
    o_o[3 * r + 2] = pz;
    float dx = d_w[3 * r + 0], dy = d_w[3 * r + 1], dz = d_w[3 * r + 2];
    float rx = cz * dx + sz * dy;
    float ry = cz * dy - sz * dx;
    float rz = dz;
    float len = sqrtf(rx * rx + ry * ry + rz * rz);
    d_o[3 * r + 0] = rx / len;
    d_o[3 * r + 1] = ry / len;
    d_o[3 * r + 2] = rz / len;
  }
}

/* Slab intersection with [-half, half]^3.  Returns 1 on hit. */
int oc_ray_aabb(const float o[3], const float d[3], const float half[3], float* t_near, float* t_far) {
  float t0 = -INFINITY, t1 = INFINITY;
  for (int a = 0; a < 3; ++a) {
    float lo = -half[a], hi = half[a];
    float inv = 1.0f / d[a];
    float ta = (lo - o[a]) * inv;
    float tb = (hi - o[a]) * inv;
    float mn = fminf(ta, tb), mx = fmaxf(ta, tb);
    t0 = (a == 0) ? mn : fmaxf(t0, mn);
    t1 = (a == 0) ? mx : fminf(t1, mx);
  }
  float tn = fmaxf(t0, 0.0f);
  *t_near = tn;
  *t_far = t1;
  return t1 > tn;
}

/* Occupancy cell of an object-frame point: 64^3 bits, x fastest (R-8). */
int oc_occupied(const uint64_t* bits, const float x[3], const float half[3]) {
  if (!bits) return 1;
  int cell[3];
  for (int a = 0; a < 3; ++a) {
    float lo = -half[a];
    float inv_ext = 1.0f / (half[a] - lo);
    float u = fminf(fmaxf((x[a] - lo) * inv_ext, 0.0f), 1.0f);
    int ci = (int)(u * 64.0f);
    cell[a] = ci > 63 ? 63 : ci;
  }
  uint32_t bit = (uint32_t)cell[0] + 64u * (uint32_t)cell[1] + 4096u * (uint32_t)cell[2];
  return (int)((bits[bit >> 6] >> (bit & 63u)) & 1u);
}

/* Samples of one ray.  jitter: 1 -> u_i from Philox (counter (step, slot,
 * JITTER, i>>2), word i&3); 0 -> midpoints u_i = 0.5.  Writes N entries of
 * t, delta, x (object frame) and live (hit and occupied).  Returns hit. */
int oc_sample_ray(const float o[3], const float d[3], const float half[3], int N, const uint32_t key[2],
                  uint32_t step, uint32_t slot, int jitter, const uint64_t* occ, float* t, float* delta,
                  float* x, uint8_t* live, float* t_near_out, float* t_far_out) {
  float tn, tf;
  int hit = oc_ray_aabb(o, d, half, &tn, &tf);
  if (t_near_out) *t_near_out = tn;
  if (t_far_out) *t_far_out = tf;
  if (!hit) {
    for (int i = 0; i < N; ++i) { t[i] = 0.0f; delta[i] = 0.0f; x[3 * i] = x[3 * i + 1] = x[3 * i + 2] = 0.0f; live[i] = 0; }
    return 0;
  }
  float step_len = (tf - tn) / (float)N;
  for (int i = 0; i < N; ++i) {
    float u = 0.5f;
    if (jitter) u = oc_u01(philox_word(step, slot, OC_PURPOSE_JITTER, (uint32_t)i >> 2, key, i & 3));
    t[i] = tn + ((float)i + u) * step_len;
  }
  for (int i = 0; i < N; ++i) delta[i] = (i + 1 < N) ? (t[i + 1] - t[i]) : (tf - t[i]);
  for (int i = 0; i < N; ++i) {
    for (int a = 0; a < 3; ++a) x[3 * i + a] = o[a] + t[i] * d[a];
    live[i] = (uint8_t)oc_occupied(occ, x + 3 * i, half);
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* Multiresolution hash encoding (R-5, R-6).                           */
/* ------------------------------------------------------------------ */
/* Corner c (bit 0: x, bit 1: y, bit 2: z) of level l for point x.  The
 * fractional position is computed in FP32 and returned promoted. */
void oc_level_corners(const oc_config* c, int l, const float x[3], const float half[3],
                      uint32_t idx[8], double w[8]) {
  int i0[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    float lo = -half[a];
    float inv_ext = 1.0f / (half[a] - lo);
    float u = fminf(fmaxf((x[a] - lo) * inv_ext, 0.0f), 1.0f);
    float pos = u * (float)c->res[l];
    int i = (int)floorf(pos);
    if (i > c->res[l] - 1) i = c->res[l] - 1;
    float fr = pos - (float)i;
    i0[a] = i;
    f[a] = (double)fr;
  }
  for (int corner = 0; corner < 8; ++corner) {
    uint32_t cx = (uint32_t)(i0[0] + (corner & 1));
    uint32_t cy = (uint32_t)(i0[1] + ((corner >> 1) & 1));
    uint32_t cz = (uint32_t)(i0[2] + ((corner >> 2) & 1));
    idx[corner] = oc_grid_index(c, l, cx, cy, cz);
    double wx = (corner & 1) ? f[0] : 1.0 - f[0];
    double wy = ((corner >> 1) & 1) ? f[1] : 1.0 - f[1];
    double wz = ((corner >> 2) & 1) ? f[2] : 1.0 - f[2];
    w[corner] = wx * wy * wz;
  }
}

/* enc[l*F + k] = sum_corner w * table[(offset_l + idx) * F + k] */
void oc_encode(const oc_config* c, const double* table, const float x[3], const float half[3], double* enc) {
  for (int l = 0; l < c->L; ++l) {
    uint32_t idx[8];
    double w[8];
    oc_level_corners(c, l, x, half, idx, w);
    uint64_t off = oc_level_offset(c, l);
    for (int k = 0; k < c->F; ++k) {
      double s = 0.0;
      for (int corner = 0; corner < 8; ++corner) s += w[corner] * table[(off + idx[corner]) * c->F + k];
      enc[l * c->F + k] = s;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Tiny MLP (R-11, R-13).                                              */
/* ------------------------------------------------------------------ */
typedef struct oc_act {
  double enc[OC_MAX_LF];
  double h1[OC_MAX_H];        /* after ReLU */
  double hx[2][OC_MAX_H];     /* single-network model: hidden layers 2 and 3, after ReLU */
  double out[1 + 31];         /* density net outputs (linear) */
  double cin[31 + 3];         /* colour net input */
  double h2[OC_MAX_H], h3[OC_MAX_H];
  double logit[3];
  double rgb[3];
  double sigma;
} oc_act;

static double relu(double v) { return v > 0.0 ? v : 0.0; }

/* y = W x for W row-major [o][n]. */
static void matvec(const double* W, int o, int n, const double* x, double* y) {
  for (int i = 0; i < o; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += W[(size_t)i * n + j] * x[j];
    y[i] = s;
  }
}

void oc_mlp_forward(const oc_config* c, const double* mlp, const double* enc, const float dir[3], oc_act* a) {
  int H = c->hidden, LF = c->L * c->F, G = c->geo, D = c->dir_dims;
  const double* W0 = mlp + oc_mlp_layer_offset(c, 0);
  const double* W1 = mlp + oc_mlp_layer_offset(c, 1);
  const double* W2 = mlp + oc_mlp_layer_offset(c, 2);
  const double* W3 = mlp + oc_mlp_layer_offset(c, 3);
  const double* W4 = mlp + oc_mlp_layer_offset(c, 4);
  for (int j = 0; j < LF; ++j) a->enc[j] = enc[j];
  matvec(W0, H, LF, a->enc, a->h1);
  for (int i = 0; i < H; ++i) a->h1[i] = relu(a->h1[i]);
  const double* last = a->h1;  /* the hidden layer that feeds layer 1 */
  for (int j = 0; j < oc_extra_layers(c); ++j) {
    matvec(mlp + oc_mlp_layer_offset(c, 5 + j), H, H, last, a->hx[j]);
    for (int i = 0; i < H; ++i) a->hx[j][i] = relu(a->hx[j][i]);
    last = a->hx[j];
  }
  matvec(W1, 1 + G, H, last, a->out);
  double o0 = a->out[0];
  if (o0 < -15.0) o0 = -15.0;
  if (o0 > 15.0) o0 = 15.0;
  a->sigma = exp(o0);
  if (c->single_net) {
    for (int j = 0; j < G + D; ++j) a->cin[j] = 0.0;
    for (int i = 0; i < H; ++i) a->h2[i] = a->h3[i] = 0.0;
    for (int k = 0; k < 3; ++k) {
      a->logit[k] = a->out[1 + k];
      a->rgb[k] = 1.0 / (1.0 + exp(-a->logit[k]));
    }
    return;
  }
  for (int j = 0; j < G; ++j) a->cin[j] = a->out[1 + j];
  for (int j = 0; j < D; ++j) a->cin[G + j] = (double)dir[j];
  matvec(W2, H, G + D, a->cin, a->h2);
  for (int i = 0; i < H; ++i) a->h2[i] = relu(a->h2[i]);
  matvec(W3, H, H, a->h2, a->h3);
  for (int i = 0; i < H; ++i) a->h3[i] = relu(a->h3[i]);
  matvec(W4, 3, H, a->h3, a->logit);
  for (int k = 0; k < 3; ++k) a->rgb[k] = 1.0 / (1.0 + exp(-a->logit[k]));
}

/* Backward of one sample: given dL/dsigma and dL/drgb, accumulate dL/dW into
 * gmlp and return dL/denc in genc.  Plain chain rule, layer by layer. */
void oc_mlp_backward(const oc_config* c, const double* mlp, const oc_act* a, double gsigma, const double grgb[3],
                     double* gmlp, double* genc) {
  int H = c->hidden, LF = c->L * c->F, G = c->geo, D = c->dir_dims;
  const double* W[5];
  double* gW[5];
  for (int l = 0; l < 5; ++l) { W[l] = mlp + oc_mlp_layer_offset(c, l); gW[l] = gmlp + oc_mlp_layer_offset(c, l); }
  const int X = oc_extra_layers(c);
  double glogit[3], gh3[OC_MAX_H], gh2[OC_MAX_H], gcin[34], gout[32], gh1[OC_MAX_H], gx[OC_MAX_H];
  for (int k = 0; k < 3; ++k) glogit[k] = grgb[k] * a->rgb[k] * (1.0 - a->rgb[k]);
  if (c->single_net) {  /* the colour logits are density-net outputs 1..3 */
    for (int j = 0; j < G; ++j) gcin[j] = j < 3 ? glogit[j] : 0.0;
    goto density_outputs;
  }
  /* layer 4: logit = W4 h3 */
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < H; ++j) gW[4][k * H + j] += glogit[k] * a->h3[j];
  for (int j = 0; j < H; ++j) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += W[4][k * H + j] * glogit[k];
    gh3[j] = a->h3[j] > 0.0 ? s : 0.0;
  }
  /* layer 3: h3 = relu(W3 h2) */
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < H; ++j) gW[3][i * H + j] += gh3[i] * a->h2[j];
  for (int j = 0; j < H; ++j) {
    double s = 0.0;
    for (int i = 0; i < H; ++i) s += W[3][i * H + j] * gh3[i];
    gh2[j] = a->h2[j] > 0.0 ? s : 0.0;
  }
  /* layer 2: h2 = relu(W2 cin) */
  int CI = G + D;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < CI; ++j) gW[2][i * CI + j] += gh2[i] * a->cin[j];
  for (int j = 0; j < CI; ++j) {
    double s = 0.0;
    for (int i = 0; i < H; ++i) s += W[2][i * CI + j] * gh2[i];
    gcin[j] = s;
  }
  /* density outputs: out0 -> sigma through exp(clamp); out1.. -> cin */
density_outputs:;
  double o0 = a->out[0];
  gout[0] = (o0 >= -15.0 && o0 <= 15.0) ? gsigma * a->sigma : 0.0;
  for (int j = 0; j < G; ++j) gout[1 + j] = gcin[j];
  /* layer 1: out = W1 h, h the last hidden layer (h1 unless the single network has more) */
  const double* last = X > 0 ? a->hx[X - 1] : a->h1;
  for (int i = 0; i < 1 + G; ++i)
    for (int j = 0; j < H; ++j) gW[1][i * H + j] += gout[i] * last[j];
  for (int j = 0; j < H; ++j) {
    double s = 0.0;
    for (int i = 0; i < 1 + G; ++i) s += W[1][i * H + j] * gout[i];
    gh1[j] = last[j] > 0.0 ? s : 0.0;
  }
  /* single-network hidden layers 5 + k, from the last: hx[k] = relu(M hprev), gh1 holding dL/d hx[k] */
  for (int k = X - 1; k >= 0; --k) {
    const double* M = mlp + oc_mlp_layer_offset(c, 5 + k);
    double* gM = gmlp + oc_mlp_layer_offset(c, 5 + k);
    const double* prev = k > 0 ? a->hx[k - 1] : a->h1;
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < H; ++j) gM[i * H + j] += gh1[i] * prev[j];
    for (int j = 0; j < H; ++j) {
      double s = 0.0;
      for (int i = 0; i < H; ++i) s += M[i * H + j] * gh1[i];
      gx[j] = prev[j] > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < H; ++j) gh1[j] = gx[j];
  }
  /* layer 0: h1 = relu(W0 enc) */
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < LF; ++j) gW[0][i * LF + j] += gh1[i] * a->enc[j];
  for (int j = 0; j < LF; ++j) {
    double s = 0.0;
    for (int i = 0; i < H; ++i) s += W[0][i * LF + j] * gh1[i];
    genc[j] = s;
  }
}

/* Scatter dL/denc into the table gradient with the trilinear weights. */
void oc_encode_backward(const oc_config* c, const float x[3], const float half[3], const double* genc, double* gtable) {
  for (int l = 0; l < c->L; ++l) {
    uint32_t idx[8];
    double w[8];
    oc_level_corners(c, l, x, half, idx, w);
    uint64_t off = oc_level_offset(c, l);
    for (int corner = 0; corner < 8; ++corner)
      for (int k = 0; k < c->F; ++k) gtable[(off + idx[corner]) * c->F + k] += w[corner] * genc[l * c->F + k];
  }
}

/* ------------------------------------------------------------------ */
/* Volume rendering, Sec. V-B (Eq. 6) with the background reading R-9.  */
/* ------------------------------------------------------------------ */
/* out[0..2] = C_hat, out[3] = D_hat, out[4] = opacity A = 1 - T_{N+1}.
 * o_i = 1 - exp(-sigma_i delta_i), w_i = o_i prod_{j<i}(1 - o_j) with the
 * product evaluated as exp(-sum_{j<i} sigma_j delta_j). */
void oc_composite(int n, const double* sigma, const double* delta, const double* t, const double* rgb,
                  const double bg[3], double out[5], double* w_out) {
  double acc = 0.0, C[3] = {0, 0, 0}, Dh = 0.0;
  for (int i = 0; i < n; ++i) {
    double Ti = exp(-acc);
    double oi = 1.0 - exp(-sigma[i] * delta[i]);
    double wi = Ti * oi;
    if (w_out) w_out[i] = wi;
    for (int k = 0; k < 3; ++k) C[k] += wi * rgb[3 * i + k];
    Dh += wi * t[i];
    acc += sigma[i] * delta[i];
  }
  double Tend = exp(-acc);
  for (int k = 0; k < 3; ++k) out[k] = C[k] + Tend * bg[k];
  out[3] = Dh;
  out[4] = 1.0 - Tend;
}

/* Adjoint of oc_composite (R-10): given gC = dL/dC_hat, gD = dL/dD_hat and
 * gA = dL/dA, write dL/dsigma_i (without any direct term) and dL/drgb_i.
 *   dC/dsigma_i = delta_i [T_{i+1} c_i - sum_{j>i} w_j c_j - T_{N+1} bg]
 *   dD/dsigma_i = delta_i [T_{i+1} t_i - sum_{j>i} w_j t_j]
 *   dA/dsigma_i = delta_i T_{N+1},   dC/dc_i = w_i                      */
void oc_composite_backward(int n, const double* sigma, const double* delta, const double* t, const double* rgb,
                           const double bg[3], const double gC[3], double gD, double gA, double* gsigma,
                           double* grgb) {
  double* Tnext = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    double Ti = exp(-acc);
    w[i] = Ti * (1.0 - exp(-sigma[i] * delta[i]));
    acc += sigma[i] * delta[i];
    Tnext[i] = exp(-acc);
  }
  double Tend = exp(-acc);
  double SC[3] = {0, 0, 0}, SD = 0.0; /* suffix sums over j > i */
  for (int i = n - 1; i >= 0; --i) {
    double g = 0.0;
    for (int k = 0; k < 3; ++k) g += gC[k] * (Tnext[i] * rgb[3 * i + k] - SC[k] - Tend * bg[k]);
    g += gD * (Tnext[i] * t[i] - SD);
    g += gA * Tend;
    gsigma[i] = delta[i] * g;
    for (int k = 0; k < 3; ++k) grgb[3 * i + k] = gC[k] * w[i];
    for (int k = 0; k < 3; ++k) SC[k] += w[i] * rgb[3 * i + k];
    SD += w[i] * t[i];
  }
  free(Tnext);
  free(w);
}

/* ------------------------------------------------------------------ */
/* Per-ray loss, Eq. 7-11 with reading R-9.                            */
/* ------------------------------------------------------------------ */
/* Returns the ray's contribution to B*L and the gradient scalars of B*L.
 * comps[0..3] accumulate the rgb, rr, depth and density terms (unweighted
 * by lambda).  sigma_sum is sum_i sigma_i over live samples. */
double oc_ray_loss(int cls, const double Chat[3], double Dhat, const float target_rgb[3], float target_depth,
                   const double bg[3], double sigma_sum, double lambda1, double lambda2, double gC[3], double* gD,
                   double* gsig_direct, double comps[4]) {
  double loss = 0.0;
  gC[0] = gC[1] = gC[2] = 0.0;
  *gD = 0.0;
  *gsig_direct = 0.0;
  if (cls == OC_CLS_OCCLUDER) return 0.0;
  const double* tgt = bg;
  double trgb[3] = {target_rgb[0], target_rgb[1], target_rgb[2]};
  if (cls == OC_CLS_OBJECT) tgt = trgb;
  double sq = 0.0;
  for (int k = 0; k < 3; ++k) {
    double e = Chat[k] - tgt[k];
    sq += e * e;
    gC[k] = 2.0 * e;
  }
  loss += sq;
  if (cls == OC_CLS_OBJECT) comps[0] += sq; else comps[1] += sq;
  if (isfinite(target_depth)) {
    double e = Dhat - (double)target_depth;
    loss += lambda1 * fabs(e);
    comps[2] += fabs(e);
    *gD = lambda1 * (e > 0.0 ? 1.0 : (e < 0.0 ? -1.0 : 0.0));
  }
  if (cls == OC_CLS_BACKGROUND) {
    loss += lambda2 * sigma_sum; /* |sigma_j - 0| = sigma_j since sigma > 0 */
    comps[3] += sigma_sum;
    *gsig_direct = lambda2;
  }
  return loss;
}

/* ------------------------------------------------------------------ */
/* Adam (R-14).                                                        */
/* ------------------------------------------------------------------ */
void oc_adam(int64_t n, double* p, double* m, double* v, const double* g, int64_t step, double lr, double beta1,
             double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------ */
/* Ray batch draw (R-1).                                               */
/* ------------------------------------------------------------------ */
/* Batch size B = min(rays_per_step, n_pool).  If rays_per_step >= n_pool the
 * whole pool is used in order; otherwise slot s draws pool index
 * mulhi32(x, n_pool) with x = Philox((step, s, RAY, 0))[0], with replacement.
 * Background of slot s: u01 of words 0..2 of Philox((step, s, BG, 0)) when
 * bg_random, else cfg->bg_const. */
int64_t oc_draw_batch(const oc_config* c, uint64_t seed, uint32_t step, int64_t n_pool, int64_t* pool_idx, double* bg) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t B = (c->rays_per_step >= n_pool) ? n_pool : c->rays_per_step;
  for (int64_t s = 0; s < B; ++s) {
    if (c->rays_per_step >= n_pool) {
      pool_idx[s] = s;
    } else {
      uint32_t x = philox_word(step, (uint32_t)s, OC_PURPOSE_RAY, 0u, key, 0);
      pool_idx[s] = (int64_t)(((uint64_t)x * (uint64_t)n_pool) >> 32);
    }
    if (c->bg_random) {
      uint32_t ctr[4] = {step, (uint32_t)s, OC_PURPOSE_BG, 0u}, out[4];
      oc_philox4x32_10(ctr, key, out);
      for (int k = 0; k < 3; ++k) bg[3 * s + k] = (double)oc_u01(out[k]);
    } else {
      for (int k = 0; k < 3; ++k) bg[3 * s + k] = c->bg_const[k];
    }
  }
  return B;
}

/* ------------------------------------------------------------------ */
/* Forward + loss + backward over explicit rays (no Adam).             */
/* ------------------------------------------------------------------ */
/* Rays are given in the object frame (o, d normalised).  For each ray r the
 * RNG slot is slot0 + r.  ray_out (nullable) receives per ray
 * [C_hat(3), D_hat, A, sigma_sum, loss_r, hit].  sample_out (nullable)
 * receives per sample [t, delta, x(3), live, sigma, dL/dsigma].  grad
 * (nullable) is accumulated (not zeroed).  Upstream ray gradients: when
 * upstream != NULL the Eq. 7-11 loss is replaced by sum_r <upstream_r,
 * (C_hat, D_hat, A, sigma_sum)> (used to test the differentiable render
 * independently of the loss).  Returns B*L summed over rays (or the
 * upstream-weighted sum).  comps (nullable, 4 doubles) accumulate loss
 * components.  inv_B scales every gradient (1/B for the training loss). */
double oc_rays_loss_grad(const oc_config* c, const double* params, const float half[3], uint64_t seed, uint32_t step,
                         int64_t slot0, int jitter, const uint64_t* occ, int64_t n, const float* o, const float* d,
                         const float* rgb, const float* depth, const uint8_t* cls, const double* bg,
                         const double* upstream, double inv_B, double* grad, double* ray_out, double* sample_out,
                         double* comps) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int N = c->n_samples;
  const double* table = params;
  const double* mlp = params + oc_hash_param_count(c);
  double* gtable = grad;
  double* gmlp = grad ? grad + oc_hash_param_count(c) : NULL;
  float* t = (float*)malloc(sizeof(float) * N);
  float* dl = (float*)malloc(sizeof(float) * N);
  float* x = (float*)malloc(sizeof(float) * 3 * N);
  uint8_t* live = (uint8_t*)malloc((size_t)N);
  double* sig = (double*)malloc(sizeof(double) * N);
  double* dd = (double*)malloc(sizeof(double) * N);
  double* td = (double*)malloc(sizeof(double) * N);
  double* col = (double*)malloc(sizeof(double) * 3 * N);
  double* gsig = (double*)malloc(sizeof(double) * N);
  double* gcol = (double*)malloc(sizeof(double) * 3 * N);
  oc_act* act = (oc_act*)malloc(sizeof(oc_act) * (size_t)N);
  double total = 0.0;
  double local_comps[4] = {0, 0, 0, 0};
  for (int64_t r = 0; r < n; ++r) {
    const float* orr = o + 3 * r;
    const float* drr = d + 3 * r;
    int hit = oc_sample_ray(orr, drr, half, N, key, step, (uint32_t)(slot0 + r), jitter, occ, t, dl, x, live, NULL, NULL);
    double sigma_sum = 0.0;
    for (int i = 0; i < N; ++i) {
      dd[i] = (double)dl[i];
      td[i] = (double)t[i];
      sig[i] = 0.0;
      col[3 * i] = col[3 * i + 1] = col[3 * i + 2] = 0.0;
      if (hit && live[i]) {
        double enc[OC_MAX_LF];
        oc_encode(c, table, x + 3 * i, half, enc);
        oc_mlp_forward(c, mlp, enc, drr, &act[i]);
        sig[i] = act[i].sigma;
        for (int k = 0; k < 3; ++k) col[3 * i + k] = act[i].rgb[k];
        sigma_sum += sig[i];
      }
    }
    int ns = hit ? N : 0;
    double out[5];
    oc_composite(ns, sig, dd, td, col, bg + 3 * r, out, NULL);
    double gC[3], gD, gA = 0.0, gdir, lr_;
    if (upstream) {
      const double* u = upstream + 6 * r;
      gC[0] = u[0]; gC[1] = u[1]; gC[2] = u[2]; gD = u[3]; gA = u[4]; gdir = u[5];
      lr_ = u[0] * out[0] + u[1] * out[1] + u[2] * out[2] + u[3] * out[3] + u[4] * out[4] + u[5] * sigma_sum;
    } else {
      lr_ = oc_ray_loss(cls[r], out, out[3], rgb + 3 * r, depth[r], bg + 3 * r, sigma_sum, c->lambda1, c->lambda2,
                        gC, &gD, &gdir, local_comps);
    }
    total += lr_;
    if (ray_out) {
      double* ro = ray_out + 8 * r;
      for (int k = 0; k < 5; ++k) ro[k] = out[k];
      ro[5] = sigma_sum;
      ro[6] = lr_;
      ro[7] = hit;
    }
    for (int k = 0; k < 3; ++k) gC[k] *= inv_B;
    gD *= inv_B; gA *= inv_B; gdir *= inv_B;
    oc_composite_backward(ns, sig, dd, td, col, bg + 3 * r, gC, gD, gA, gsig, gcol);
    for (int i = 0; i < N; ++i) {
      int is_live = hit && live[i];
      double gs = is_live ? gsig[i] + gdir : 0.0;
      if (sample_out) {
        double* so = sample_out + 8 * ((size_t)r * N + i);
        so[0] = t[i]; so[1] = dl[i]; so[2] = x[3 * i]; so[3] = x[3 * i + 1]; so[4] = x[3 * i + 2];
        so[5] = is_live; so[6] = sig[i]; so[7] = gs;
      }
      if (is_live && grad) {
        double genc[OC_MAX_LF];
        oc_mlp_backward(c, mlp, &act[i], gs, gcol + 3 * i, gmlp, genc);
        oc_encode_backward(c, x + 3 * i, half, genc, gtable);
      }
    }
  }
  if (comps) for (int k = 0; k < 4; ++k) comps[k] += local_comps[k];
  free(t); free(dl); free(x); free(live); free(sig); free(dd); free(td); free(col); free(gsig); free(gcol); free(act);
  return total;
}

/* ------------------------------------------------------------------ */
/* One training step of one object (Sec. V-A/V-B, Eq. 11, Adam).        */
/* ------------------------------------------------------------------ */
/* Pool rays are in the object frame.  params, m, v are updated in place
 * when do_adam; grad_out (nullable, n_params) receives dL/dparams.  loss_out
 * (5 doubles): L, then the rgb, rr, depth and density sums divided by B.
 * pool_idx_out (B), bg_out (3B), ray_out (8B), sample_out (8BN) nullable.
 * Returns B. */
int64_t oc_train_step(const oc_config* c, const float half[3], uint64_t seed, uint32_t step, const uint64_t* occ,
                      int64_t n_pool, const float* o, const float* d, const float* rgb, const float* depth,
                      const uint8_t* cls, double* params, double* m, double* v, int do_adam, double* grad_out,
                      double* loss_out, int64_t* pool_idx_out, double* bg_out, double* ray_out, double* sample_out) {
  int64_t cap = (c->rays_per_step >= n_pool) ? n_pool : c->rays_per_step;
  if (cap <= 0) return 0;
  int64_t* pidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  double* bg = (double*)malloc(sizeof(double) * 3 * (size_t)cap);
  int64_t B = oc_draw_batch(c, seed, step, n_pool, pidx, bg);
  float* bo = (float*)malloc(sizeof(float) * 3 * (size_t)B);
  float* bd = (float*)malloc(sizeof(float) * 3 * (size_t)B);
  float* brgb = (float*)malloc(sizeof(float) * 3 * (size_t)B);
  float* bdep = (float*)malloc(sizeof(float) * (size_t)B);
  uint8_t* bcls = (uint8_t*)malloc((size_t)B);
  for (int64_t s = 0; s < B; ++s) {
    int64_t p = pidx[s];
    for (int k = 0; k < 3; ++k) { bo[3 * s + k] = o[3 * p + k]; bd[3 * s + k] = d[3 * p + k]; brgb[3 * s + k] = rgb[3 * p + k]; }
    bdep[s] = depth[p];
    bcls[s] = cls[p];
  }
  uint64_t P = oc_param_count(c);
  double* g = (double*)calloc((size_t)P, sizeof(double));
  double comps[4] = {0, 0, 0, 0};
  double invB = 1.0 / (double)B;
  double total = oc_rays_loss_grad(c, params, half, seed, step, 0, 1, occ, B, bo, bd, brgb, bdep, bcls, bg, NULL, invB,
                                   g, ray_out, sample_out, comps);
  if (loss_out) {
    loss_out[0] = total * invB;
    for (int k = 0; k < 4; ++k) loss_out[1 + k] = comps[k] * invB;
  }
  if (grad_out) memcpy(grad_out, g, sizeof(double) * (size_t)P);
  if (do_adam) oc_adam((int64_t)P, params, m, v, g, (int64_t)step, c->lr, c->beta1, c->beta2, c->eps);
  if (pool_idx_out) memcpy(pool_idx_out, pidx, sizeof(int64_t) * (size_t)B);
  if (bg_out) memcpy(bg_out, bg, sizeof(double) * 3 * (size_t)B);
  free(pidx); free(bg); free(bo); free(bd); free(brgb); free(bdep); free(bcls); free(g);
  return B;
}

/* ------------------------------------------------------------------ */
/* Occupancy grid from the learned density.  Not in the paper (which   */
/* samples the whole box); the build's scope table defines it as an    */
/* exponential moving maximum of the density at the 64^3 cell centres, */
/* thresholded into the bitgrid that culls samples (R-8).              */
/* ------------------------------------------------------------------ */
/* Centre of cell (ix, iy, iz) of the object box, FP32 in a fixed order:
 * x_a = -a + (i + 0.5) * ((a - (-a)) / 64). */
void oc_cell_centre(const float half[3], int ix, int iy, int iz, float x[3]) {
  const int idx[3] = {ix, iy, iz};
  for (int a = 0; a < 3; ++a) {
    float lo = -half[a];
    float w = (half[a] - lo) / 64.0f;
    x[a] = lo + ((float)idx[a] + 0.5f) * w;
  }
}

/* sigma = exp(clamp(o_0, -15, 15)) of the density net (R-11, R-13) at one
 * object-frame point: encoding, first layer with ReLU (then the single
 * network's further hidden layers), output 0 of layer 1. */
double oc_density(const oc_config* c, const double* params, const float x[3], const float half[3]) {
  double enc[OC_MAX_LF], h[OC_MAX_H], hn[OC_MAX_H];
  int H = c->hidden, LF = c->L * c->F;
  const double* mlp = params + oc_hash_param_count(c);
  const double* W0 = mlp + oc_mlp_layer_offset(c, 0);
  const double* W1 = mlp + oc_mlp_layer_offset(c, 1);
  oc_encode(c, params, x, half, enc);
  for (int i = 0; i < H; ++i) {
    double s = 0.0;
    for (int j = 0; j < LF; ++j) s += W0[(size_t)i * LF + j] * enc[j];
    h[i] = relu(s);
  }
  for (int k = 0; k < oc_extra_layers(c); ++k) {
    matvec(mlp + oc_mlp_layer_offset(c, 5 + k), H, H, h, hn);
    for (int i = 0; i < H; ++i) h[i] = relu(hn[i]);
  }
  double o0 = 0.0;
  for (int i = 0; i < H; ++i) o0 += W1[i] * h[i];
  if (o0 < -15.0) o0 = -15.0;
  if (o0 > 15.0) o0 = 15.0;
  return exp(o0);
}

/* sigma at all 64^3 cell centres; cell index x + 64 y + 4096 z. */
void oc_density_grid(const oc_config* c, const double* params, const float half[3], double* sigma) {
  for (int z = 0; z < 64; ++z)
    for (int y = 0; y < 64; ++y)
      for (int x = 0; x < 64; ++x) {
        float p[3];
        oc_cell_centre(half, x, y, z, p);
        sigma[x + 64 * y + 4096 * z] = oc_density(c, params, p, half);
      }
}

/* One update of n cells: density = max(decay * density, sigma); bit i of
 * bits (word i / 64, bit i % 64) = density_i > threshold. */
void oc_occupancy_update(int64_t n, const double* sigma, double decay, double threshold, double* density,
                         uint64_t* bits) {
  memset(bits, 0, sizeof(uint64_t) * (size_t)((n + 63) / 64));
  for (int64_t i = 0; i < n; ++i) {
    double d = decay * density[i];
    if (sigma[i] > d) d = sigma[i];
    density[i] = d;
    if (d > threshold) bits[i >> 6] |= (uint64_t)1 << (i & 63);
  }
}

/* ------------------------------------------------------------------ */
/* Incremental training-data rule (Sec. V-A-1, Eq. 5).                 */
/* ------------------------------------------------------------------ */
/* Rotation angle, in degrees, between the last updated image I_m and the
 * current image I_n as seen from the object: the angle between the vectors
 * from the object centre t_O to the two camera centres (FP64).  The cosine
 * is clamped to [-1, 1] against rounding.  Degenerate vectors (a camera at
 * the object centre) give 180 degrees, i.e. always update. */
double oc_view_angle_deg(const double t_m[3], const double t_n[3], const double t_o[3]) {
  double a[3], b[3], ab = 0.0, aa = 0.0, bb = 0.0;
  for (int k = 0; k < 3; ++k) {
    a[k] = t_m[k] - t_o[k];
    b[k] = t_n[k] - t_o[k];
    ab += a[k] * b[k];
    aa += a[k] * a[k];
    bb += b[k] * b[k];
  }
  if (aa == 0.0 || bb == 0.0) return 180.0;
  double c = ab / (sqrt(aa) * sqrt(bb));
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  return acos(c) * (180.0 / 3.14159265358979323846);
}

/* The rule: update when no image has been used yet, or when the angle is
 * larger than the threshold (Sec. VI: 25 degrees). */
int oc_should_update(int have_last, const double t_m[3], const double t_n[3], const double t_o[3],
                     double threshold_deg) {
  if (!have_last) return 1;
  return oc_view_angle_deg(t_m, t_n, t_o) > threshold_deg;
}

/* ------------------------------------------------------------------ */
/* Mesh extraction (Table 3: marching cubes, 64^3).  The oracle        */
/* computes what any correct triangulation shares: the lattice         */
/* densities and one vertex per lattice edge whose ends lie on         */
/* opposite sides of the iso-level, placed by linear interpolation.    */
/* ------------------------------------------------------------------ */
/* Lattice vertex (i, j, k), 0..64 per axis, FP32 in a fixed order:
 * x_a = -a + i * ((a - (-a)) / 64). */
void oc_lattice_vertex(const float half[3], int i, int j, int k, float x[3]) {
  const int idx[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    float lo = -half[a];
    float w = (half[a] - lo) / 64.0f;
    x[a] = lo + (float)idx[a] * w;
  }
}

/* Densities at the 65^3 lattice vertices, index i + 65 j + 65^2 k. */
void oc_density_lattice(const oc_config* c, const double* params, const float half[3], double* sigma) {
  for (int k = 0; k <= 64; ++k)
    for (int j = 0; j <= 64; ++j)
      for (int i = 0; i <= 64; ++i) {
        float p[3];
        oc_lattice_vertex(half, i, j, k, p);
        sigma[i + 65 * j + 65 * 65 * k] = oc_density(c, params, p, half);
      }
}

/* Edge-crossing vertices: for every lattice edge from vertex v along axis d
 * (v and its neighbour inside the lattice) with (sigma_v > iso) !=
 * (sigma_n > iso), in the order (vertex index, axis), writes the edge code
 * 3 v + d and the position p_v + t (p_n - p_v), t = (iso - sigma_v) /
 * (sigma_n - sigma_v), in FP64 from the FP32 lattice vertices.  Returns the
 * number of crossings (codes/pos may be NULL to count only). */
int64_t oc_mesh_vertices(const double* sigma, const float half[3], double iso, int64_t* codes, double* pos) {
  int64_t n = 0;
  for (int k = 0; k <= 64; ++k)
    for (int j = 0; j <= 64; ++j)
      for (int i = 0; i <= 64; ++i) {
        const int64_t v = i + 65 * j + 65 * 65 * k;
        const int ijk[3] = {i, j, k};
        for (int d = 0; d < 3; ++d) {
          if (ijk[d] == 64) continue;
          int nb[3] = {i, j, k};
          nb[d] += 1;
          const int64_t u = nb[0] + 65 * nb[1] + 65 * 65 * nb[2];
          if ((sigma[v] > iso) == (sigma[u] > iso)) continue;
          if (codes) codes[n] = 3 * v + d;
          if (pos) {
            float pv[3], pu[3];
            oc_lattice_vertex(half, i, j, k, pv);
            oc_lattice_vertex(half, nb[0], nb[1], nb[2], pu);
            const double t = (iso - sigma[v]) / (sigma[u] - sigma[v]);
            for (int a = 0; a < 3; ++a) pos[3 * n + a] = (double)pv[a] + t * ((double)pu[a] - (double)pv[a]);
          }
          ++n;
        }
      }
  return n;
}
