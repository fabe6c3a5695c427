/*
 * romap.h -- C ABI of the GB300 per-object NeRF training library.
 *
 * The library trains one small neural radiance field per detected object, as
 * in RO-MAP (Han et al., RA-L 2023): each object instance gets its own model
 * made of a multiresolution hash encoding and a tiny MLP (Sec. V), receives
 * rays from keyframes incrementally (Sec. V-A-1), and is trained by volume
 * rendering (Sec. V-B, Eq. 6) against the losses of Eq. 7-11 with Adam.  Many
 * objects train side by side on one GPU (Sec. V-A-2): one call of
 * romap_train_step runs a step of every listed object in one batched launch
 * sequence.
 *
 * Conventions
 *  - Every function returns a romap_status: ROMAP_OK (0) or a negative error.
 *    romap_last_error() returns the message of the calling thread's last
 *    error.  No C++ exception crosses this boundary.
 *  - The library owns all per-object device state (parameters, Adam moments,
 *    ray pools).  The caller owns every buffer it passes.  Host buffers are
 *    consumed before the call returns.  Device buffers (flag
 *    ROMAP_DEVICE_PTR, or the functional API below) must stay valid until the
 *    context's stream has passed the call.
 *  - All GPU work is enqueued on the CUDA stream given to romap_init.  Calls
 *    that return host data synchronise that stream.
 *  - A context is not thread-safe: use one per host thread, or lock.
 *  - Frames: rays are given in the world frame unless ROMAP_OBJECT_FRAME.
 *    The object frame is x_o = R_z(yaw)^T (x_w - t) (Sec. IV-B: objects have
 *    a translation and a yaw); its box is [-a, a] with a = half_size (Eq. 4).
 *    Directions are normalised by the library; depths are distances along
 *    the unit direction.
 */
#ifndef ROMAP_H
#define ROMAP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ROMAP_API __attribute__((visibility("default")))
#else
#define ROMAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t romap_status;
#define ROMAP_OK 0
#define ROMAP_ERR_INVALID_ARG (-1) /* null pointer, bad size or flag */
#define ROMAP_ERR_NOT_FOUND (-2)   /* unknown object id */
#define ROMAP_ERR_OOM (-3)         /* device or host allocation failed */
#define ROMAP_ERR_CAPACITY (-4)    /* more objects or rays than configured */
#define ROMAP_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define ROMAP_ERR_NONFINITE (-6)   /* NaN/Inf in inputs or in the loss */
#define ROMAP_ERR_TIMEOUT (-7)     /* a bounded device wait gave up */
#define ROMAP_ERR_BAD_STATE (-8)   /* call not valid in the object's state */
#define ROMAP_ERR_UNSUPPORTED (-9) /* configuration not built */
#define ROMAP_ERR_BOUNDS (-10)     /* libromap_checked.so: a device index failed its bounds check */

/* flags */
#define ROMAP_DEVICE_PTR 0x1u   /* pointers are device pointers */
#define ROMAP_OBJECT_FRAME 0x2u /* rays are already in the object frame */
#define ROMAP_REPLACE 0x4u      /* romap_add_rays: replace the pool instead of appending */
#define ROMAP_JITTER 0x8u       /* functional forward: stratified jitter instead of midpoints */
#define ROMAP_ASYNC_HOST 0x10u  /* romap_add_rays(_multi): page-locked host arrays are copied asynchronously on the
                                   context's stream; the caller keeps them unchanged until the stream has passed
                                   the call (without the flag the call waits for the copy) */
#define ROMAP_STORE_ACT 0x20u   /* functional forward/backward: the forward stores every sample's MLP activations
                                   (encoding, hidden layers, density-net outputs: about 4 (L F + 208) bytes per
                                   sample slot) in the workspace and the backward reads them back; without the flag
                                   (recompute) the backward re-gathers the encoding and recomputes the forward.  Both
                                   calls of a pair pass the same flags. */

/* ray classes from the instance mask (Sec. V-B) */
#define ROMAP_CLS_OBJECT 0     /* R_o: photometric loss, Eq. 7 */
#define ROMAP_CLS_BACKGROUND 1 /* R_b: random-colour loss and density loss, Eq. 9-10 */
#define ROMAP_CLS_OCCLUDER 2   /* no loss */

/* precision of the training step */
#define ROMAP_PREC_FP32 0       /* FP32 tables, FP32 SIMT MLP */
#define ROMAP_PREC_MIXED_BF16 1 /* FP16 table copy + FP32 masters, BF16 tensor-core MLP, FP32 accumulation */
#define ROMAP_PREC_MIXED_FP8 2  /* as MIXED_BF16, with the forward GEMM of the hidden 64x64 layer (colour net,
                                   second layer) in FP8 E4M3: each output row of the layer's weights scaled by
                                   448 / its max |W|, each sample's input activations by 448 / their max, FP32
                                   accumulation, dequantised before the ReLU; the backward stays BF16 */
#define ROMAP_PREC_MIXED_FP16 3 /* as MIXED_BF16 with FP16 MLP operands (11-bit significand instead of 8, range
                                   +-65504, saturated there); the backward's gradient operands are scaled by the
                                   object's batch size B (the losses are means over B rays) before rounding and the
                                   FP32 results unscaled */

typedef struct romap_ctx romap_ctx;

/* Model, loss and optimiser configuration (fixed per context).
 * Hash grid (Mueller et al. 2022, cited in Sec. II): n_levels levels of
 * n_features features; level l has resolution
 *   N_l = floor(base_resolution * b^l + 1e-6),
 * b = growth, or exp((ln max_resolution - ln base_resolution)/(n_levels-1))
 * when growth <= 0.  Level l is a dense grid of (N_l+1)^3 entries when that
 * is <= 2^log2_table_size, else a spatial hash of 2^log2_table_size entries.
 * MLP (Sec. V, "single-layer MLP", hidden 64): density net (L*F)->64->16
 * with ReLU, sigma = exp(clamp(out_0, -15, 15)); colour net
 * (15 geometry features + dir_dims)->64->64->3 with ReLU and sigmoid; no
 * biases (single_net = 0).  Loss weights lambda1, lambda2 of Eq. 11. */
typedef struct romap_config {
  int32_t n_levels;        /* L, 1..16 */
  int32_t n_features;      /* F, must be 2 */
  int32_t log2_table_size; /* log2 T, 8..24 */
  int32_t base_resolution; /* N_min >= 1 */
  double growth;           /* b; <= 0 to derive it from max_resolution */
  int32_t max_resolution;  /* N_max (used when growth <= 0) */
  int32_t hidden;          /* must be 64 */
  int32_t dir_dims;        /* 0 or 3 */
  int32_t n_samples;       /* N samples per ray, 1..1024 (Sec. V-B) */
  int32_t rays_per_step;   /* rays drawn per object per step (default) */
  float lambda1;           /* depth loss weight (Eq. 11) */
  float lambda2;           /* density loss weight (Eq. 11) */
  float lr, beta1, beta2, eps; /* Adam */
  int32_t bg_random;       /* 1: each ray composites over a random colour redrawn every step (Eq. 9) */
  float bg_const[3];       /* background colour when bg_random == 0 */
  int32_t precision;       /* ROMAP_PREC_* */
  int32_t max_objects;     /* capacity of live objects */
  int64_t max_rays_per_object; /* ray-pool capacity of one object */
  int32_t accuracy_mode;   /* 1: the FP32 path accumulates the transmittance log-sum (the prefix of
                              sigma * delta) and the compositing weights in FP64 (Eq. 6) */
  int32_t single_net;      /* 1: the single-network model of Sec. V (one hidden layer, position input
                              only): the colour logits are density-net outputs 1..3 and the colour-net
                              weights are neither read nor updated (their gradient stays 0).  Not
                              combined with ROMAP_PREC_MIXED_FP8. */
  int32_t hidden_layers;   /* hidden layers of width 64 of the single-network model (1..3, Table 4;
                              0 reads as 1); must be 0 or 1 when single_net == 0.  Layers 2 and 3 are
                              64x64 with ReLU, between the first hidden layer and the output layer. */
  int32_t deterministic;   /* 1: bit-reproducible training (ROMAP_PREC_FP32 only, else ROMAP_ERR_UNSUPPORTED):
                              every gradient contribution of the backward (hash scatter and MLP weight
                              gradients) and every per-ray loss term is rounded once to a 64-bit fixed-point
                              integer (2^-46 for gradients, 2^-32 for loss sums) and added with an integer
                              atomic, so sums do not depend on the order the GPU adds them in: two runs with the
                              same inputs give the same bits, and a batch of objects gives each object the bits
                              of its own separate step.  A contribution above 1024 in magnitude (2^20 for a
                              ray's loss) is not added and the step reports ROMAP_ERR_CAPACITY; per-entry sums
                              must stay within +-2^17.  Applies to training steps (romap_fn_backward keeps
                              floating-point atomics). */
  int32_t per_object;      /* 1: romap_train_step(_async) runs one launch sequence (one CUDA graph) per listed
                              object and step instead of one batched sequence for all of them (the plain
                              per-object path); 0: batched */
  int32_t reserved;        /* 0 */
  /* Optional device allocator (both or neither).  alloc returns NULL on
   * failure, which the library reports as ROMAP_ERR_OOM; a pointer that is
   * not 256-byte aligned is handed back to dealloc and reported as
   * ROMAP_ERR_INVALID_ARG. */
  void* (*alloc)(void* user, size_t bytes);
  void (*dealloc)(void* user, void* ptr);
  void* alloc_user;
} romap_config;

/* An object landmark: cuboid pose and size (Sec. IV-B, Eq. 1 and 4). */
typedef struct romap_object_desc {
  float t[3];            /* translation (world) */
  double yaw;            /* rotation about world z, radians */
  float half_size[3];    /* half extents a of the box */
  uint64_t seed;         /* random stream of this object (Philox4x32-10 key) */
  int32_t rays_per_step; /* rays per step for this object; 0 = config default */
} romap_object_desc;

/* Training rays, structure of arrays, n entries each (Sec. V-A-1: RGB,
 * instance mask class, sparse depth). */
typedef struct romap_rays {
  const float* origin;  /* [3n] */
  const float* dir;     /* [3n], any non-zero length */
  const float* rgb;     /* [3n] target colour in [0,1] */
  const float* depth;   /* [n] target depth, NaN = none; NULL = no depth */
  const uint8_t* cls;   /* [n] ROMAP_CLS_*; NULL = all object rays */
} romap_rays;

/* Parameter layout of one object (host-side description). */
typedef struct romap_layout {
  int64_t n_params;          /* hash entries * F + MLP weights */
  int64_t n_hash_params;
  int32_t n_levels;
  int32_t resolution[16];    /* N_l */
  int32_t dense[16];         /* 1 if level l is dense */
  int64_t level_offset[16];  /* first entry of level l: a multiple of 8; entries
                                between (N_l+1)^3 and the next level are unused */
  int64_t mlp_offset[7];     /* parameter offset of MLP layers: density 1, density 2 (output), colour 1, colour 2,
                                colour 3, then the single-network model's hidden layers 2 and 3 */
  int32_t mlp_rows[7], mlp_cols[7]; /* row-major [out][in] */
  int32_t n_mlp_layers;      /* 5, or 5 + hidden_layers - 1 for the single-network model */
} romap_layout;

/* Checkpoint of one object: caller-owned arrays of n_params floats each
 * (host, or device with ROMAP_DEVICE_PTR in flags). */
typedef struct romap_state {
  float* params;
  float* adam_m;
  float* adam_v;
  int64_t n_params;
  int64_t step;       /* Adam steps taken so far */
  uint32_t flags;
} romap_state;

/* Counters accumulated by the context since romap_reset_stats. */
typedef struct romap_stats {
  int64_t steps;          /* object-steps run */
  int64_t rays;           /* rays drawn */
  int64_t live_samples;   /* samples that went through forward, backward and Adam */
  int64_t kernel_launches;/* kernels enqueued by the library */
  int64_t graph_captures; /* training-step CUDA graphs captured (one per new batch composition) */
  int64_t graph_replays;  /* training steps run by replaying a cached graph */
} romap_stats;

/* ---- lifetime ---------------------------------------------------------- */
/* Validates cfg, selects the current CUDA device and binds the context to
 * cuda_stream (a cudaStream_t; NULL = legacy default stream). */
ROMAP_API romap_status romap_init(const romap_config* cfg, void* cuda_stream, romap_ctx** out);
ROMAP_API romap_status romap_destroy(romap_ctx* ctx);
ROMAP_API const char* romap_status_string(romap_status s);
/* Copies the calling thread's last error message (NUL-terminated). */
ROMAP_API romap_status romap_last_error(char* buf, size_t n);
/* Host-only: parameter layout implied by cfg (no GPU needed). */
ROMAP_API romap_status romap_param_layout(const romap_config* cfg, romap_layout* out);

/* ---- objects (Sec. V: one model per detected instance) ----------------- */
/* Allocates the object's parameters, Adam moments and ray pool, and
 * initialises the parameters: hash table U(-1e-4, 1e-4), MLP weights
 * Glorot-uniform, both from Philox4x32-10 keyed by desc->seed. */
ROMAP_API romap_status romap_create_object(romap_ctx* ctx, const romap_object_desc* desc, int32_t* out_id);
ROMAP_API romap_status romap_destroy_object(romap_ctx* ctx, int32_t id);
/* Occupancy bitgrid of 64^3 cells over the object's box, bit index
 * x + 64 y + 4096 z in 4096 uint64 words; samples in empty cells are
 * skipped (density 0).  bits == NULL removes the grid. */
ROMAP_API romap_status romap_set_occupancy(romap_ctx* ctx, int32_t id, const uint64_t* bits, uint32_t flags);
/* Occupancy from the learned density (empty-space skipping; not in the
 * paper).  Evaluates the object's density net (FP32 master parameters) at
 * the centre of each of the 64^3 cells of its box, x_a = -a + (i + 0.5)
 * (2a / 64) in FP32, keeps per cell d = max(decay * d, sigma) (d starts at
 * sigma on the first call and with flags ROMAP_REPLACE), and replaces the
 * object's bitgrid with d > threshold; later steps cull samples in cells
 * whose bit is 0.  decay in [0, 1], threshold finite and >= 0, else
 * ROMAP_ERR_INVALID_ARG.  Enqueued on the context's stream. */
ROMAP_API romap_status romap_update_occupancy(romap_ctx* ctx, int32_t id, float decay, float threshold,
                                              uint32_t flags);
/* Copies the object's bitgrid (4096 uint64 words) and/or the per-cell
 * densities of romap_update_occupancy (64^3 floats, x fastest) to host
 * memory; either pointer may be NULL.  ROMAP_ERR_BAD_STATE if a requested
 * array does not exist yet. */
ROMAP_API romap_status romap_get_occupancy(romap_ctx* ctx, int32_t id, uint64_t* bits, float* density);
/* Appends n rays to the object's pool (incremental data, Sec. V-A-1), or
 * replaces the pool with ROMAP_REPLACE.  Rays are moved to the object frame
 * and their directions normalised on the device. */
ROMAP_API romap_status romap_add_rays(romap_ctx* ctx, int32_t id, const romap_rays* rays, int64_t n, uint32_t flags);
/* romap_add_rays for several objects in one call: one keyframe's rays of
 * every object it shows (Sec. V-A-1 feeds each object's model the rays of
 * its detection box in every new keyframe).  rays holds the concatenation:
 * counts[k] rays of object ids[k] follow the counts[k-1] rays of ids[k-1].
 * n_ids distinct ids (else ROMAP_ERR_INVALID_ARG), counts[k] >= 0 (0 leaves
 * the pool, or with ROMAP_REPLACE empties it).  Flags, host checks and
 * ownership as romap_add_rays; host arrays are copied once and every
 * object's rays are transformed by one launch.  Every argument and capacity
 * is checked before any pool changes. */
ROMAP_API romap_status romap_add_rays_multi(romap_ctx* ctx, const int32_t* ids, const int64_t* counts, int32_t n_ids,
                                            const romap_rays* rays, uint32_t flags);
ROMAP_API romap_status romap_pool_size(romap_ctx* ctx, int32_t id, int64_t* out_n);

/* ---- training (Sec. V-A, V-B; Eq. 6-11; Adam) -------------------------- */
/* Runs n_steps training steps of every listed object (one batched launch
 * sequence per step; with per_object, one per object and step).  The first
 * step of a batch composition (the listed objects and their rays per step)
 * runs eagerly and is captured as a CUDA graph; later steps of that
 * composition replay it.  The context keeps the graphs of up to 128
 * compositions and evicts the least recently used one beyond that.  Each step of an
 * object draws B = min(rays_per_step, pool size) rays (uniformly with
 * replacement, or the whole pool in order when B equals the pool size),
 * samples N stratified points in the box per ray, encodes and evaluates
 * them, composites (Eq. 6), evaluates L = L_rgb + L_rr + lambda1 L_depth +
 * lambda2 L_density (Eq. 11, every term divided by B), backpropagates and
 * applies Adam.  out_loss (host, nullable) receives n_ids losses of the
 * last step.  Listed ids must be distinct. */
ROMAP_API romap_status romap_train_step(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, int32_t n_steps, float* out_loss);
/* romap_train_step without waiting for the device: the steps and, when
 * out_loss is not NULL, a copy of the last step's n_ids losses into out_loss
 * (page-locked host or device memory; other host memory makes the call wait
 * for the copy) are enqueued on the context's stream and the call returns.
 * Read out_loss after the stream has passed the call (an event recorded on
 * the stream after it, or a stream synchronisation), so that the host can
 * prepare the next step's rays while the device trains.  Device-side errors
 * of these steps (a non-finite loss, which also shows in out_loss, or a
 * bounded wait that gave up) are reported by romap_check_device_status or
 * by the next call that reads losses synchronously. */
ROMAP_API romap_status romap_train_step_async(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, int32_t n_steps,
                                              float* out_loss);
/* Waits for the context's stream and reports (then clears) the device
 * status word: ROMAP_ERR_NONFINITE for a non-finite loss, ROMAP_ERR_TIMEOUT
 * for a bounded device wait that gave up, else ROMAP_OK. */
ROMAP_API romap_status romap_check_device_status(romap_ctx* ctx);
/* The forward/backward half of a step without Adam: gradients are left in
 * the objects' gradient buffers (read them with romap_get_grad).
 * out_loss (host, nullable): 5 floats per object: L, then the rgb, rr,
 * depth and density sums divided by B. */
ROMAP_API romap_status romap_forward_backward(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, float* out_loss);
/* Adam on the listed objects' gradients; zeroes the gradients. */
ROMAP_API romap_status romap_adam_step(romap_ctx* ctx, const int32_t* ids, int32_t n_ids);
/* Copies the object's gradient buffer (n_params floats). */
ROMAP_API romap_status romap_get_grad(romap_ctx* ctx, int32_t id, float* out, uint32_t flags);
/* Copies the last step's ray draw of an object: pool index (int64) and
 * background colour (3 floats) per ray.  Either pointer may be NULL. */
ROMAP_API romap_status romap_last_batch(romap_ctx* ctx, int32_t id, int64_t* pool_idx, float* bg, int64_t* out_n);
/* Copies the per-ray outputs of the object's rays in the last step, in ray
 * slot order: [C_hat rgb (3), D_hat, opacity A, sum of sigma] (Eq. 6), 6
 * floats per ray, computed in the step's precision.  out may be NULL. */
ROMAP_API romap_status romap_last_outputs(romap_ctx* ctx, int32_t id, float* out, int64_t* out_n);

/* ---- incremental training data and budgeted training ------------------- */
/* Eq. 5 (Sec. V-A-1): the angle, in degrees, between the vectors from the
 * object centre to the camera centre of the last image used for training
 * (cam_last) and to the current camera centre (cam_now); world frame, FP64.
 * A camera at the object centre gives 180.  Host-only, needs no context. */
ROMAP_API romap_status romap_view_angle(const double cam_last[3], const double cam_now[3], const double center[3],
                                        double* out_deg);
/* The incremental data rule: if the object has no image yet, or the Eq. 5
 * angle between its last used camera centre and cam_center (world) around
 * the object's centre (desc t) exceeds threshold_deg (Sec. VI: 25), appends
 * the rays (as romap_add_rays with flags) , records cam_center as the last
 * used image and grants `iterations` more training steps (Sec. VI: 300);
 * otherwise the rays are ignored.  *out_updated (nullable) = 1 / 0. */
ROMAP_API romap_status romap_observe(romap_ctx* ctx, int32_t id, const double cam_center[3], float threshold_deg,
                                     const romap_rays* rays, int64_t n, uint32_t flags, int32_t iterations,
                                     int32_t* out_updated);
/* Training steps still owed to the object (granted by romap_observe,
 * consumed by romap_train_budget). */
ROMAP_API romap_status romap_pending(romap_ctx* ctx, int32_t id, int64_t* out);
ROMAP_API romap_status romap_set_pending(romap_ctx* ctx, int32_t id, int64_t pending);
/* Budgeted training of the listed objects that still owe steps: batched
 * steps (CUDA-graph replays) of all of them, in chunks of at most max_chunk
 * (<= 0: 64), while the device time of the steps so far plus the step time
 * of the batch fits in budget_ms.  The step time of a batch composition is
 * the measured one, else predicted from the measured time per ray; with
 * nothing measured yet, one step runs to measure it.  When the whole batch
 * no longer fits, one step trains the objects that owe the most steps, as
 * many as fit.  An object leaves the batch when its owed steps reach 0.
 * Blocks until the steps finish.  out_steps: batched steps run; out_ms:
 * their device time; out_loss (n_ids, nullable): each object's last loss,
 * NaN if it did not train. */
ROMAP_API romap_status romap_train_budget(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, float budget_ms,
                                          int32_t max_chunk, int32_t* out_steps, float* out_ms, float* out_loss);

/* ---- mesh extraction (Table 3: marching cubes, 64^3) -------------------- */
/* Densities of the object's density net (FP32 master parameters) at the
 * 65^3 lattice vertices of its box, x_a = -a + i (2a / 64) (FP32), index
 * i + 65 j + 65^2 k, into out (host, or device with ROMAP_DEVICE_PTR). */
ROMAP_API romap_status romap_density_lattice(romap_ctx* ctx, int32_t id, float* out, uint32_t flags);
/* Marching cubes (Lorensen & Cline 1987) over the 64^3 cubes of the
 * object's box at density iso-level `iso`: one vertex (object frame, 3
 * floats) per lattice edge whose end densities lie on opposite sides of
 * iso, by linear interpolation, numbered in lattice-vertex order (x fastest)
 * then axis; per cube the triangles of its case (romap_mc_case_table) as
 * vertex-index triples, in cube order, facing from the dense side to the
 * empty side.  The surface is closed except where it meets the box.  The
 * counts go to *out_n_vertices / *out_n_triangles (nullable); if they exceed
 * max_vertices / max_triangles nothing is written and ROMAP_ERR_CAPACITY is
 * returned, so a caller can size its buffers and call again.  Outputs are
 * host memory, or device memory with ROMAP_DEVICE_PTR. */
ROMAP_API romap_status romap_extract_mesh(romap_ctx* ctx, int32_t id, float iso, float* vertices,
                                          int64_t max_vertices, int32_t* triangles, int64_t max_triangles,
                                          int64_t* out_n_vertices, int64_t* out_n_triangles, uint32_t flags);
/* The marching-cubes case table the mesh extraction uses, built by
 * construction at load time: for each of the 256 inside/outside patterns of
 * a cube's corners (corner c at (c & 1, (c >> 1) & 1, (c >> 2) & 1); bit c
 * set = density above the iso-level), counts[case] triangles listed in
 * triangles[case * 16 ..] as triples of edge numbers (edge 4 d + q along
 * axis d; q = the other two axes' corner bits, lower axis first), -1 after
 * the last; triangles face from inside to outside.  Host-only. */
ROMAP_API romap_status romap_mc_case_table(int8_t* triangles, uint8_t* counts);

/* ---- inference --------------------------------------------------------- */
/* Renders n rays (world frame unless ROMAP_OBJECT_FRAME) with midpoint
 * samples over bg (3 floats, host).  Outputs per ray (nullable each):
 * out_rgb [3n], out_depth [n], out_opacity [n]; host unless
 * ROMAP_DEVICE_PTR, in which case every pointer is a device pointer. */
ROMAP_API romap_status romap_render(romap_ctx* ctx, int32_t id, const float* origin, const float* dir, int64_t n,
                          const float bg[3], float* out_rgb, float* out_depth, float* out_opacity, uint32_t flags);

/* ---- checkpoint -------------------------------------------------------- */
ROMAP_API romap_status romap_get_state(romap_ctx* ctx, int32_t id, romap_state* out);
ROMAP_API romap_status romap_set_state(romap_ctx* ctx, int32_t id, const romap_state* in);

/* ---- functional, differentiable API (device buffers only) ------------- */
/* These run the same kernels as training on caller-owned device buffers so
 * that a differentiable wrapper can call forward and backward separately.
 * rays: n object-frame rays (origin [3n], dir [3n], unit length), bg [3n].
 * The RNG of ray r uses key seed and counter (step, r, purpose, .).
 * Outputs per ray: out_ray [6n] = (C_hat rgb, D_hat, opacity A = 1 -
 * T_{N+1}, sum_i sigma_i over live samples).  workspace holds the samples
 * (and with ROMAP_STORE_ACT the activations) between forward and backward;
 * its size comes from romap_fn_workspace_size with the same n and flags.
 * Flags: ROMAP_JITTER, ROMAP_STORE_ACT.  n in 1..2^24. */
ROMAP_API romap_status romap_fn_workspace_size(romap_ctx* ctx, int64_t n, uint32_t flags, size_t* bytes);
ROMAP_API romap_status romap_fn_forward(romap_ctx* ctx, const float* params, const float half_size[3], uint64_t seed,
                              uint32_t step, const uint64_t* occupancy, const float* origin, const float* dir,
                              const float* bg, int64_t n, uint32_t flags, void* workspace, size_t ws_bytes,
                              float* out_ray, float* out_samples);
/* Backward of romap_fn_forward given dL/d(out_ray) grad_ray [6n]; adds
 * dL/dparams into grad_params (n_params floats, device, 16-byte aligned,
 * else ROMAP_ERR_INVALID_ARG).  out_dsigma
 * (nullable, [n*N]) receives dL/dsigma per sample slot (0 for missed or
 * culled slots).  flags: as in the forward (ROMAP_JITTER, ROMAP_STORE_ACT).
 * The gradient uses floating-point atomics even in the deterministic
 * mode. */
ROMAP_API romap_status romap_fn_backward(romap_ctx* ctx, const float* params, const float half_size[3], uint64_t seed,
                               uint32_t step, const uint64_t* occupancy, const float* origin, const float* dir,
                               const float* bg, int64_t n, uint32_t flags, void* workspace, size_t ws_bytes,
                               const float* grad_ray, float* grad_params, float* out_dsigma);

/* Same as romap_fn_forward, without a context and without any device
 * allocation by the library or the caller: for callers that cannot allocate
 * device memory where they render (a plugin whose host framework owns all
 * device memory and offers no allocator; a real-time loop that must not call
 * cudaMalloc/cudaFree because they can synchronise the device).  The paper
 * has no counterpart; this is a deployment convenience.
 *  - Scratch lives in one static 32 MiB device array inside the library.
 *    A device reserves it when the library's device code is first loaded
 *    there (with lazy module loading, possibly at this call) and holds it
 *    until process exit.  n must be in 1..2^24, and calls whose scratch
 *    would not fit (about n * (105 + 60 * n_samples) bytes) return
 *    ROMAP_ERR_CAPACITY with the largest n that fits.
 *  - The first call on each device resolves the array's device address
 *    (cudaGetSymbolAddress) with that device current.  cuda_stream must
 *    belong to the current device, else ROMAP_ERR_INVALID_ARG.
 *  - The object record and batch arrays are written into the array by a
 *    kernel that receives them by value: nothing is read from host memory
 *    after the call returns.
 *  - All calls on a device share the array: calls that overlap on the GPU
 *    race and must be serialised by the caller.
 * cfg as for romap_init (validated, nothing allocated); cuda_stream is a
 * cudaStream_t (NULL = legacy default stream); every pointer is a device
 * pointer except cfg and half_size (host); out_ray [6n] as for
 * romap_fn_forward. */
ROMAP_API romap_status romap_fn_forward_noalloc(const romap_config* cfg, void* cuda_stream, const float* params,
                                                const float half_size[3], uint64_t seed, uint32_t step,
                                                const uint64_t* occupancy, const float* origin, const float* dir,
                                                const float* bg, int64_t n, uint32_t flags, float* out_ray);

/* ---- counters ---------------------------------------------------------- */
ROMAP_API romap_status romap_get_stats(romap_ctx* ctx, romap_stats* out);
/* Also clears the phase times below. */
ROMAP_API romap_status romap_reset_stats(romap_ctx* ctx);
/* Phase timing: while on, every phase of a step is bracketed by CUDA events
 * on the context's stream.  romap_phase_times synchronises the stream and
 * returns, per phase, the device milliseconds and kernel launches since the
 * last reset: [0] sampling (ray draw, scan, sample write), [1] MLP forward,
 * [2] compositing + loss + adjoint, [3] MLP backward + hash scatter,
 * [4] Adam.  ms and launches point to ROMAP_N_PHASES entries (launches
 * nullable). */
#define ROMAP_N_PHASES 5
/* Autotuner of the mixed-precision step: the first mixed step of a context
 * times each candidate fused tile kernel on that batch and keeps the
 * fastest.  chosen receives its index (-1 before the first mixed step), ms
 * (n entries) the measured milliseconds per launch, names (nullable) the
 * candidates' names separated by ';'. */
/* Failure-detection self-test: runs a kernel whose bounded wait on an
 * mbarrier that nothing signals gives up after poll_limit polls, records
 * the time-out in the device status word, frees its tensor memory and
 * returns.  Returns ROMAP_ERR_TIMEOUT when the device reported the time-out
 * (the expected outcome); the context stays usable. */
ROMAP_API romap_status romap_selftest_wait_timeout(romap_ctx* ctx, int32_t poll_limit);
/* Forces candidate `index`, or -1 to autotune again at the next mixed
 * step.  Candidates: 0 = lockstep tile pairs, 1 = warp-specialized, each
 * giving every CTA a contiguous range of the tile plan; 2 and 3 = the same
 * kernels with the plan interleaved over the CTAs (CTA c takes every
 * grid-th pair or tile from c, so all CTAs work on the same few objects at
 * a time); 4, 5 and 6, 7 = interleaved in chunks of 2 and 4 consecutive
 * pairs or tiles (longer runs of one object per CTA); 8, 9, 10, 11 = the
 * lockstep kernel on single tiles of 128 slots, two CTAs per SM, with the
 * contiguous, interleaved, by-2 and by-4 orders; 12, 13, 14, 15 = tile
 * pairs whose two warpgroups run decoupled (own MMA issue and barriers,
 * meeting only at object changes), same orders.  Only 0, 2, 4 and 6 run
 * ROMAP_PREC_MIXED_FP8 or the single_net model: ROMAP_ERR_UNSUPPORTED for
 * the others there. */
ROMAP_API romap_status romap_set_tile_kernel(romap_ctx* ctx, int32_t index);
ROMAP_API romap_status romap_autotune_report(romap_ctx* ctx, int32_t* chosen, float* ms, int32_t n, char* names,
                                             size_t names_len);
ROMAP_API romap_status romap_set_profiling(romap_ctx* ctx, int32_t on);
/* Adam (Kingma & Ba) skips parameter chunks (256 parameters) whose
 * gradient has been zero at every step so far: their moments are then 0 and
 * their update is exactly 0, so the skip changes no bit of the parameters,
 * moments or FP16 table copy; it saves the traffic of untouched table
 * regions (empty space of a culled object).  on = 0 updates every chunk
 * (dense Adam, for comparison); on = 1 (the default) skips.  A state load
 * (romap_set_state) marks the chunks whose loaded moments are non-zero.
 * Drops the captured step graphs. */
ROMAP_API romap_status romap_set_adam_skip(romap_ctx* ctx, int32_t on);
/* on = 0: training steps launch their kernels eagerly, every step (no CUDA
 * graph capture or replay; drops the cached graphs); on = 1 (the default):
 * the first step of a composition is captured and later ones replayed. */
ROMAP_API romap_status romap_set_graphs(romap_ctx* ctx, int32_t on);

/* ---- bounds-checked build ------------------------------------------------
 * libromap_checked.so is this library compiled with ROMAP_CHECKED: every
 * device index into a ray pool, a hash table level, the ray and sample
 * records and the tile plan is checked against its logical size; a failed
 * check records the violation in the context's status word and the kernel
 * uses a safe in-range index (or skips the write) instead, never a trap.
 * Calls that report device status (loss reads, romap_check_device_status)
 * then return ROMAP_ERR_BOUNDS.  The unchecked library compiles the checks
 * away.  romap_checked_build tells which one is loaded (*out = 1 checked). */
ROMAP_API romap_status romap_checked_build(int32_t* out);
/* Test hook for the bounds checks: sets the object's pool size as the
 * kernels see it to n (0..its pool size), leaving its rays per step and its
 * pool as they are, so that the next step's ray draw indexes past the
 * logical pool while staying inside the allocated one.  Drops the captured
 * step graphs. */
ROMAP_API romap_status romap_debug_set_pool_size(romap_ctx* ctx, int32_t id, int64_t n);
ROMAP_API romap_status romap_phase_times(romap_ctx* ctx, double* ms, int64_t* launches);

/* Measurement utility (no counterpart in the paper): the request rates that
 * bound the fused training kernel's hash gather and scatter, measured on
 * the current device.  Every lane issues its own pseudo-random request into
 * an L2-resident buffer (32 MiB of 4-byte words; 64 MiB of float pairs),
 * 8 in flight per thread, 2048 threads per SM.  out[0] = 4-byte loads per
 * second, out[1] = red.global.add.v2.f32 reductions per second, out[2] =
 * load + reduction pairs per second (the fused kernel issues one 4-byte
 * gather and one 8-byte reduction per corner and level).  Best of three
 * timed launches on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream); allocates about 96 MiB with cudaMalloc for the duration of the
 * call and synchronises the stream. */
ROMAP_API romap_status romap_measure_request_rates(void* cuda_stream, double* out);

#ifdef __cplusplus
}
#endif
#endif /* ROMAP_H */
