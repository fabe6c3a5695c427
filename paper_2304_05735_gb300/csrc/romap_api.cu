// Host runtime of libromap: the C ABI declared in include/romap.h.
//
// It owns contexts, objects (parameters, Adam moments, ray pools, occupancy
// grids), the per-step workspace, and the launch sequence of a training
// step on the context's stream:
//   ray setup -> scan -> sample write -> tile forward -> composite/loss/adjoint
//   -> tile backward -> Adam (+ step counter advance)
// Every object's step counter (the Philox counter of its ray draw and the
// Adam bias-correction exponent) lives on the device and is advanced by the
// Adam launch, so a step's launch sequence does not depend on host state
// that changes from step to step.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <limits>
#include <string>
#include <map>
#include <vector>

#include "romap.h"
#include "romap_internal.cuh"

using namespace romap;

namespace {

thread_local std::string g_last_error;

romap_status fail(romap_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (expr);                                                                            \
    if (e_ != cudaSuccess) return fail(ROMAP_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                             \
  } while (0)

#define ROMAP_TRY(expr)            \
  do {                             \
    romap_status s_ = (expr);      \
    if (s_ != ROMAP_OK) return s_; \
  } while (0)

struct Object {
  bool alive = false;
  romap_object_desc desc{};
  float* params = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  uint16_t* table_h = nullptr;
  float* pool_o = nullptr;
  float* pool_d = nullptr;
  float* pool_rgb = nullptr;
  float* pool_depth = nullptr;
  uint8_t* pool_cls = nullptr;
  int64_t pool_n = 0, pool_cap = 0;
  uint64_t* occ = nullptr;
  float* occ_density = nullptr;  // per-cell moving maximum of the learned density (romap_update_occupancy)
  unsigned long long* gfix = nullptr;  // deterministic mode: fixed-point gradient accumulator
  uint8_t* touched = nullptr;          // Adam's per-chunk touched flags
  // incremental training data (Eq. 5): camera centre of the last image used, training iterations still owed
  bool have_view = false;
  double last_view[3] = {0, 0, 0};
  int64_t pending = 0;
  int64_t steps_done = 0;
  int32_t rays_per_step = 0;
};

// A device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct romap_ctx {
  romap_config cfg{};
  GridParams g{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sms = 0;
  std::vector<Object> objs;
  std::vector<ObjectDev> objs_host;  // mirror of objs_dev
  ObjectDev* objs_dev = nullptr;
  ObjectDev* fn_obj_dev = nullptr;   // object record of functional calls
  // step workspace
  DevBuf ws_rays, ws_samples, ws_blocks, ws_batch, ws_dyn, ws_stage, ws_plan, ws_mesh, ws_mesh_out, ws_loss;
  int64_t cap_rays = 0, cap_samples = 0, cap_blocks = 0, cap_batch = 0;
  // tile plan of the mixed-precision path (capacities: rays, ray blocks, batch entries, tiles)
  int64_t cap_plan[4] = {0, 0, 0, 0};
  struct PlanView {
    uint32_t* hist = nullptr;
    uint32_t* bcnt = nullptr;
    int4* pat = nullptr;
    int32_t* npat = nullptr;
    int4* seg = nullptr;
    int32_t* nseg = nullptr;
    int32_t* ent = nullptr;
    int32_t* perm = nullptr;
    int32_t* rstart = nullptr;
    int2* slot = nullptr;
    int4* tiles = nullptr;
    int32_t* npairs = nullptr;
  } plan;
  RayBuf R{};
  SampleBuf S{};
  uint32_t* block_sums = nullptr;
  BatchDyn* dyn = nullptr;
  int32_t* totals = nullptr;
  int32_t* status = nullptr;
  unsigned long long* live_counter = nullptr;
  int32_t* batch_arrays = nullptr;
  std::vector<int32_t> batch_key;  // host copy of the batch arrays uploaded to ws_batch
  int batch_n = 0;                 // entries of the uploaded batch
  std::vector<int32_t> last_batch; // batch arrays of the last step that ran (eager or replayed)
  int last_batch_n = 0;
  const int32_t* batch_override = nullptr;  // while capturing: the graph's own copy of its batch arrays
  BatchDyn* dyn_host = nullptr;    // pinned
  BatchDyn* dyn_gather = nullptr;  // per_object: each listed object's BatchDyn after its last step [max_objects]
  BatchDyn* dyn_gather_host = nullptr;  // pinned [max_objects]
  romap_stats stats{};
  int64_t launches = 0;
  // autotuned choice of the mixed-precision tile kernel: -1 until tuned, then an index of kTileKernels
  int tile_kernel = -1;
  float tile_kernel_ms[16] = {};
  // CUDA graphs of one training step, one per batch composition (captured on cap_stream, replayed on stream), least
  // recently used first out beyond kMaxStepGraphs
  struct StepGraph {
    std::vector<int32_t> key;
    cudaGraphExec_t exec = nullptr;
    int32_t* batch_dev = nullptr;      // the graph's own device copy of its batch arrays
    std::vector<int32_t> batch;        // host copy of them
    int batch_n = 0;
    int launches = 0;                  // kernels one replay runs
    uint64_t last_use = 0;
    uint64_t ws_generation = 0;        // workspace generation it was captured against
  };
  cudaStream_t cap_stream = nullptr;
  // a second stream on which a step's Adam update of the step before overlaps the step's sampling (n_steps > 1 in
  // one call): side_stream for eager launches, cap_side while a graph is captured, side the one in use
  cudaStream_t side_stream = nullptr, cap_side = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<StepGraph> graphs;
  uint64_t graph_clock = 0;
  int64_t graph_captures = 0, graph_replays = 0;
  uint64_t ws_generation = 0;   // bumped whenever a workspace buffer moves
  bool graphs_enabled = true;
  // budgeted training: measured step time of each batch composition (ms, moving average)
  std::map<std::vector<int32_t>, double> step_ms_est;
  double ms_per_ray = -1.0;  // device time of one step per ray of the batch (moving average), -1 until measured
  // phase timing
  bool profiling = false;
  struct Prof { int phase; cudaEvent_t a, b; int launches; };
  std::vector<Prof> prof;
  double phase_ms[ROMAP_N_PHASES] = {0};
  int64_t phase_launches[ROMAP_N_PHASES] = {0};
};

namespace {

romap_status dev_alloc(romap_ctx* ctx, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->cfg.alloc) {
    *out = ctx->cfg.alloc(ctx->cfg.alloc_user, bytes);
    if (!*out) return fail(ROMAP_ERR_OOM, "device allocation of %zu bytes failed (caller allocator)", bytes);
    if (reinterpret_cast<uintptr_t>(*out) % 256 != 0) {  // vector loads and reductions assume aligned bases
      ctx->cfg.dealloc(ctx->cfg.alloc_user, *out);
      *out = nullptr;
      return fail(ROMAP_ERR_INVALID_ARG, "the caller allocator returned a pointer that is not 256-byte aligned");
    }
    return ROMAP_OK;
  }
  cudaError_t e = cudaMallocAsync(out, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return fail(ROMAP_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  return ROMAP_OK;
}

void dev_free(romap_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->cfg.alloc) ctx->cfg.dealloc(ctx->cfg.alloc_user, p);
  else cudaFreeAsync(p, ctx->stream);
}

template <class T>
romap_status dev_alloc_t(romap_ctx* ctx, size_t count, T** out) {
  void* p = nullptr;
  romap_status s = dev_alloc(ctx, count * sizeof(T), &p);
  *out = static_cast<T*>(p);
  return s;
}

romap_status grow(romap_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return ROMAP_OK;
  size_t nb = bytes + bytes / 4;
  void* p = nullptr;
  ROMAP_TRY(dev_alloc(ctx, nb, &p));
  dev_free(ctx, b.p);
  b.p = p;
  b.bytes = nb;
  ctx->ws_generation += 1;
  return ROMAP_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves a RayBuf of capacity nr from base; returns bytes used.  with_mask: the live-candidate masks of the tile
// plan (mixed-precision training).
size_t carve_rays(char* base, int64_t nr, RayBuf* R, bool with_mask = false) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + o : nullptr;
    o = align_up(o + bytes, 256);
    return p;
  };
  R->o = (float*)take(sizeof(float) * 3 * nr);
  R->d = (float*)take(sizeof(float) * 3 * nr);
  R->tn = (float*)take(sizeof(float) * nr);
  R->tf = (float*)take(sizeof(float) * nr);
  R->bg = (float*)take(sizeof(float) * 3 * nr);
  R->rgb = (float*)take(sizeof(float) * 3 * nr);
  R->depth = (float*)take(sizeof(float) * nr);
  R->cls = (uint8_t*)take(nr);
  R->pool_idx = (int64_t*)take(sizeof(int64_t) * nr);
  R->count = (uint32_t*)take(sizeof(uint32_t) * nr);
  R->off = (uint32_t*)take(sizeof(uint32_t) * nr);
  R->obj = (int32_t*)take(sizeof(int32_t) * nr);
  R->out = (float*)take(sizeof(float) * 6 * nr);
  R->mask = with_mask ? (uint32_t*)take(sizeof(uint32_t) * 4 * nr) : nullptr;
  R->gout = nullptr;
  return o;
}

// Carves the tile-plan arrays for capacities cap = {rays, ray blocks, batch entries, tiles}; returns bytes used.
size_t carve_plan(char* base, const int64_t cap[4], romap_ctx::PlanView* P) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + o : nullptr;
    o = align_up(o + bytes, 256);
    return p;
  };
  P->hist = (uint32_t*)take(sizeof(uint32_t) * kPlanCounts * cap[2]);
  P->bcnt = (uint32_t*)take(sizeof(uint32_t) * kPlanCounts * cap[1]);
  P->pat = (int4*)take(sizeof(int4) * 2 * kPlanMaxPat * cap[2]);
  P->npat = (int32_t*)take(sizeof(int32_t) * cap[2]);
  P->seg = (int4*)take(sizeof(int4) * 2 * kPlanSegsPerCount * kPlanCounts * cap[2]);
  P->nseg = (int32_t*)take(sizeof(int32_t) * kPlanCounts * cap[2]);
  P->ent = (int32_t*)take(sizeof(int32_t) * cap[2]);
  P->perm = (int32_t*)take(sizeof(int32_t) * cap[0]);
  P->rstart = (int32_t*)take(sizeof(int32_t) * cap[0]);
  P->slot = (int2*)take(sizeof(int2) * kTile * cap[3]);
  P->tiles = (int4*)take(sizeof(int4) * cap[3]);
  P->npairs = (int32_t*)take(sizeof(int32_t));
  return o;
}

romap_status ensure_plan(romap_ctx* ctx, int64_t nr, int64_t nblocks, int64_t nbatch, int64_t ntiles) {
  const int64_t need[4] = {nr, nblocks, nbatch, ntiles};
  bool fits = true;
  for (int k = 0; k < 4; ++k) fits = fits && need[k] <= ctx->cap_plan[k];
  if (fits) return ROMAP_OK;
  int64_t cap[4];
  for (int k = 0; k < 4; ++k) {
    cap[k] = ctx->cap_plan[k];
    if (need[k] > cap[k]) cap[k] = need[k] + need[k] / 4 + 64;
  }
  romap_ctx::PlanView pv;
  ROMAP_TRY(grow(ctx, ctx->ws_plan, carve_plan(nullptr, cap, &pv)));
  carve_plan((char*)ctx->ws_plan.p, cap, &ctx->plan);
  for (int k = 0; k < 4; ++k) ctx->cap_plan[k] = cap[k];
  // the count histograms start at zero; each step's pattern kernel resets the entries it read
  CUDA_TRY(cudaMemsetAsync(ctx->plan.hist, 0, sizeof(uint32_t) * kPlanCounts * cap[2], ctx->stream));
  ctx->ws_generation += 1;
  return ROMAP_OK;
}

size_t carve_samples(char* base, int64_t ns, SampleBuf* S) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + o : nullptr;
    o = align_up(o + bytes, 256);
    return p;
  };
  S->x = (float*)take(sizeof(float) * 3 * ns);
  S->t = (float*)take(sizeof(float) * ns);
  S->dt = (float*)take(sizeof(float) * ns);
  S->ray = (uint32_t*)take(sizeof(uint32_t) * ns);
  S->cand = (uint32_t*)take(sizeof(uint32_t) * ns);
  S->sigma = (float*)take(sizeof(float) * ns);
  S->rgb = (float*)take(sizeof(float) * 3 * ns);
  S->dsigma = (float*)take(sizeof(float) * ns);
  S->drgb = (float*)take(sizeof(float) * 3 * ns);
  S->act = nullptr;  // stored activations are carved separately (functional API with ROMAP_STORE_ACT)
  return o;
}

romap_status ensure_workspace(romap_ctx* ctx, int64_t nr, int64_t ns, int64_t nblocks, int64_t nbatch) {
  if (nr > ctx->cap_rays) {
    int64_t cap = nr + nr / 4 + 256;
    ROMAP_TRY(grow(ctx, ctx->ws_rays, carve_rays(nullptr, cap, &ctx->R, true)));
    carve_rays((char*)ctx->ws_rays.p, cap, &ctx->R, true);
    ctx->cap_rays = cap;
  }
  if (ns > ctx->cap_samples) {
    int64_t cap = ns + ns / 4 + 1024;
    ROMAP_TRY(grow(ctx, ctx->ws_samples, carve_samples(nullptr, cap, &ctx->S)));
    carve_samples((char*)ctx->ws_samples.p, cap, &ctx->S);
    ctx->cap_samples = cap;
  }
  if (nblocks > ctx->cap_blocks) {
    int64_t cap = nblocks + 64;
    ROMAP_TRY(grow(ctx, ctx->ws_blocks, sizeof(uint32_t) * cap));
    ctx->block_sums = (uint32_t*)ctx->ws_blocks.p;
    ctx->cap_blocks = cap;
  }
  if (nbatch > ctx->cap_batch) {
    int64_t cap = nbatch < 64 ? 64 : nbatch;
    ROMAP_TRY(grow(ctx, ctx->ws_dyn, sizeof(BatchDyn) * cap));
    ctx->dyn = (BatchDyn*)ctx->ws_dyn.p;
    if (ctx->dyn_host) cudaFreeHost(ctx->dyn_host);
    CUDA_TRY(cudaMallocHost((void**)&ctx->dyn_host, sizeof(BatchDyn) * cap));
    ctx->cap_batch = cap;
  }
  return ROMAP_OK;
}

// Batch arrays: slot[n], ray_base[n+1], block_base[n+1], tile_base[n+1], block_obj[n_blocks].
struct HostBatch {
  std::vector<int32_t> arr;
  int n = 0, n_blocks = 0, n_rays = 0, n_tiles = 0;
};

void build_batch(const std::vector<int32_t>& slots, const std::vector<int32_t>& rays, HostBatch* hb) {
  int n = (int)slots.size();
  hb->n = n;
  std::vector<int32_t> ray_base(n + 1, 0), block_base(n + 1, 0), tile_base(n + 1, 0), block_obj;
  for (int i = 0; i < n; ++i) {
    ray_base[i + 1] = ray_base[i] + rays[i];
    int nb = (rays[i] + 255) / 256;
    block_base[i + 1] = block_base[i] + nb;
    for (int k = 0; k < nb; ++k) block_obj.push_back(i);
    tile_base[i + 1] = tile_base[i];  // (tiles of the FP32 path are placed on the device)
  }
  hb->n_rays = ray_base[n];
  hb->n_blocks = block_base[n];
  hb->n_tiles = tile_base[n];
  hb->arr.clear();
  hb->arr.insert(hb->arr.end(), slots.begin(), slots.end());
  hb->arr.insert(hb->arr.end(), ray_base.begin(), ray_base.end());
  hb->arr.insert(hb->arr.end(), block_base.begin(), block_base.end());
  hb->arr.insert(hb->arr.end(), tile_base.begin(), tile_base.end());
  hb->arr.insert(hb->arr.end(), block_obj.begin(), block_obj.end());
}

BatchDesc desc_from(const HostBatch& hb, const int32_t* dev, ObjectDev* objs) {
  BatchDesc b{};
  b.n = hb.n;
  b.n_blocks = hb.n_blocks;
  b.n_rays = hb.n_rays;
  b.slot = dev;
  b.ray_base = dev + hb.n;
  b.block_base = dev + 2 * hb.n + 1;
  b.tile_base = dev + 3 * hb.n + 2;
  b.block_obj = dev + 4 * hb.n + 3;
  b.objs = objs;
  b.jitter = 1;
  return b;
}

romap_status upload_batch(romap_ctx* ctx, const HostBatch& hb, BatchDesc* out) {
  if (ctx->batch_override) {  // capturing a step graph: its kernels read the graph's own copy of these arrays
    *out = desc_from(hb, ctx->batch_override, ctx->objs_dev);
    return ROMAP_OK;
  }
  size_t bytes = sizeof(int32_t) * hb.arr.size();
  if (ctx->batch_key != hb.arr) {
    ROMAP_TRY(grow(ctx, ctx->ws_batch, bytes));
    CUDA_TRY(cudaMemcpyAsync(ctx->ws_batch.p, hb.arr.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->batch_key = hb.arr;
    ctx->batch_n = hb.n;
  }
  *out = desc_from(hb, (const int32_t*)ctx->ws_batch.p, ctx->objs_dev);
  return ROMAP_OK;
}

romap_status sync_object(romap_ctx* ctx, int slot) {
  const Object& o = ctx->objs[slot];
  ObjectDev& d = ctx->objs_host[slot];
  d.params = o.params;
  d.grad = o.grad;
  d.m = o.m;
  d.v = o.v;
  d.table_h = o.table_h;
  d.pool_o = o.pool_o;
  d.pool_d = o.pool_d;
  d.pool_rgb = o.pool_rgb;
  d.pool_depth = o.pool_depth;
  d.pool_cls = o.pool_cls;
  d.pool_n = o.pool_n;
  d.occ = o.occ;
  for (int a = 0; a < 3; ++a) {
    d.half[a] = o.desc.half_size[a];
    d.inv_ext[a] = 1.0f / (o.desc.half_size[a] - (-o.desc.half_size[a]));
  }
  d.key0 = (uint32_t)o.desc.seed;
  d.key1 = (uint32_t)(o.desc.seed >> 32);
  int64_t B = o.rays_per_step < o.pool_n ? o.rays_per_step : o.pool_n;
  d.n_rays = (int32_t)B;
  d.whole_pool = o.rays_per_step >= o.pool_n ? 1 : 0;
  set_object_step(d, (uint32_t)(o.steps_done + 1), ctx->cfg.beta1, ctx->cfg.beta2);
  d.pad_ = 0;
  d.gfix = o.gfix;
  d.touched = o.touched;
  CUDA_TRY(cudaMemcpyAsync(ctx->objs_dev + slot, &d, sizeof(ObjectDev), cudaMemcpyHostToDevice, ctx->stream));
  return ROMAP_OK;
}

romap_status check_ctx(romap_ctx* ctx) {
  if (!ctx) return fail(ROMAP_ERR_INVALID_ARG, "ctx is NULL");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ROMAP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return ROMAP_OK;
}

romap_status check_id(romap_ctx* ctx, int32_t id) {
  if (id < 0 || id >= (int32_t)ctx->objs.size() || !ctx->objs[id].alive)
    return fail(ROMAP_ERR_NOT_FOUND, "object id %d does not exist", id);
  return ROMAP_OK;
}

romap_status make_grid(const romap_config* c, GridParams* g) {
  if (!c) return fail(ROMAP_ERR_INVALID_ARG, "config is NULL");
  if (c->n_levels < 1 || c->n_levels > kMaxL) return fail(ROMAP_ERR_INVALID_ARG, "n_levels must be in 1..16");
  if (c->n_features != 2) return fail(ROMAP_ERR_UNSUPPORTED, "n_features must be 2");
  if (c->log2_table_size < 8 || c->log2_table_size > 24)
    return fail(ROMAP_ERR_INVALID_ARG, "log2_table_size must be in 8..24");
  if (c->base_resolution < 1) return fail(ROMAP_ERR_INVALID_ARG, "base_resolution must be >= 1");
  if (!(c->growth > 0.0) && (c->max_resolution < c->base_resolution || c->n_levels < 2) && c->n_levels > 1)
    return fail(ROMAP_ERR_INVALID_ARG, "growth <= 0 needs max_resolution >= base_resolution");
  if (c->hidden != kH) return fail(ROMAP_ERR_UNSUPPORTED, "hidden must be 64");
  if (c->dir_dims != 0 && c->dir_dims != 3) return fail(ROMAP_ERR_INVALID_ARG, "dir_dims must be 0 or 3");
  if (c->n_samples < 1 || c->n_samples > 1024) return fail(ROMAP_ERR_INVALID_ARG, "n_samples must be in 1..1024");
  if (c->rays_per_step < 1) return fail(ROMAP_ERR_INVALID_ARG, "rays_per_step must be >= 1");
  if (!(c->lambda1 >= 0.f) || !(c->lambda2 >= 0.f)) return fail(ROMAP_ERR_INVALID_ARG, "loss weights must be >= 0");
  if (!(c->lr > 0.f) || !(c->beta1 >= 0.f && c->beta1 < 1.f) || !(c->beta2 >= 0.f && c->beta2 < 1.f) ||
      !(c->eps >= 0.f))
    return fail(ROMAP_ERR_INVALID_ARG, "invalid Adam hyperparameters");
  if (c->precision != ROMAP_PREC_FP32 && c->precision != ROMAP_PREC_MIXED_BF16 && c->precision != ROMAP_PREC_MIXED_FP8 &&
      c->precision != ROMAP_PREC_MIXED_FP16)
    return fail(ROMAP_ERR_INVALID_ARG, "unknown precision %d", c->precision);
  if (c->accuracy_mode != 0 && c->accuracy_mode != 1) return fail(ROMAP_ERR_INVALID_ARG, "accuracy_mode is 0 or 1");
  if (c->single_net != 0 && c->single_net != 1) return fail(ROMAP_ERR_INVALID_ARG, "single_net is 0 or 1");
  if (c->hidden_layers < 0 || c->hidden_layers > 3)
    return fail(ROMAP_ERR_INVALID_ARG, "hidden_layers must be in 0..3");
  if (c->hidden_layers > 1 && !c->single_net)
    return fail(ROMAP_ERR_UNSUPPORTED, "more than one hidden layer needs the single-network model");
  if (c->reserved != 0) return fail(ROMAP_ERR_INVALID_ARG, "reserved must be 0");
  if (c->deterministic != 0 && c->deterministic != 1) return fail(ROMAP_ERR_INVALID_ARG, "deterministic is 0 or 1");
  if (c->per_object != 0 && c->per_object != 1) return fail(ROMAP_ERR_INVALID_ARG, "per_object is 0 or 1");
  if (c->deterministic && c->precision != ROMAP_PREC_FP32)
    return fail(ROMAP_ERR_UNSUPPORTED, "the deterministic mode is built for ROMAP_PREC_FP32 only");
  if (c->single_net && c->precision == ROMAP_PREC_MIXED_FP8)
    return fail(ROMAP_ERR_UNSUPPORTED, "the single-network model has no 64x64 hidden layer to run in FP8");
  if (c->max_objects < 1 || c->max_objects > 1024) return fail(ROMAP_ERR_INVALID_ARG, "max_objects must be in 1..1024");
  if (c->max_rays_per_object < 1 || c->max_rays_per_object > (int64_t)1 << 31)
    return fail(ROMAP_ERR_INVALID_ARG, "max_rays_per_object must be in 1..2^31");
  if ((c->alloc == nullptr) != (c->dealloc == nullptr))
    return fail(ROMAP_ERR_INVALID_ARG, "alloc and dealloc must be given together");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->bg_const[k])) return fail(ROMAP_ERR_INVALID_ARG, "bg_const must be finite");
  GridParams G{};
  G.L = c->n_levels;
  G.F = 2;
  G.LF = 2 * G.L;
  G.T = 1u << c->log2_table_size;
  double b = c->growth;
  if (!(b > 0.0)) b = G.L > 1 ? std::exp((std::log((double)c->max_resolution) - std::log((double)c->base_resolution)) /
                                         (double)(G.L - 1))
                              : 1.0;
  uint64_t off = 0;
  for (int l = 0; l < G.L; ++l) {
    double r = std::floor((double)c->base_resolution * std::pow(b, (double)l) + 1e-6);
    if (r < 1.0 || r > (double)(1 << 20)) return fail(ROMAP_ERR_INVALID_ARG, "level %d resolution out of range", l);
    G.res[l] = (int)r;
    uint64_t n1 = (uint64_t)G.res[l] + 1;
    uint64_t dense = n1 * n1 * n1;
    G.dense[l] = dense <= (uint64_t)G.T ? 1 : 0;
    G.off[l] = (uint32_t)off;
    off += ((G.dense[l] ? dense : (uint64_t)G.T) + 7u) / 8u * 8u;  // levels start at multiples of 8 entries
    if (off >= ((uint64_t)1 << 31)) return fail(ROMAP_ERR_INVALID_ARG, "hash table too large");
  }
  G.n_hash = (int64_t)off * 2;
  G.dir_dims = c->dir_dims;
  G.cin = kGeo + c->dir_dims;
  G.mlp_off[0] = G.n_hash;
  G.mlp_off[1] = G.mlp_off[0] + (int64_t)kH * G.LF;
  G.mlp_off[2] = G.mlp_off[1] + (int64_t)kDOut * kH;
  G.mlp_off[3] = G.mlp_off[2] + (int64_t)kH * G.cin;
  G.mlp_off[4] = G.mlp_off[3] + (int64_t)kH * kH;
  G.extra = c->single_net && c->hidden_layers > 1 ? c->hidden_layers - 1 : 0;
  G.mlp_off[5] = G.mlp_off[4] + 3 * kH;
  G.mlp_off[6] = G.mlp_off[5] + (int64_t)kH * kH;
  G.n_params = G.mlp_off[5] + (int64_t)G.extra * kH * kH;
  G.n_params_pad = (G.n_params + 3) / 4 * 4;
  G.n_samples = c->n_samples;
  G.lambda1 = c->lambda1;
  G.lambda2 = c->lambda2;
  G.lr = c->lr;
  G.beta1 = c->beta1;
  G.beta2 = c->beta2;
  G.eps = c->eps;
  G.bg_random = c->bg_random ? 1 : 0;
  for (int k = 0; k < 3; ++k) G.bg_const[k] = c->bg_const[k];
  G.accuracy = c->accuracy_mode ? 1 : 0;
  G.fp8 = c->precision == ROMAP_PREC_MIXED_FP8 ? 1 : 0;
  G.f16 = c->precision == ROMAP_PREC_MIXED_FP16 ? 1 : 0;
  G.single_net = c->single_net ? 1 : 0;
  G.det = c->deterministic ? 1 : 0;
  *g = G;
  return ROMAP_OK;
}

void free_object(romap_ctx* ctx, Object& o) {
  dev_free(ctx, o.params);
  dev_free(ctx, o.grad);
  dev_free(ctx, o.m);
  dev_free(ctx, o.v);
  dev_free(ctx, o.table_h);
  dev_free(ctx, o.pool_o);
  dev_free(ctx, o.pool_d);
  dev_free(ctx, o.pool_rgb);
  dev_free(ctx, o.pool_depth);
  dev_free(ctx, o.pool_cls);
  dev_free(ctx, o.occ);
  dev_free(ctx, o.occ_density);
  dev_free(ctx, o.gfix);
  dev_free(ctx, o.touched);
  o = Object{};
}

// Brackets a phase with CUDA events when profiling is on.
struct PhaseScope {
  romap_ctx* ctx;
  romap_ctx::Prof p{};
  bool on;
  PhaseScope(romap_ctx* c, int phase, int launches) : ctx(c), on(c->profiling) {
    if (!on) return;
    p.phase = phase;
    p.launches = launches;
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecord(p.a, ctx->stream);
  }
  ~PhaseScope() {
    if (!on) return;
    cudaEventRecord(p.b, ctx->stream);
    ctx->prof.push_back(p);
  }
};

// Runs the sampling stage for a batch: ray setup, scan, sample write.
romap_status run_sampling(romap_ctx* ctx, const BatchDesc& b, RayBuf R, SampleBuf S, uint32_t* block_sums,
                          BatchDyn* dyn, int32_t* totals, bool count_live) {
  PhaseScope ps(ctx, 0, 3);
  launch_ray_setup(ctx->g, b, R, block_sums, ctx->stream);
  launch_scan(ctx->g, b, block_sums, dyn, totals, S, count_live ? ctx->live_counter : nullptr, ctx->stream);
  launch_write_samples(ctx->g, b, R, block_sums, dyn, S, ctx->stream);
  ctx->launches += 3;
  CUDA_TRY(cudaGetLastError());
  return ROMAP_OK;
}

int tile_ctas(romap_ctx* ctx) { return ctx->n_sms > 0 ? ctx->n_sms : 1; }

// Candidate fused tile kernels of the mixed path (same results, different schedules): the lockstep kernel on tile
// pairs (one CTA per SM) and the warp-specialized kernel (0..7, even and odd indices), then the lockstep kernel on
// single tiles with two CTAs per SM (8..11) and the tile-pair kernel with its two warpgroups decoupled (12..15), each
// with contiguous per-CTA ranges of the tile plan or with the plan dealt round-robin over the CTAs in chunks of 1, 2
// or 4 work items (tile pairs, or tiles).  Only the tile-pair lockstep kernel has the FP8 and single-network
// variants.
typedef void (*TileKernelFn)(const GridParams&, const BatchDesc&, BatchDyn*, RayBuf, int32_t*, int, int,
                             cudaStream_t);
template <void (*F)(const GridParams&, const BatchDesc&, BatchDyn*, RayBuf, int32_t*, int, int, int, cudaStream_t),
          int IL>
void launch_tile_order(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                       int max_tiles, int n_ctas, cudaStream_t stream) {
  F(g, b, dyn, r, status, max_tiles, n_ctas, IL, stream);
}
const TileKernelFn kTileKernels[] = {launch_tile_order<launch_tile_tc, 0>, launch_tile_order<launch_tile_ws, 0>,
                                     launch_tile_order<launch_tile_tc, 1>, launch_tile_order<launch_tile_ws, 1>,
                                     launch_tile_order<launch_tile_tc, 2>, launch_tile_order<launch_tile_ws, 2>,
                                     launch_tile_order<launch_tile_tc, 4>, launch_tile_order<launch_tile_ws, 4>,
                                     launch_tile_order<launch_tile_tc1, 0>, launch_tile_order<launch_tile_tc1, 1>,
                                     launch_tile_order<launch_tile_tc1, 2>, launch_tile_order<launch_tile_tc1, 4>,
                                     launch_tile_order<launch_tile_tcd, 0>, launch_tile_order<launch_tile_tcd, 1>,
                                     launch_tile_order<launch_tile_tcd, 2>, launch_tile_order<launch_tile_tcd, 4>};
const char* const kTileKernelNames[] = {"lockstep tile pairs", "warp-specialized", "lockstep tile pairs, interleaved",
                                        "warp-specialized, interleaved", "lockstep tile pairs, interleaved by 2",
                                        "warp-specialized, interleaved by 2", "lockstep tile pairs, interleaved by 4",
                                        "warp-specialized, interleaved by 4", "lockstep single tiles, 2 CTAs per SM",
                                        "lockstep single tiles, 2 CTAs per SM, interleaved",
                                        "lockstep single tiles, 2 CTAs per SM, interleaved by 2",
                                        "lockstep single tiles, 2 CTAs per SM, interleaved by 4",
                                        "decoupled tile pairs", "decoupled tile pairs, interleaved",
                                        "decoupled tile pairs, interleaved by 2", "decoupled tile pairs, interleaved by 4"};
constexpr int kNumTileKernels = 16;
static_assert(sizeof(kTileKernels) / sizeof(kTileKernels[0]) == kNumTileKernels, "candidate table");
// the candidates with the FP8 and single-network variants (the tile-pair lockstep kernel)
bool lockstep_kernel(int k) { return k < 8 && k % 2 == 0; }

// Sampling stage of the mixed path: ray draw + slab + live counts and masks, the per-object scan (live-sample
// counter, loss reset) with the tile plan, and the placement of every ray in the plan.  Samples are formed inside the
// fused kernel from the masks, so no sample records are written.
romap_status run_sampling_mixed(romap_ctx* ctx, const BatchDesc& b, RayBuf R, SampleBuf S, uint32_t* block_sums,
                                BatchDyn* dyn, int32_t* totals) {
  PhaseScope ps(ctx, 0, 4);
  launch_ray_setup(ctx->g, b, R, block_sums, ctx->stream);
  launch_plan_patterns(b, ctx->stream);
  launch_scan(ctx->g, b, block_sums, dyn, totals, S, ctx->live_counter, ctx->stream);
  launch_plan_rays(ctx->g, b, R, dyn, ctx->stream);
  ctx->launches += 4;
  CUDA_TRY(cudaGetLastError());
  return ROMAP_OK;
}

const std::vector<int32_t>& v_ids_for_tuning(const std::vector<int32_t>& ids) { return ids; }

// Times every candidate tile kernel on this batch (two launches each, CUDA events on the context's stream), keeps
// the fastest, and undoes the candidates' side effects: their gradients are zeroed here, and the caller's sampling
// stage that follows rewrites the ray records and resets the losses.
romap_status autotune_tile_kernel(romap_ctx* ctx, const std::vector<int32_t>& ids, const BatchDesc& b,
                                  int max_tiles) {
  SampleBuf none{};
  ROMAP_TRY(run_sampling_mixed(ctx, b, ctx->R, none, ctx->block_sums, ctx->dyn, ctx->totals));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int best = 0;
  for (int k = 0; k < kNumTileKernels; ++k) {
    if ((ctx->g.fp8 || ctx->g.single_net) && !lockstep_kernel(k)) {  // only the lockstep kernel has these variants
      ctx->tile_kernel_ms[k] = 0.f;
      continue;
    }
    kTileKernels[k](ctx->g, b, ctx->dyn, ctx->R, ctx->status, max_tiles, tile_ctas(ctx), ctx->stream);  // warm
    CUDA_TRY(cudaEventRecord(e0, ctx->stream));
    for (int rep = 0; rep < 2; ++rep)
      kTileKernels[k](ctx->g, b, ctx->dyn, ctx->R, ctx->status, max_tiles, tile_ctas(ctx), ctx->stream);
    CUDA_TRY(cudaEventRecord(e1, ctx->stream));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    ctx->tile_kernel_ms[k] = ms / 2.f;
    if (ctx->tile_kernel_ms[k] < ctx->tile_kernel_ms[best] || ctx->tile_kernel_ms[best] <= 0.f) best = k;
    ctx->launches += 3;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CUDA_TRY(cudaGetLastError());
  for (int32_t id : ids)
    CUDA_TRY(cudaMemsetAsync(ctx->objs[id].grad, 0, sizeof(float) * ctx->g.n_params_pad, ctx->stream));
  CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  ctx->tile_kernel = best;
  return ROMAP_OK;
}

// tile plan bound: per entry at most one partly filled tile per class plus the even padding
// (every tile of the plan holds at least one ray, and each entry adds at most one padding tile)
int64_t plan_max_tiles(const HostBatch& hb) { return (int64_t)hb.n_rays + 2 * (int64_t)hb.n; }

// Grows the step workspace (and the tile plan of the mixed path) to hold one step of a batch with these rays per
// entry.
romap_status ensure_step_workspace(romap_ctx* ctx, const std::vector<int32_t>& rays) {
  HostBatch hb;
  build_batch(std::vector<int32_t>(rays.size(), 0), rays, &hb);
  const bool mixed = ctx->cfg.precision != ROMAP_PREC_FP32;
  int64_t ns = mixed ? 0 : (int64_t)hb.n_rays * ctx->g.n_samples + (int64_t)hb.n * kTile;
  ROMAP_TRY(ensure_workspace(ctx, hb.n_rays, ns, hb.n_blocks, hb.n));
  if (mixed) ROMAP_TRY(ensure_plan(ctx, hb.n_rays, hb.n_blocks, hb.n, plan_max_tiles(hb)));
  return ROMAP_OK;
}

// forward + loss + backward of a batch (no Adam)
// The side stream (lowest priority, so that the sampling kernels it overlaps are scheduled first) and the fork/join
// events, created on first use.
romap_status ensure_side(romap_ctx* ctx) {
  if (ctx->side_stream) return ROMAP_OK;
  int least = 0, greatest = 0;
  CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  CUDA_TRY(cudaStreamCreateWithPriority(&ctx->side_stream, cudaStreamNonBlocking, least));
  CUDA_TRY(cudaStreamCreateWithPriority(&ctx->cap_side, cudaStreamNonBlocking, least));
  CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  ctx->side = ctx->side_stream;
  return ROMAP_OK;
}

// Enqueues the Adam update of the batch's previous step on the side stream after everything on the stream so far.
romap_status fork_prev_adam(romap_ctx* ctx, const BatchDesc& b) {
  ROMAP_TRY(ensure_side(ctx));
  CUDA_TRY(cudaEventRecord(ctx->ev_fork, ctx->stream));
  CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  launch_adam_update(ctx->g, b, ctx->cfg.precision != ROMAP_PREC_FP32, 1, ctx->side);
  CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->side));
  ctx->launches += 1;
  return ROMAP_OK;
}

// overlap_prev_adam: the Adam update of the step before (launch_adam_update with prev) runs on the side stream,
// forked after the batch is uploaded and joined before the first kernel that reads the parameters, so that it
// overlaps this step's sampling (which reads none).
romap_status run_fwd_bwd(romap_ctx* ctx, const std::vector<int32_t>& ids, BatchDesc* out_b,
                         bool overlap_prev_adam = false) {
  std::vector<int32_t> slots(ids.begin(), ids.end()), rays(ids.size());
  for (size_t i = 0; i < ids.size(); ++i) {
    rays[i] = ctx->objs_host[ids[i]].n_rays;
    if (rays[i] < 1) return fail(ROMAP_ERR_BAD_STATE, "object %d has no training rays", ids[i]);
  }
  const bool mixed = ctx->cfg.precision != ROMAP_PREC_FP32;
  HostBatch hb;
  build_batch(slots, rays, &hb);
  ROMAP_TRY(ensure_step_workspace(ctx, rays));
  const int64_t max_tiles = plan_max_tiles(hb);
  BatchDesc b;
  ROMAP_TRY(upload_batch(ctx, hb, &b));
  b.status = ctx->status;
  ctx->last_batch = hb.arr;
  ctx->last_batch_n = hb.n;
  if (mixed) {
    b.plan = 1;
    b.plan_hist = ctx->plan.hist;
    b.plan_bcnt = ctx->plan.bcnt;
    b.plan_pat = ctx->plan.pat;
    b.plan_npat = ctx->plan.npat;
    b.plan_seg = ctx->plan.seg;
    b.plan_nseg = ctx->plan.nseg;
    b.plan_ent = ctx->plan.ent;
    b.plan_perm = ctx->plan.perm;
    b.plan_rstart = ctx->plan.rstart;
    b.plan_slot = ctx->plan.slot;
    b.plan_tiles = ctx->plan.tiles;
    b.plan_npairs = ctx->plan.npairs;
    b.plan_cap_tiles = (int32_t)ctx->cap_plan[3];
    SampleBuf none{};
    if (ctx->tile_kernel < 0) ROMAP_TRY(autotune_tile_kernel(ctx, v_ids_for_tuning(ids), b, (int)max_tiles));
    if (overlap_prev_adam) ROMAP_TRY(fork_prev_adam(ctx, b));
    ROMAP_TRY(run_sampling_mixed(ctx, b, ctx->R, none, ctx->block_sums, ctx->dyn, ctx->totals));
    if (overlap_prev_adam) CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    PhaseScope ps(ctx, 3, 1);
    kTileKernels[ctx->tile_kernel](ctx->g, b, ctx->dyn, ctx->R, ctx->status, (int)max_tiles, tile_ctas(ctx),
                                   ctx->stream);
    ctx->launches += 1;
  } else {
    if (overlap_prev_adam) ROMAP_TRY(fork_prev_adam(ctx, b));
    ROMAP_TRY(run_sampling(ctx, b, ctx->R, ctx->S, ctx->block_sums, ctx->dyn, ctx->totals, true));
    if (overlap_prev_adam) CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    {
      PhaseScope ps(ctx, 1, 1);
      launch_tile_mlp(0, ctx->g, b, ctx->dyn, ctx->totals, ctx->R, ctx->S, tile_ctas(ctx), ctx->stream);
    }
    {
      PhaseScope ps(ctx, 2, 1);
      launch_composite(1, ctx->g, b, ctx->R, ctx->S, ctx->dyn, ctx->status, ctx->stream);
    }
    {
      PhaseScope ps(ctx, 3, ctx->g.det ? 2 : 1);
      launch_tile_mlp(1, ctx->g, b, ctx->dyn, ctx->totals, ctx->R, ctx->S, tile_ctas(ctx), ctx->stream);
      if (ctx->g.det) launch_fix_finish(ctx->g, b, ctx->dyn, ctx->stream);
    }
    ctx->launches += ctx->g.det ? 4 : 3;
  }
  CUDA_TRY(cudaGetLastError());
  ctx->stats.steps += hb.n;
  ctx->stats.rays += hb.n_rays;
  *out_b = b;
  return ROMAP_OK;
}

romap_status validate_ids(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, std::vector<int32_t>* out) {
  if (!ids || n_ids < 1) return fail(ROMAP_ERR_INVALID_ARG, "ids must be a non-empty array");
  if (n_ids > ctx->cfg.max_objects) return fail(ROMAP_ERR_CAPACITY, "more ids than max_objects");
  std::vector<char> seen(ctx->objs.size(), 0);
  out->clear();
  for (int i = 0; i < n_ids; ++i) {
    ROMAP_TRY(check_id(ctx, ids[i]));
    if (seen[ids[i]]) return fail(ROMAP_ERR_INVALID_ARG, "object id %d listed twice", ids[i]);
    seen[ids[i]] = 1;
    out->push_back(ids[i]);
  }
  return ROMAP_OK;
}

// The error a non-zero device status word stands for.
romap_status status_error(int32_t st) {
  if (st & kStatusTimeout) return fail(ROMAP_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", st);
  if (st & kStatusNonfinite) return fail(ROMAP_ERR_NONFINITE, "non-finite loss or gradient (status %d)", st);
  if (st & kStatusBounds)
    return fail(ROMAP_ERR_BOUNDS, "a device index failed its bounds check (status %d)", st);
  if (st & kStatusFixRange)
    return fail(ROMAP_ERR_CAPACITY,
                "a gradient or loss contribution exceeded the deterministic mode's fixed-point range (status %d)", st);
  return fail(ROMAP_ERR_NONFINITE, "non-finite loss (status %d)", st);
}

romap_status read_losses(romap_ctx* ctx, int n, float* out_loss, int per_obj, const std::vector<int32_t>& ids,
                         bool gathered = false) {
  BatchDyn* host = gathered ? ctx->dyn_gather_host : ctx->dyn_host;
  CUDA_TRY(cudaMemcpyAsync(host, gathered ? ctx->dyn_gather : ctx->dyn, sizeof(BatchDyn) * n, cudaMemcpyDeviceToHost,
                           ctx->stream));
  int32_t st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  bool bad = st != 0;
  for (int i = 0; i < n; ++i) {
    float B = (float)ctx->objs_host[ids[i]].n_rays;
    float inv = B > 0 ? 1.0f / B : 0.0f;
    for (int k = 0; k < per_obj; ++k) {
      float v = host[i].loss[k] * inv;
      out_loss[per_obj * i + k] = v;
      if (!std::isfinite(v)) bad = true;
    }
  }
  if (bad) {
    CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
    if (st) return status_error(st);
    return fail(ROMAP_ERR_NONFINITE, "non-finite loss");
  }
  return ROMAP_OK;
}

}  // namespace

extern "C" {

const char* romap_status_string(romap_status s) {
  switch (s) {
    case ROMAP_OK: return "ok";
    case ROMAP_ERR_INVALID_ARG: return "invalid argument";
    case ROMAP_ERR_NOT_FOUND: return "object not found";
    case ROMAP_ERR_OOM: return "out of memory";
    case ROMAP_ERR_CAPACITY: return "capacity exceeded";
    case ROMAP_ERR_CUDA: return "CUDA error";
    case ROMAP_ERR_NONFINITE: return "non-finite value";
    case ROMAP_ERR_TIMEOUT: return "device wait timed out";
    case ROMAP_ERR_BAD_STATE: return "bad state";
    case ROMAP_ERR_UNSUPPORTED: return "unsupported configuration";
    case ROMAP_ERR_BOUNDS: return "device index out of bounds";
    default: return "unknown status";
  }
}

romap_status romap_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return ROMAP_ERR_INVALID_ARG;
  snprintf(buf, n, "%s", g_last_error.c_str());
  return ROMAP_OK;
}

romap_status romap_param_layout(const romap_config* cfg, romap_layout* out) {
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is NULL");
  GridParams g;
  ROMAP_TRY(make_grid(cfg, &g));
  memset(out, 0, sizeof(*out));
  out->n_params = g.n_params;
  out->n_hash_params = g.n_hash;
  out->n_levels = g.L;
  for (int l = 0; l < g.L; ++l) {
    out->resolution[l] = g.res[l];
    out->dense[l] = g.dense[l];
    out->level_offset[l] = g.off[l];
  }
  int rows[7] = {kH, kDOut, kH, kH, 3, kH, kH}, cols[7] = {g.LF, kH, g.cin, kH, kH, kH, kH};
  out->n_mlp_layers = 5 + g.extra;
  for (int i = 0; i < out->n_mlp_layers; ++i) {
    out->mlp_offset[i] = g.mlp_off[i];
    out->mlp_rows[i] = rows[i];
    out->mlp_cols[i] = cols[i];
  }
  return ROMAP_OK;
}

romap_status romap_init(const romap_config* cfg, void* cuda_stream, romap_ctx** out) {
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  GridParams g;
  ROMAP_TRY(make_grid(cfg, &g));
  if (cfg->precision != ROMAP_PREC_FP32 && cfg->n_samples > kTile)
    return fail(ROMAP_ERR_UNSUPPORTED, "mixed precision needs n_samples <= %d", kTile);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  romap_ctx* ctx = new romap_ctx();
  ctx->cfg = *cfg;
  ctx->g = g;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->device = dev;
  ctx->n_sms = prop.multiProcessorCount;
  ctx->objs.resize(cfg->max_objects);
  ctx->objs_host.resize(cfg->max_objects);
  memset(ctx->objs_host.data(), 0, sizeof(ObjectDev) * ctx->objs_host.size());
  romap_status s = dev_alloc_t(ctx, cfg->max_objects, &ctx->objs_dev);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, 1, &ctx->fn_obj_dev);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, 4, &ctx->totals);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, 1, &ctx->status);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, 1, &ctx->live_counter);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, cfg->max_objects, &ctx->dyn_gather);
  if (s == ROMAP_OK && cudaMallocHost((void**)&ctx->dyn_gather_host, sizeof(BatchDyn) * cfg->max_objects) != cudaSuccess)
    s = fail(ROMAP_ERR_OOM, "page-locked allocation of the loss buffer failed");
  if (s == ROMAP_OK) {
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->live_counter, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->objs_dev, 0, sizeof(ObjectDev) * cfg->max_objects, ctx->stream);
    if (e != cudaSuccess) s = fail(ROMAP_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  if (s == ROMAP_OK) s = ensure_workspace(ctx, 1024, 1024 * 8, 8, 8);
  ctx->g.status = ctx->status;  // bounds checks of the checked build report here
  if (s != ROMAP_OK) {
    romap_destroy(ctx);
    return s;
  }
  *out = ctx;
  return ROMAP_OK;
}

static void drop_graph(romap_ctx* ctx);

romap_status romap_destroy(romap_ctx* ctx) {
  if (!ctx) return fail(ROMAP_ERR_INVALID_ARG, "ctx is NULL");
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->cap_side) cudaStreamDestroy(ctx->cap_side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (auto& o : ctx->objs)
    if (o.alive) free_object(ctx, o);
  dev_free(ctx, ctx->objs_dev);
  dev_free(ctx, ctx->fn_obj_dev);
  dev_free(ctx, ctx->totals);
  dev_free(ctx, ctx->status);
  dev_free(ctx, ctx->live_counter);
  dev_free(ctx, ctx->dyn_gather);
  for (DevBuf* b : {&ctx->ws_rays, &ctx->ws_samples, &ctx->ws_blocks, &ctx->ws_batch, &ctx->ws_dyn, &ctx->ws_stage,
                    &ctx->ws_plan, &ctx->ws_mesh, &ctx->ws_mesh_out, &ctx->ws_loss})
    dev_free(ctx, b->p);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->dyn_host) cudaFreeHost(ctx->dyn_host);
  if (ctx->dyn_gather_host) cudaFreeHost(ctx->dyn_gather_host);
  for (auto& p : ctx->prof) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  delete ctx;
  return ROMAP_OK;
}

romap_status romap_create_object(romap_ctx* ctx, const romap_object_desc* d, int32_t* out_id) {
  ROMAP_TRY(check_ctx(ctx));
  if (!d || !out_id) return fail(ROMAP_ERR_INVALID_ARG, "desc and out_id must not be NULL");
  for (int a = 0; a < 3; ++a) {
    if (!(d->half_size[a] > 0.f) || !std::isfinite(d->half_size[a]))
      return fail(ROMAP_ERR_INVALID_ARG, "half_size must be positive and finite");
    if (!std::isfinite(d->t[a])) return fail(ROMAP_ERR_INVALID_ARG, "t must be finite");
  }
  if (!std::isfinite(d->yaw)) return fail(ROMAP_ERR_INVALID_ARG, "yaw must be finite");
  if (d->rays_per_step < 0) return fail(ROMAP_ERR_INVALID_ARG, "rays_per_step must be >= 0");
  int slot = -1;
  for (int i = 0; i < (int)ctx->objs.size(); ++i)
    if (!ctx->objs[i].alive) { slot = i; break; }
  if (slot < 0) return fail(ROMAP_ERR_CAPACITY, "all %d object slots are in use", ctx->cfg.max_objects);
  Object o;
  o.desc = *d;
  o.rays_per_step = d->rays_per_step > 0 ? d->rays_per_step : ctx->cfg.rays_per_step;
  size_t np = (size_t)ctx->g.n_params_pad;
  romap_status s = dev_alloc_t(ctx, np, &o.params);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, np, &o.grad);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, np, &o.m);
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, np, &o.v);
  if (s == ROMAP_OK && ctx->cfg.precision != ROMAP_PREC_FP32)
    s = dev_alloc_t(ctx, (size_t)ctx->g.n_hash + 8, &o.table_h);
  const size_t n_chunks = (np + kAdamChunk - 1) / kAdamChunk;
  if (s == ROMAP_OK) s = dev_alloc_t(ctx, n_chunks, &o.touched);
  if (s == ROMAP_OK && ctx->g.det) s = dev_alloc_t(ctx, np, &o.gfix);
  if (s != ROMAP_OK) {
    o.alive = true;
    free_object(ctx, o);
    return s;
  }
  cudaMemsetAsync(o.grad, 0, np * sizeof(float), ctx->stream);
  cudaMemsetAsync(o.m, 0, np * sizeof(float), ctx->stream);
  cudaMemsetAsync(o.v, 0, np * sizeof(float), ctx->stream);
  cudaMemsetAsync(o.touched, 0, n_chunks, ctx->stream);
  if (o.gfix) cudaMemsetAsync(o.gfix, 0, np * sizeof(unsigned long long), ctx->stream);
  launch_init_params(ctx->g, o.params, (uint32_t)d->seed, (uint32_t)(d->seed >> 32), ctx->stream);
  ctx->launches += 1;
  if (o.table_h) {
    launch_to_half(o.params, o.table_h, ctx->g.n_hash, ctx->stream);
    ctx->launches += 1;
  }
  CUDA_TRY(cudaGetLastError());
  o.alive = true;
  ctx->objs[slot] = o;
  ROMAP_TRY(sync_object(ctx, slot));
  *out_id = slot;
  return ROMAP_OK;
}

romap_status romap_destroy_object(romap_ctx* ctx, int32_t id) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  free_object(ctx, ctx->objs[id]);
  memset(&ctx->objs_host[id], 0, sizeof(ObjectDev));
  CUDA_TRY(cudaMemsetAsync(ctx->objs_dev + id, 0, sizeof(ObjectDev), ctx->stream));
  return ROMAP_OK;
}

romap_status romap_set_occupancy(romap_ctx* ctx, int32_t id, const uint64_t* bits, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  Object& o = ctx->objs[id];
  if (!bits) {
    dev_free(ctx, o.occ);
    o.occ = nullptr;
    return sync_object(ctx, id);
  }
  if (!o.occ) ROMAP_TRY(dev_alloc_t(ctx, 4096, &o.occ));
  CUDA_TRY(cudaMemcpyAsync(o.occ, bits, 4096 * sizeof(uint64_t),
                           (flags & ROMAP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           ctx->stream));
  return sync_object(ctx, id);
}

romap_status romap_update_occupancy(romap_ctx* ctx, int32_t id, float decay, float threshold, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!(decay >= 0.f && decay <= 1.f)) return fail(ROMAP_ERR_INVALID_ARG, "decay must be in [0, 1]");
  if (!(threshold >= 0.f) || !std::isfinite(threshold))
    return fail(ROMAP_ERR_INVALID_ARG, "threshold must be finite and >= 0");
  if (flags & ~ROMAP_REPLACE) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  Object& o = ctx->objs[id];
  bool fresh = false;
  if (!o.occ_density) {
    ROMAP_TRY(dev_alloc_t(ctx, (size_t)64 * 64 * 64, &o.occ_density));
    fresh = true;
  }
  if (!o.occ) ROMAP_TRY(dev_alloc_t(ctx, 4096, &o.occ));
  ROMAP_TRY(sync_object(ctx, id));
  launch_occ_update(ctx->g, ctx->objs_dev, id, decay, threshold, (fresh || (flags & ROMAP_REPLACE)) ? 1 : 0,
                    o.occ_density, o.occ, ctx->stream);
  ctx->launches += 1;
  CUDA_TRY(cudaGetLastError());
  return ROMAP_OK;
}

romap_status romap_get_occupancy(romap_ctx* ctx, int32_t id, uint64_t* bits, float* density) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  const Object& o = ctx->objs[id];
  if (bits && !o.occ) return fail(ROMAP_ERR_BAD_STATE, "object %d has no occupancy grid", id);
  if (density && !o.occ_density) return fail(ROMAP_ERR_BAD_STATE, "object %d has no occupancy densities", id);
  if (bits) CUDA_TRY(cudaMemcpyAsync(bits, o.occ, 4096 * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  if (density)
    CUDA_TRY(cudaMemcpyAsync(density, o.occ_density, sizeof(float) * 64 * 64 * 64, cudaMemcpyDeviceToHost,
                             ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

// ---- mesh extraction (Table 3: marching cubes, 64^3) ----------------------------------------------------------------
namespace {
int8_t g_mc_tri[256][3 * kMcMaxTri + 1];
uint8_t g_mc_cnt[256];
std::once_flag g_mc_once;
int g_mc_built = -1;

romap_status mesh_workspace(romap_ctx* ctx, char** ws, uint32_t** totals) {
  std::call_once(g_mc_once, [] { g_mc_built = build_mc_table(g_mc_tri, g_mc_cnt); });
  if (g_mc_built < 0) return fail(ROMAP_ERR_BAD_STATE, "marching-cubes table construction failed");
  const size_t bytes = mc_workspace_bytes();
  if (ctx->ws_mesh.bytes < bytes) ROMAP_TRY(grow(ctx, ctx->ws_mesh, bytes));
  *ws = (char*)ctx->ws_mesh.p;
  *totals = (uint32_t*)((char*)ctx->ws_mesh.p + bytes - 8 * 256);
  return ROMAP_OK;
}
}  // namespace

romap_status romap_density_lattice(romap_ctx* ctx, int32_t id, float* out, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is required");
  if (flags & ~ROMAP_DEVICE_PTR) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  char* ws;
  uint32_t* totals;
  ROMAP_TRY(mesh_workspace(ctx, &ws, &totals));
  launch_lattice_density(ctx->g, ctx->objs_dev, id, (float*)ws, ctx->stream);
  ctx->launches += 1;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(out, ws, sizeof(float) * mc_lattice_points(),
                           (flags & ROMAP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           ctx->stream));
  if (!(flags & ROMAP_DEVICE_PTR)) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

romap_status romap_extract_mesh(romap_ctx* ctx, int32_t id, float iso, float* vertices, int64_t max_vertices,
                                int32_t* triangles, int64_t max_triangles, int64_t* out_n_vertices,
                                int64_t* out_n_triangles, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!std::isfinite(iso)) return fail(ROMAP_ERR_INVALID_ARG, "iso must be finite");
  if (max_vertices < 0 || max_triangles < 0) return fail(ROMAP_ERR_INVALID_ARG, "negative capacity");
  if ((max_vertices > 0 && !vertices) || (max_triangles > 0 && !triangles))
    return fail(ROMAP_ERR_INVALID_ARG, "NULL output with a non-zero capacity");
  if (flags & ~ROMAP_DEVICE_PTR) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  char* ws;
  uint32_t* totals;
  ROMAP_TRY(mesh_workspace(ctx, &ws, &totals));
  ctx->launches += launch_mc(ctx->g, ctx->objs_dev, id, iso, ws, 0, 0, nullptr, 0, nullptr, totals, &g_mc_tri[0][0],
                             g_mc_cnt, ctx->stream);
  CUDA_TRY(cudaGetLastError());
  uint32_t nvt[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(nvt, totals, sizeof(nvt), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (out_n_vertices) *out_n_vertices = nvt[0];
  if (out_n_triangles) *out_n_triangles = nvt[1];
  if ((int64_t)nvt[0] > max_vertices || (int64_t)nvt[1] > max_triangles)
    return fail(ROMAP_ERR_CAPACITY, "mesh has %u vertices and %u triangles", nvt[0], nvt[1]);
  if (nvt[0] == 0) return ROMAP_OK;
  const bool dev = flags & ROMAP_DEVICE_PTR;
  float* v = vertices;
  int32_t* t = triangles;
  if (!dev) {
    const size_t bytes = 12 * (size_t)nvt[0] + 12 * (size_t)nvt[1] + 256;
    if (ctx->ws_mesh_out.bytes < bytes) ROMAP_TRY(grow(ctx, ctx->ws_mesh_out, bytes));
    v = (float*)ctx->ws_mesh_out.p;
    t = (int32_t*)((char*)ctx->ws_mesh_out.p + ((12 * (size_t)nvt[0] + 255) / 256) * 256);
  }
  ctx->launches += launch_mc(ctx->g, ctx->objs_dev, id, iso, ws, 1, nvt[0], v, nvt[1], t, totals, nullptr, nullptr,
                             ctx->stream);
  CUDA_TRY(cudaGetLastError());
  if (!dev) {
    CUDA_TRY(cudaMemcpyAsync(vertices, v, 12 * (size_t)nvt[0], cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(triangles, t, 12 * (size_t)nvt[1], cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return ROMAP_OK;
}

namespace {

bool finite_bits(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return (b & 0x7f800000u) != 0x7f800000u;
}

// Host ray arrays (n rays): origin, direction and colour finite, depth not infinite (NaN = none), class 0..2,
// direction of non-zero length.  The first pass is branch-free so that the compiler vectorises it; the loop that
// names the first bad ray runs only when the first pass found one.
romap_status check_host_rays(const romap_rays* r, int64_t n) {
  uint32_t bad = 0;
  for (int64_t i = 0; i < 3 * n; ++i)
    bad |= (uint32_t)!finite_bits(r->origin[i]) | (uint32_t)!finite_bits(r->dir[i]) | (uint32_t)!finite_bits(r->rgb[i]);
  if (r->depth)
    for (int64_t i = 0; i < n; ++i) {
      uint32_t b;
      std::memcpy(&b, r->depth + i, 4);
      bad |= (uint32_t)((b & 0x7fffffffu) == 0x7f800000u);
    }
  if (r->cls)
    for (int64_t i = 0; i < n; ++i) bad |= (uint32_t)(r->cls[i] > 2);
  for (int64_t i = 0; i < n; ++i) {
    const float* d = r->dir + 3 * i;
    bad |= (uint32_t)!(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] > 0.f);
  }
  if (!bad) return ROMAP_OK;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(r->origin[i]) || !std::isfinite(r->dir[i]) || !std::isfinite(r->rgb[i]))
      return fail(ROMAP_ERR_NONFINITE, "non-finite origin, dir or rgb at ray %lld", (long long)(i / 3));
  for (int64_t i = 0; i < n; ++i) {
    if (r->depth && std::isinf(r->depth[i])) return fail(ROMAP_ERR_NONFINITE, "infinite depth at ray %lld", (long long)i);
    if (r->cls && r->cls[i] > 2) return fail(ROMAP_ERR_INVALID_ARG, "class %d at ray %lld", r->cls[i], (long long)i);
    float dd = r->dir[3 * i] * r->dir[3 * i] + r->dir[3 * i + 1] * r->dir[3 * i + 1] + r->dir[3 * i + 2] * r->dir[3 * i + 2];
    if (!(dd > 0.f)) return fail(ROMAP_ERR_INVALID_ARG, "zero direction at ray %lld", (long long)i);
  }
  return ROMAP_OK;
}

// Grows the object's pool so that it holds `need` rays, keeping its first `keep` rays.
romap_status ensure_pool(romap_ctx* ctx, Object& o, int64_t keep, int64_t need) {
  if (need <= o.pool_cap) return ROMAP_OK;
  int64_t cap = need > 2 * o.pool_cap ? need : 2 * o.pool_cap;
  if (cap > ctx->cfg.max_rays_per_object) cap = ctx->cfg.max_rays_per_object;
  float *po, *pd, *prgb, *pdep;
  uint8_t* pcls;
  ROMAP_TRY(dev_alloc_t(ctx, 3 * cap, &po));
  ROMAP_TRY(dev_alloc_t(ctx, 3 * cap, &pd));
  ROMAP_TRY(dev_alloc_t(ctx, 3 * cap, &prgb));
  ROMAP_TRY(dev_alloc_t(ctx, cap, &pdep));
  ROMAP_TRY(dev_alloc_t(ctx, cap, &pcls));
  if (keep > 0) {
    CUDA_TRY(cudaMemcpyAsync(po, o.pool_o, 12 * keep, cudaMemcpyDeviceToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(pd, o.pool_d, 12 * keep, cudaMemcpyDeviceToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(prgb, o.pool_rgb, 12 * keep, cudaMemcpyDeviceToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(pdep, o.pool_depth, 4 * keep, cudaMemcpyDeviceToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(pcls, o.pool_cls, keep, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  dev_free(ctx, o.pool_o); dev_free(ctx, o.pool_d); dev_free(ctx, o.pool_rgb);
  dev_free(ctx, o.pool_depth); dev_free(ctx, o.pool_cls);
  o.pool_o = po; o.pool_d = pd; o.pool_rgb = prgb; o.pool_depth = pdep; o.pool_cls = pcls;
  o.pool_cap = cap;
  return ROMAP_OK;
}

// Input arrays of an append on the device: host arrays are copied into the staging buffer (followed by `extra`
// bytes for the caller), device arrays are used in place (the staging buffer then holds only the extra bytes).
struct StagedRays {
  const float *o = nullptr, *d = nullptr, *rgb = nullptr, *depth = nullptr;
  const uint8_t* cls = nullptr;
  char* extra = nullptr;
  bool pinned = false;  // host arrays in page-locked memory: copied asynchronously, so the call waits for them
};
romap_status stage_rays(romap_ctx* ctx, const romap_rays* r, int64_t n, bool dev, size_t extra, StagedRays* out) {
  *out = StagedRays{};
  out->o = r->origin; out->d = r->dir; out->rgb = r->rgb; out->depth = r->depth; out->cls = r->cls;
  if (dev) {
    if (extra) {
      ROMAP_TRY(grow(ctx, ctx->ws_stage, extra));
      out->extra = (char*)ctx->ws_stage.p;
    }
    return ROMAP_OK;
  }
  size_t b3 = align_up(12 * (size_t)n, 256), b1 = align_up(4 * (size_t)n, 256), bc = align_up((size_t)n, 256);
  ROMAP_TRY(grow(ctx, ctx->ws_stage, 3 * b3 + b1 + bc + extra));
  char* st = (char*)ctx->ws_stage.p;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, r->origin) == cudaSuccess && attr.type == cudaMemoryTypeHost) out->pinned = true;
  cudaGetLastError();
  CUDA_TRY(cudaMemcpyAsync(st, r->origin, 12 * n, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(st + b3, r->dir, 12 * n, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(st + 2 * b3, r->rgb, 12 * n, cudaMemcpyHostToDevice, ctx->stream));
  out->o = (const float*)st;
  out->d = (const float*)(st + b3);
  out->rgb = (const float*)(st + 2 * b3);
  if (r->depth) {
    CUDA_TRY(cudaMemcpyAsync(st + 3 * b3, r->depth, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    out->depth = (const float*)(st + 3 * b3);
  }
  if (r->cls) {
    CUDA_TRY(cudaMemcpyAsync(st + 3 * b3 + b1, r->cls, n, cudaMemcpyHostToDevice, ctx->stream));
    out->cls = (const uint8_t*)(st + 3 * b3 + b1);
  }
  out->extra = st + 3 * b3 + b1 + bc;
  return ROMAP_OK;
}

}  // namespace

romap_status romap_add_rays(romap_ctx* ctx, int32_t id, const romap_rays* r, int64_t n, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!r || n < 0) return fail(ROMAP_ERR_INVALID_ARG, "rays must not be NULL and n >= 0");
  if (n > 0 && (!r->origin || !r->dir || !r->rgb)) return fail(ROMAP_ERR_INVALID_ARG, "origin, dir and rgb are required");
  if (flags & ~(ROMAP_DEVICE_PTR | ROMAP_OBJECT_FRAME | ROMAP_REPLACE | ROMAP_ASYNC_HOST))
    return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  Object& o = ctx->objs[id];
  bool dev = (flags & ROMAP_DEVICE_PTR) != 0;
  int64_t start = (flags & ROMAP_REPLACE) ? 0 : o.pool_n;
  int64_t need = start + n;
  if (need > ctx->cfg.max_rays_per_object)
    return fail(ROMAP_ERR_CAPACITY, "pool of object %d would hold %lld rays (max %lld)", id, (long long)need,
                (long long)ctx->cfg.max_rays_per_object);
  if (!dev) ROMAP_TRY(check_host_rays(r, n));
  if (n == 0) {
    if (flags & ROMAP_REPLACE) {
      o.pool_n = 0;
      return sync_object(ctx, id);
    }
    return ROMAP_OK;
  }
  ROMAP_TRY(ensure_pool(ctx, o, start, need));
  StagedRays sr;
  ROMAP_TRY(stage_rays(ctx, r, n, dev, 0, &sr));
  float cz = (float)std::cos(o.desc.yaw), sz = (float)std::sin(o.desc.yaw);
  launch_transform_rays(sr.o, sr.d, sr.rgb, sr.depth, sr.cls, n, (flags & ROMAP_OBJECT_FRAME) ? 1 : 0, o.desc.t[0],
                        o.desc.t[1], o.desc.t[2], cz, sz, o.pool_o + 3 * start, o.pool_d + 3 * start,
                        o.pool_rgb + 3 * start, o.pool_depth + start, o.pool_cls + start, ctx->stream);
  ctx->launches += 1;
  CUDA_TRY(cudaGetLastError());
  // page-locked host buffers are read asynchronously: wait for them unless the caller keeps them (ROMAP_ASYNC_HOST)
  if (sr.pinned && !(flags & ROMAP_ASYNC_HOST)) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  o.pool_n = need;
  return sync_object(ctx, id);
}

romap_status romap_add_rays_multi(romap_ctx* ctx, const int32_t* ids, const int64_t* counts, int32_t n_ids,
                                  const romap_rays* r, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  std::vector<int32_t> v;
  ROMAP_TRY(validate_ids(ctx, ids, n_ids, &v));
  if (!counts || !r) return fail(ROMAP_ERR_INVALID_ARG, "counts and rays must not be NULL");
  if (flags & ~(ROMAP_DEVICE_PTR | ROMAP_OBJECT_FRAME | ROMAP_REPLACE | ROMAP_ASYNC_HOST))
    return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  const bool dev = (flags & ROMAP_DEVICE_PTR) != 0, replace = (flags & ROMAP_REPLACE) != 0;
  int64_t n = 0;
  for (int k = 0; k < n_ids; ++k) {
    if (counts[k] < 0) return fail(ROMAP_ERR_INVALID_ARG, "counts[%d] = %lld < 0", k, (long long)counts[k]);
    const int64_t need = (replace ? 0 : ctx->objs[ids[k]].pool_n) + counts[k];
    if (need > ctx->cfg.max_rays_per_object)
      return fail(ROMAP_ERR_CAPACITY, "pool of object %d would hold %lld rays (max %lld)", ids[k], (long long)need,
                  (long long)ctx->cfg.max_rays_per_object);
    n += counts[k];
  }
  if (n > 0 && (!r->origin || !r->dir || !r->rgb)) return fail(ROMAP_ERR_INVALID_ARG, "origin, dir and rgb are required");
  if (!dev) ROMAP_TRY(check_host_rays(r, n));
  std::vector<XformObj> xo;
  int64_t first = 0;
  for (int k = 0; k < n_ids; ++k) {
    Object& o = ctx->objs[ids[k]];
    const int64_t start = replace ? 0 : o.pool_n;
    if (counts[k] > 0) {
      ROMAP_TRY(ensure_pool(ctx, o, start, start + counts[k]));
      XformObj x;
      x.first = first;
      for (int a = 0; a < 3; ++a) x.t[a] = o.desc.t[a];
      x.cz = (float)std::cos(o.desc.yaw);
      x.sz = (float)std::sin(o.desc.yaw);
      x.o_out = o.pool_o + 3 * start;
      x.d_out = o.pool_d + 3 * start;
      x.rgb_out = o.pool_rgb + 3 * start;
      x.depth_out = o.pool_depth + start;
      x.cls_out = o.pool_cls + start;
      xo.push_back(x);
    }
    first += counts[k];
  }
  bool pinned = false;
  if (!xo.empty()) {
    StagedRays sr;
    ROMAP_TRY(stage_rays(ctx, r, n, dev, sizeof(XformObj) * xo.size(), &sr));
    CUDA_TRY(cudaMemcpyAsync(sr.extra, xo.data(), sizeof(XformObj) * xo.size(), cudaMemcpyHostToDevice, ctx->stream));
    launch_transform_rays_multi(sr.o, sr.d, sr.rgb, sr.depth, sr.cls, n, (flags & ROMAP_OBJECT_FRAME) ? 1 : 0,
                                reinterpret_cast<const XformObj*>(sr.extra), (int)xo.size(), ctx->stream);
    ctx->launches += 1;
    CUDA_TRY(cudaGetLastError());
    pinned = sr.pinned;
  }
  // page-locked host buffers are read asynchronously: wait for them unless the caller keeps them (ROMAP_ASYNC_HOST)
  if (pinned && !(flags & ROMAP_ASYNC_HOST)) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < n_ids; ++k) {
    Object& o = ctx->objs[ids[k]];
    o.pool_n = (replace ? 0 : o.pool_n) + counts[k];
    ROMAP_TRY(sync_object(ctx, ids[k]));
  }
  return ROMAP_OK;
}

romap_status romap_pool_size(romap_ctx* ctx, int32_t id, int64_t* out_n) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!out_n) return fail(ROMAP_ERR_INVALID_ARG, "out_n is NULL");
  *out_n = ctx->objs[id].pool_n;
  return ROMAP_OK;
}

romap_status romap_forward_backward(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, float* out_loss) {
  ROMAP_TRY(check_ctx(ctx));
  std::vector<int32_t> v;
  ROMAP_TRY(validate_ids(ctx, ids, n_ids, &v));
  BatchDesc b;
  ROMAP_TRY(run_fwd_bwd(ctx, v, &b));
  if (out_loss) ROMAP_TRY(read_losses(ctx, n_ids, out_loss, 5, v));
  return ROMAP_OK;
}

romap_status romap_adam_step(romap_ctx* ctx, const int32_t* ids, int32_t n_ids) {
  ROMAP_TRY(check_ctx(ctx));
  std::vector<int32_t> v;
  ROMAP_TRY(validate_ids(ctx, ids, n_ids, &v));
  std::vector<int32_t> rays(v.size(), 0);
  HostBatch hb;
  build_batch(v, rays, &hb);
  BatchDesc b;
  ROMAP_TRY(upload_batch(ctx, hb, &b));
  {
    PhaseScope ps(ctx, 4, 2);
    launch_adam(ctx->g, b, ctx->cfg.precision != ROMAP_PREC_FP32, ctx->stream);
  }
  ctx->launches += 2;
  CUDA_TRY(cudaGetLastError());
  for (int32_t id : v) {
    ctx->objs[id].steps_done += 1;
    set_object_step(ctx->objs_host[id], (uint32_t)(ctx->objs[id].steps_done + 1), ctx->cfg.beta1, ctx->cfg.beta2);
  }
  return ROMAP_OK;
}

// One training step (forward, loss, backward, Adam) of a batch on ctx->stream.
static romap_status enqueue_step(romap_ctx* ctx, const std::vector<int32_t>& v) {
  BatchDesc b;
  ROMAP_TRY(run_fwd_bwd(ctx, v, &b));
  {
    PhaseScope ps(ctx, 4, 2);
    launch_adam(ctx->g, b, ctx->cfg.precision != ROMAP_PREC_FP32, ctx->stream);
  }
  ctx->launches += 2;
  CUDA_TRY(cudaGetLastError());
  for (int32_t id : v) {
    ctx->objs[id].steps_done += 1;
    set_object_step(ctx->objs_host[id], (uint32_t)(ctx->objs[id].steps_done + 1), ctx->cfg.beta1, ctx->cfg.beta2);
  }
  return ROMAP_OK;
}

// Pieces of a pipelined run of n_steps > 1 steps of one batch in one call: kind 1, the first step without its Adam
// update; kind 2, a step whose sampling overlaps the previous step's Adam update; kind 3, the last step's update.
// Kind 0 is a whole step (enqueue_step).  The parameters after kinds 1, 2 x (n - 1), 3 are those after n whole
// steps, bit for bit: the sampling reads no parameter, and the update of a step uses that step's bias corrections.
static romap_status enqueue_kind(romap_ctx* ctx, const std::vector<int32_t>& v, int kind) {
  if (kind == 0) return enqueue_step(ctx, v);
  if (kind == 3) {
    std::vector<int32_t> rays(v.size());
    for (size_t i = 0; i < v.size(); ++i) rays[i] = ctx->objs_host[v[i]].n_rays;
    HostBatch hb;
    build_batch(v, rays, &hb);
    BatchDesc b;
    ROMAP_TRY(upload_batch(ctx, hb, &b));
    launch_adam_update(ctx->g, b, ctx->cfg.precision != ROMAP_PREC_FP32, 1, ctx->stream);
    ctx->launches += 1;
    CUDA_TRY(cudaGetLastError());
    return ROMAP_OK;
  }
  BatchDesc b;
  ROMAP_TRY(run_fwd_bwd(ctx, v, &b, kind == 2));
  launch_advance_step(ctx->g, b, ctx->stream);
  ctx->launches += 1;
  CUDA_TRY(cudaGetLastError());
  for (int32_t id : v) {
    ctx->objs[id].steps_done += 1;
    set_object_step(ctx->objs_host[id], (uint32_t)(ctx->objs[id].steps_done + 1), ctx->cfg.beta1, ctx->cfg.beta2);
  }
  return ROMAP_OK;
}

constexpr int kMaxStepGraphs = 128;

static void free_graph(romap_ctx* ctx, romap_ctx::StepGraph& sg) {
  if (sg.exec) cudaGraphExecDestroy(sg.exec);
  dev_free(ctx, sg.batch_dev);
  sg = romap_ctx::StepGraph{};
}

// Drops every cached step graph.
static void drop_graph(romap_ctx* ctx) {
  for (auto& sg : ctx->graphs) free_graph(ctx, sg);
  ctx->graphs.clear();
}

// The cached graph of composition `key`, or null.  Graphs captured before a workspace buffer moved are dropped
// (their kernels hold the old addresses).
static romap_ctx::StepGraph* find_graph(romap_ctx* ctx, const std::vector<int32_t>& key) {
  for (size_t i = 0; i < ctx->graphs.size();) {
    if (ctx->graphs[i].ws_generation != ctx->ws_generation) {
      free_graph(ctx, ctx->graphs[i]);
      ctx->graphs.erase(ctx->graphs.begin() + (ptrdiff_t)i);
    } else {
      ++i;
    }
  }
  for (auto& sg : ctx->graphs)
    if (sg.key == key) return &sg;
  return nullptr;
}

// Captures one step of batch v (nothing executes during capture) into a new cache entry, evicting the least recently
// used entry when the cache is full.  The graph reads its batch arrays from its own device copy, so graphs of
// different compositions replay in any order without re-uploading anything.
static romap_status capture_step(romap_ctx* ctx, const std::vector<int32_t>& v, const std::vector<int32_t>& key,
                                 int kind = 0) {
  if (!ctx->cap_stream) {  // the highest priority: a captured step's sampling goes ahead of the overlapping update
    int least = 0, greatest = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CUDA_TRY(cudaStreamCreateWithPriority(&ctx->cap_stream, cudaStreamNonBlocking, greatest));
  }
  if ((int)ctx->graphs.size() >= kMaxStepGraphs) {
    size_t lru = 0;
    for (size_t i = 1; i < ctx->graphs.size(); ++i)
      if (ctx->graphs[i].last_use < ctx->graphs[lru].last_use) lru = i;
    free_graph(ctx, ctx->graphs[lru]);
    ctx->graphs.erase(ctx->graphs.begin() + (ptrdiff_t)lru);
  }
  romap_ctx::StepGraph sg;
  sg.key = key;
  sg.batch = ctx->last_batch;  // the eager step that just ran had this composition
  sg.batch_n = ctx->last_batch_n;
  ROMAP_TRY(dev_alloc_t(ctx, sg.batch.size(), &sg.batch_dev));
  CUDA_TRY(cudaMemcpyAsync(sg.batch_dev, sg.batch.data(), sizeof(int32_t) * sg.batch.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
  // the copy above is pageable: wait for it so that the host vector may change while the graph lives
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  // the capture records launches only; host-side counters are restored afterwards and advanced per replay
  std::vector<int64_t> done(v.size());
  for (size_t i = 0; i < v.size(); ++i) done[i] = ctx->objs[v[i]].steps_done;
  romap_stats saved = ctx->stats;
  int64_t saved_launches = ctx->launches;
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap_stream;
  if (kind == 2) {  // the fork joins the capture through the events
    ROMAP_TRY(ensure_side(ctx));
    ctx->side = ctx->cap_side;
  }
  ctx->batch_override = sg.batch_dev;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  romap_status st = ROMAP_OK;
  if (e == cudaSuccess) {
    st = enqueue_kind(ctx, v, kind);
    e = cudaStreamEndCapture(ctx->cap_stream, &graph);
  }
  ctx->batch_override = nullptr;
  ctx->stream = user;
  if (ctx->side_stream) ctx->side = ctx->side_stream;
  for (size_t i = 0; i < v.size(); ++i) {
    ctx->objs[v[i]].steps_done = done[i];
    set_object_step(ctx->objs_host[v[i]], (uint32_t)(done[i] + 1), ctx->cfg.beta1, ctx->cfg.beta2);
  }
  sg.launches = (int)(ctx->launches - saved_launches);
  ctx->stats = saved;
  ctx->launches = saved_launches;
  if (e == cudaSuccess && st == ROMAP_OK && graph) {
    e = cudaGraphInstantiate(&sg.exec, graph, 0);
    if (e != cudaSuccess) sg.exec = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || st != ROMAP_OK || !sg.exec) {
    cudaGetLastError();
    free_graph(ctx, sg);
    ctx->graphs_enabled = false;  // fall back to eager launches for the rest of the context
    return ROMAP_OK;
  }
  sg.last_use = ++ctx->graph_clock;
  sg.ws_generation = ctx->ws_generation;
  ctx->graph_captures += 1;
  ctx->graphs.push_back(std::move(sg));
  return ROMAP_OK;
}

namespace {

// n_steps training steps of the validated batch v (CUDA-graph replay once captured), all enqueued on the stream
romap_status run_train_steps(romap_ctx* ctx, const std::vector<int32_t>& v, int32_t n_steps) {
  // size the workspace for this batch and for the largest single live object up front, so that alternating
  // single-object compositions (the per-object path) do not move it and invalidate each other's graphs
  {
    std::vector<int32_t> rays;
    for (int32_t id : v) rays.push_back(ctx->objs_host[id].n_rays);
    ROMAP_TRY(ensure_step_workspace(ctx, rays));
    int32_t largest = 0;
    for (size_t i = 0; i < ctx->objs.size(); ++i)
      if (ctx->objs[i].alive) largest = std::max(largest, ctx->objs_host[i].n_rays);
    if (largest > 0) ROMAP_TRY(ensure_step_workspace(ctx, std::vector<int32_t>{largest}));
  }
  // the graph key: the batch composition (object slots and their rays per step), the precision and the kind of piece
  std::vector<int32_t> key(v.begin(), v.end());
  for (int32_t id : v) key.push_back(ctx->objs_host[id].n_rays);
  key.push_back(ctx->cfg.precision);
  // n_steps > 1: each step's sampling overlaps the previous step's Adam update (kinds 1, 2 ..., 3; enqueue_kind)
  const bool pipelined = n_steps > 1 && !ctx->profiling;
  auto run_piece = [&](int kind) -> romap_status {
    std::vector<int32_t> k = key;
    k.push_back(kind);
    const bool use_graph = ctx->graphs_enabled && !ctx->profiling;
    romap_ctx::StepGraph* sg = use_graph ? find_graph(ctx, k) : nullptr;
    if (sg) {
      CUDA_TRY(cudaGraphLaunch(sg->exec, ctx->stream));
      sg->last_use = ++ctx->graph_clock;
      ctx->graph_replays += 1;
      ctx->launches += sg->launches;
      if (kind == 3) return ROMAP_OK;
      ctx->last_batch = sg->batch;
      ctx->last_batch_n = sg->batch_n;
      // what enqueue_step does on the host for each step
      int64_t rays = 0;
      for (int32_t id : v) {
        rays += ctx->objs_host[id].n_rays;
        ctx->objs[id].steps_done += 1;
        set_object_step(ctx->objs_host[id], (uint32_t)(ctx->objs[id].steps_done + 1), ctx->cfg.beta1, ctx->cfg.beta2);
      }
      ctx->stats.steps += (int64_t)v.size();
      ctx->stats.rays += rays;
      return ROMAP_OK;
    }
    ROMAP_TRY(enqueue_kind(ctx, v, kind));
    if (use_graph) ROMAP_TRY(capture_step(ctx, v, k, kind));
    return ROMAP_OK;
  };
  for (int s = 0; s < n_steps; ++s) ROMAP_TRY(run_piece(pipelined ? (s == 0 ? 1 : 2) : 0));
  if (pipelined) ROMAP_TRY(run_piece(3));
  return ROMAP_OK;
}

// Steps of the listed objects: one batched launch sequence per step, or with per_object one sequence per object
// (each object's steps back to back).  per_object: losses (5 floats per object) of each object's last step are
// copied to dyn_host[k] on the stream as the object finishes, since every single-object step reuses dyn[0].
romap_status run_listed_steps(romap_ctx* ctx, const std::vector<int32_t>& v, int32_t n_steps, bool gather_losses) {
  if (!ctx->cfg.per_object) return run_train_steps(ctx, v, n_steps);
  for (size_t k = 0; k < v.size(); ++k) {
    ROMAP_TRY(run_train_steps(ctx, std::vector<int32_t>{v[k]}, n_steps));
    if (gather_losses)
      CUDA_TRY(cudaMemcpyAsync(ctx->dyn_gather + k, ctx->dyn, sizeof(BatchDyn), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return ROMAP_OK;
}

}  // namespace

romap_status romap_train_step(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, int32_t n_steps, float* out_loss) {
  ROMAP_TRY(check_ctx(ctx));
  if (n_steps < 1) return fail(ROMAP_ERR_INVALID_ARG, "n_steps must be >= 1");
  std::vector<int32_t> v;
  ROMAP_TRY(validate_ids(ctx, ids, n_ids, &v));
  ROMAP_TRY(run_listed_steps(ctx, v, n_steps, out_loss != nullptr));
  if (out_loss) {
    std::vector<float> tmp(5 * (size_t)n_ids);
    ROMAP_TRY(read_losses(ctx, n_ids, tmp.data(), 5, v, ctx->cfg.per_object != 0));
    for (int i = 0; i < n_ids; ++i) out_loss[i] = tmp[5 * i];
  }
  return ROMAP_OK;
}

romap_status romap_train_step_async(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, int32_t n_steps,
                                    float* out_loss) {
  ROMAP_TRY(check_ctx(ctx));
  if (n_steps < 1) return fail(ROMAP_ERR_INVALID_ARG, "n_steps must be >= 1");
  std::vector<int32_t> v;
  ROMAP_TRY(validate_ids(ctx, ids, n_ids, &v));
  ROMAP_TRY(run_listed_steps(ctx, v, n_steps, out_loss != nullptr));
  if (out_loss) {  // L = loss sum / B on the device, then one asynchronous copy into the caller's buffer
    std::vector<int32_t> rays(v.size());
    for (size_t i = 0; i < v.size(); ++i) rays[i] = ctx->objs_host[v[i]].n_rays;
    HostBatch hb;
    build_batch(v, rays, &hb);
    BatchDesc b;
    ROMAP_TRY(upload_batch(ctx, hb, &b));  // (the step left these arrays in place: no copy)
    ROMAP_TRY(grow(ctx, ctx->ws_loss, sizeof(float) * v.size()));
    launch_final_losses(ctx->cfg.per_object ? ctx->dyn_gather : ctx->dyn, b, (float*)ctx->ws_loss.p, ctx->stream);
    ctx->launches += 1;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out_loss, ctx->ws_loss.p, sizeof(float) * v.size(), cudaMemcpyDefault, ctx->stream));
  }
  return ROMAP_OK;
}

romap_status romap_check_device_status(romap_ctx* ctx) {
  ROMAP_TRY(check_ctx(ctx));
  int32_t st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (st == 0) return ROMAP_OK;
  CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  return status_error(st);
}

// ---- incremental training data and budgeted training (Sec. V-A-1, Eq. 5; Sec. VI) ---------------------------------
romap_status romap_view_angle(const double cam_last[3], const double cam_now[3], const double center[3],
                              double* out_deg) {
  if (!cam_last || !cam_now || !center || !out_deg) return fail(ROMAP_ERR_INVALID_ARG, "NULL argument");
  double dot = 0.0, n_last = 0.0, n_now = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double u = cam_last[a] - center[a], w = cam_now[a] - center[a];
    dot += u * w;
    n_last += u * u;
    n_now += w * w;
  }
  if (!(n_last > 0.0) || !(n_now > 0.0)) {  // a camera at the object centre: no direction, always new data
    *out_deg = 180.0;
    return std::isfinite(n_last) && std::isfinite(n_now) ? ROMAP_OK : fail(ROMAP_ERR_NONFINITE, "non-finite input");
  }
  const double c = std::min(1.0, std::max(-1.0, dot / std::sqrt(n_last * n_now)));
  if (!std::isfinite(c)) return fail(ROMAP_ERR_NONFINITE, "non-finite input");
  *out_deg = std::acos(c) * (180.0 / 3.14159265358979323846);
  return ROMAP_OK;
}

romap_status romap_observe(romap_ctx* ctx, int32_t id, const double cam_center[3], float threshold_deg,
                           const romap_rays* rays, int64_t n, uint32_t flags, int32_t iterations, int32_t* out_updated) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!cam_center) return fail(ROMAP_ERR_INVALID_ARG, "cam_center is required");
  if (!(threshold_deg >= 0.f && threshold_deg <= 180.f)) return fail(ROMAP_ERR_INVALID_ARG, "threshold_deg in [0, 180]");
  if (iterations < 0) return fail(ROMAP_ERR_INVALID_ARG, "iterations must be >= 0");
  Object& o = ctx->objs[id];
  const double center[3] = {o.desc.t[0], o.desc.t[1], o.desc.t[2]};
  bool update = !o.have_view;
  if (!update) {
    double deg = 0.0;
    ROMAP_TRY(romap_view_angle(o.last_view, cam_center, center, &deg));
    update = deg > (double)threshold_deg;
  } else {
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(cam_center[a])) return fail(ROMAP_ERR_NONFINITE, "non-finite camera centre");
  }
  if (update) {
    if (rays && n > 0) ROMAP_TRY(romap_add_rays(ctx, id, rays, n, flags));
    o.have_view = true;
    for (int a = 0; a < 3; ++a) o.last_view[a] = cam_center[a];
    o.pending += iterations;
  }
  if (out_updated) *out_updated = update ? 1 : 0;
  return ROMAP_OK;
}

romap_status romap_pending(romap_ctx* ctx, int32_t id, int64_t* out) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is required");
  *out = ctx->objs[id].pending;
  return ROMAP_OK;
}

romap_status romap_set_pending(romap_ctx* ctx, int32_t id, int64_t pending) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (pending < 0) return fail(ROMAP_ERR_INVALID_ARG, "pending must be >= 0");
  ctx->objs[id].pending = pending;
  return ROMAP_OK;
}

romap_status romap_train_budget(romap_ctx* ctx, const int32_t* ids, int32_t n_ids, float budget_ms,
                                int32_t max_chunk, int32_t* out_steps, float* out_ms, float* out_loss) {
  ROMAP_TRY(check_ctx(ctx));
  std::vector<int32_t> all;
  ROMAP_TRY(validate_ids(ctx, ids, n_ids, &all));
  if (!(budget_ms >= 0.f) || !std::isfinite(budget_ms)) return fail(ROMAP_ERR_INVALID_ARG, "budget_ms must be >= 0");
  if (max_chunk < 1) max_chunk = 64;
  if (out_loss)
    for (int i = 0; i < n_ids; ++i) out_loss[i] = std::numeric_limits<float>::quiet_NaN();
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  double elapsed = 0.0;
  int32_t steps = 0;
  romap_status st = ROMAP_OK;
  std::vector<float> loss;
  while (st == ROMAP_OK) {
    std::vector<int32_t> act;
    for (int32_t id : all)
      if (ctx->objs[id].pending > 0) act.push_back(id);
    if (act.empty()) break;
    auto rays_of = [&](const std::vector<int32_t>& v) {
      int64_t r = 0;
      for (int32_t id : v) r += ctx->objs_host[id].n_rays;
      return r;
    };
    auto key_of = [&](const std::vector<int32_t>& v) {
      std::vector<int32_t> key(v);
      for (int32_t id : v) key.push_back(ctx->objs_host[id].n_rays);
      return key;
    };
    const double left = (double)budget_ms - elapsed;
    std::vector<int32_t> key = key_of(act);
    auto it = ctx->step_ms_est.find(key);
    // the step time of this composition: measured, else predicted from the time per ray, else unknown
    double est = it != ctx->step_ms_est.end() ? it->second
                 : (ctx->ms_per_ray > 0.0 ? ctx->ms_per_ray * (double)rays_of(act) : -1.0);
    int64_t k = 1;
    if (est < 0.0) {
      if (elapsed > 0.0 && elapsed >= (double)budget_ms) break;  // nothing known: one step to measure
    } else if (est <= left) {
      int64_t min_pending = INT64_MAX;
      for (int32_t id : act) min_pending = std::min(min_pending, ctx->objs[id].pending);
      k = std::min<int64_t>(std::min<int64_t>(est > 0.0 ? (int64_t)(left / est) : max_chunk, max_chunk),
                            min_pending);
    } else {
      // the whole batch does not fit: one step of the objects that owe the most steps, as many as fit
      if (!(ctx->ms_per_ray > 0.0)) break;
      std::vector<int32_t> order(act);
      std::stable_sort(order.begin(), order.end(),
                       [&](int32_t a, int32_t b) { return ctx->objs[a].pending > ctx->objs[b].pending; });
      std::vector<int32_t> sub;
      double acc = 0.0;
      for (int32_t id : order) {
        const double c = ctx->ms_per_ray * (double)ctx->objs_host[id].n_rays;
        if (acc + c <= left) {
          sub.push_back(id);
          acc += c;
        }
      }
      if (sub.empty()) break;
      std::sort(sub.begin(), sub.end());
      act = sub;
      key = key_of(act);
      it = ctx->step_ms_est.find(key);
    }
    loss.assign(act.size(), 0.f);
    CUDA_TRY(cudaEventRecord(e0, ctx->stream));
    st = romap_train_step(ctx, act.data(), (int32_t)act.size(), (int32_t)k, loss.data());
    CUDA_TRY(cudaEventRecord(e1, ctx->stream));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    elapsed += ms;
    const double per = ms / (double)k;
    // a composition's first step includes its graph capture: later, replayed steps refine the estimate
    if (it == ctx->step_ms_est.end()) ctx->step_ms_est[key] = per;
    else it->second = 0.5 * it->second + 0.5 * per;
    const double per_ray = per / (double)std::max<int64_t>(1, rays_of(act));
    ctx->ms_per_ray = ctx->ms_per_ray > 0.0 ? 0.8 * ctx->ms_per_ray + 0.2 * per_ray : per_ray;
    steps += (int32_t)k;
    for (int32_t id : act) ctx->objs[id].pending -= k;
    if (out_loss)
      for (size_t j = 0; j < act.size(); ++j)
        for (int i = 0; i < n_ids; ++i)
          if (ids[i] == act[j]) out_loss[i] = loss[j];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out_steps) *out_steps = steps;
  if (out_ms) *out_ms = (float)elapsed;
  return st;
}

romap_status romap_get_grad(romap_ctx* ctx, int32_t id, float* out, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is NULL");
  bool dev = flags & ROMAP_DEVICE_PTR;
  CUDA_TRY(cudaMemcpyAsync(out, ctx->objs[id].grad, sizeof(float) * ctx->g.n_params,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!dev) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

romap_status romap_last_batch(romap_ctx* ctx, int32_t id, int64_t* pool_idx, float* bg, int64_t* out_n) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  const std::vector<int32_t>& k = ctx->last_batch;
  if (k.empty()) return fail(ROMAP_ERR_BAD_STATE, "no step has run");
  const int n = ctx->last_batch_n;
  int pos = -1;
  for (int i = 0; i < n; ++i)
    if (k[i] == id) pos = i;
  if (pos < 0) return fail(ROMAP_ERR_BAD_STATE, "object %d was not in the last step", id);
  int64_t r0 = k[n + pos], r1 = k[n + pos + 1];
  if (out_n) *out_n = r1 - r0;
  if (pool_idx)
    CUDA_TRY(cudaMemcpyAsync(pool_idx, ctx->R.pool_idx + r0, sizeof(int64_t) * (r1 - r0), cudaMemcpyDeviceToHost,
                             ctx->stream));
  if (bg) CUDA_TRY(cudaMemcpyAsync(bg, ctx->R.bg + 3 * r0, sizeof(float) * 3 * (r1 - r0), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

romap_status romap_last_outputs(romap_ctx* ctx, int32_t id, float* out, int64_t* out_n) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  const std::vector<int32_t>& k = ctx->last_batch;
  if (k.empty()) return fail(ROMAP_ERR_BAD_STATE, "no step has run");
  const int n = ctx->last_batch_n;
  int pos = -1;
  for (int i = 0; i < n; ++i)
    if (k[i] == id) pos = i;
  if (pos < 0) return fail(ROMAP_ERR_BAD_STATE, "object %d was not in the last step", id);
  int64_t r0 = k[n + pos], r1 = k[n + pos + 1];
  if (out_n) *out_n = r1 - r0;
  if (out)
    CUDA_TRY(cudaMemcpyAsync(out, ctx->R.out + 6 * r0, sizeof(float) * 6 * (r1 - r0), cudaMemcpyDeviceToHost,
                             ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

romap_status romap_get_state(romap_ctx* ctx, int32_t id, romap_state* out) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!out || !out->params || !out->adam_m || !out->adam_v)
    return fail(ROMAP_ERR_INVALID_ARG, "state buffers must not be NULL");
  if (out->n_params != ctx->g.n_params)
    return fail(ROMAP_ERR_INVALID_ARG, "n_params is %lld, expected %lld", (long long)out->n_params,
                (long long)ctx->g.n_params);
  const Object& o = ctx->objs[id];
  cudaMemcpyKind k = (out->flags & ROMAP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  size_t bytes = sizeof(float) * ctx->g.n_params;
  CUDA_TRY(cudaMemcpyAsync(out->params, o.params, bytes, k, ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(out->adam_m, o.m, bytes, k, ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(out->adam_v, o.v, bytes, k, ctx->stream));
  out->step = o.steps_done;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

romap_status romap_set_state(romap_ctx* ctx, int32_t id, const romap_state* in) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!in || !in->params || !in->adam_m || !in->adam_v)
    return fail(ROMAP_ERR_INVALID_ARG, "state buffers must not be NULL");
  if (in->n_params != ctx->g.n_params) return fail(ROMAP_ERR_INVALID_ARG, "n_params mismatch");
  if (in->step < 0 || in->step > 0x7fffffff) return fail(ROMAP_ERR_INVALID_ARG, "step out of range");
  Object& o = ctx->objs[id];
  cudaMemcpyKind k = (in->flags & ROMAP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  size_t bytes = sizeof(float) * ctx->g.n_params;
  CUDA_TRY(cudaMemcpyAsync(o.params, in->params, bytes, k, ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(o.m, in->adam_m, bytes, k, ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(o.v, in->adam_v, bytes, k, ctx->stream));
  CUDA_TRY(cudaMemsetAsync(o.grad, 0, sizeof(float) * ctx->g.n_params_pad, ctx->stream));
  if (o.gfix) CUDA_TRY(cudaMemsetAsync(o.gfix, 0, sizeof(unsigned long long) * ctx->g.n_params_pad, ctx->stream));
  if (o.table_h) launch_to_half(o.params, o.table_h, ctx->g.n_hash, ctx->stream);
  launch_touched_from_moments(ctx->g, o.m, o.v, o.touched, ctx->stream);  // the loaded moments decide
  CUDA_TRY(cudaGetLastError());
  o.steps_done = in->step;
  ROMAP_TRY(sync_object(ctx, id));
  if (!(in->flags & ROMAP_DEVICE_PTR)) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

romap_status romap_get_stats(romap_ctx* ctx, romap_stats* out) {
  ROMAP_TRY(check_ctx(ctx));
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is NULL");
  unsigned long long live = 0;
  CUDA_TRY(cudaMemcpyAsync(&live, ctx->live_counter, sizeof(live), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *out = ctx->stats;
  out->live_samples = (int64_t)live;
  out->kernel_launches = ctx->launches;
  out->graph_captures = ctx->graph_captures;
  out->graph_replays = ctx->graph_replays;
  return ROMAP_OK;
}

romap_status romap_selftest_wait_timeout(romap_ctx* ctx, int32_t poll_limit) {
  ROMAP_TRY(check_ctx(ctx));
  if (poll_limit < 1) return fail(ROMAP_ERR_INVALID_ARG, "poll_limit must be >= 1");
  CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  launch_selftest_wait(ctx->status, poll_limit, ctx->stream);
  ctx->launches += 1;
  CUDA_TRY(cudaGetLastError());
  int32_t st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  if (st & kStatusTimeout) return fail(ROMAP_ERR_TIMEOUT, "self-test: the bounded wait gave up as expected");
  return ROMAP_OK;
}

romap_status romap_set_tile_kernel(romap_ctx* ctx, int32_t index) {
  ROMAP_TRY(check_ctx(ctx));
  if (index < -1 || index >= kNumTileKernels) return fail(ROMAP_ERR_INVALID_ARG, "tile kernel %d out of range", index);
  if (ctx->g.fp8 && index >= 0 && !lockstep_kernel(index))
    return fail(ROMAP_ERR_UNSUPPORTED, "the FP8 precision runs on the tile-pair lockstep kernels (0, 2, 4, 6) only");
  if (ctx->g.single_net && index >= 0 && !lockstep_kernel(index))
    return fail(ROMAP_ERR_UNSUPPORTED, "the single-network model runs on the tile-pair lockstep kernels (0, 2, 4, 6) only");
  ctx->tile_kernel = index;
  drop_graph(ctx);
  return ROMAP_OK;
}

romap_status romap_autotune_report(romap_ctx* ctx, int32_t* chosen, float* ms, int32_t n, char* names,
                                   size_t names_len) {
  ROMAP_TRY(check_ctx(ctx));
  if (chosen) *chosen = ctx->tile_kernel;
  for (int i = 0; ms && i < n && i < kNumTileKernels; ++i) ms[i] = ctx->tile_kernel_ms[i];
  if (names && names_len) {
    std::string all;
    for (int i = 0; i < kNumTileKernels; ++i) all += std::string(i ? ";" : "") + kTileKernelNames[i];
    snprintf(names, names_len, "%s", all.c_str());
  }
  return ROMAP_OK;
}

romap_status romap_set_adam_skip(romap_ctx* ctx, int32_t on) {
  ROMAP_TRY(check_ctx(ctx));
  if (on != 0 && on != 1) return fail(ROMAP_ERR_INVALID_ARG, "on must be 0 or 1");
  ctx->g.adam_dense = on ? 0 : 1;
  drop_graph(ctx);  // the captured steps carry the old setting
  return ROMAP_OK;
}

romap_status romap_debug_set_pool_size(romap_ctx* ctx, int32_t id, int64_t n) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (n < 0 || n > ctx->objs[id].pool_n)
    return fail(ROMAP_ERR_INVALID_ARG, "n must be in 0..%lld (the pool size)", (long long)ctx->objs[id].pool_n);
  ObjectDev& d = ctx->objs_host[id];
  d.pool_n = n;  // the device record only: the rays per step and the host pool keep their sizes
  CUDA_TRY(cudaMemcpyAsync(ctx->objs_dev + id, &d, sizeof(ObjectDev), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  drop_graph(ctx);
  return ROMAP_OK;
}

romap_status romap_checked_build(int32_t* out) {
  if (!out) return fail(ROMAP_ERR_INVALID_ARG, "out is NULL");
#ifdef ROMAP_CHECKED
  *out = 1;
#else
  *out = 0;
#endif
  return ROMAP_OK;
}

romap_status romap_set_graphs(romap_ctx* ctx, int32_t on) {
  ROMAP_TRY(check_ctx(ctx));
  if (on != 0 && on != 1) return fail(ROMAP_ERR_INVALID_ARG, "on must be 0 or 1");
  ctx->graphs_enabled = on != 0;
  drop_graph(ctx);
  return ROMAP_OK;
}

romap_status romap_set_profiling(romap_ctx* ctx, int32_t on) {
  ROMAP_TRY(check_ctx(ctx));
  ctx->profiling = on != 0;
  return ROMAP_OK;
}

romap_status romap_phase_times(romap_ctx* ctx, double* ms, int64_t* launches) {
  ROMAP_TRY(check_ctx(ctx));
  if (!ms) return fail(ROMAP_ERR_INVALID_ARG, "ms is NULL");
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (auto& p : ctx->prof) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ctx->phase_ms[p.phase] += t;
    ctx->phase_launches[p.phase] += p.launches;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  ctx->prof.clear();
  for (int i = 0; i < ROMAP_N_PHASES; ++i) {
    ms[i] = ctx->phase_ms[i];
    if (launches) launches[i] = ctx->phase_launches[i];
  }
  return ROMAP_OK;
}

romap_status romap_reset_stats(romap_ctx* ctx) {
  ROMAP_TRY(check_ctx(ctx));
  ctx->stats = romap_stats{};
  ctx->launches = 0;
  ctx->graph_captures = 0;
  ctx->graph_replays = 0;
  cudaStreamSynchronize(ctx->stream);
  for (auto& p : ctx->prof) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  ctx->prof.clear();
  for (int i = 0; i < ROMAP_N_PHASES; ++i) {
    ctx->phase_ms[i] = 0.0;
    ctx->phase_launches[i] = 0;
  }
  CUDA_TRY(cudaMemsetAsync(ctx->live_counter, 0, sizeof(unsigned long long), ctx->stream));
  return ROMAP_OK;
}

// ---------------------------------------------------------------------------
// Functional API and rendering: one object record (params given), explicit
// rays, workspace carved from a caller buffer or the context.
// ---------------------------------------------------------------------------
struct FnLayout {
  size_t rays, samples, blocks, batch, dyn, totals, act, total;
  int64_t nr, ns, nb;
};

// store_act: room for the stored activations of every tile (ROMAP_STORE_ACT)
static FnLayout fn_layout(const GridParams& g, int64_t n, bool store_act = false) {
  FnLayout L{};
  L.nr = n;
  L.ns = n * g.n_samples + kTile;
  L.nb = (n + 255) / 256;
  RayBuf R;
  SampleBuf S;
  L.rays = carve_rays(nullptr, n, &R);
  L.samples = carve_samples(nullptr, L.ns, &S);
  L.blocks = align_up(sizeof(uint32_t) * (L.nb + 1), 256);
  L.batch = align_up(sizeof(int32_t) * (4 + L.nb + 8), 256);
  L.dyn = align_up(sizeof(BatchDyn), 256);
  L.totals = 256;
  const int64_t tiles = (L.ns + kTile - 1) / kTile;  // one object: its samples start at tile 0
  L.act = store_act ? align_up(sizeof(float) * (size_t)tiles * act_rows_for(g.LF) * kTile, 256) : 0;
  L.total = L.rays + L.samples + L.blocks + L.batch + L.dyn + L.totals + L.act + 256;
  return L;
}

struct FnView {
  RayBuf R;
  SampleBuf S;
  uint32_t* blocks;
  int32_t* batch;
  BatchDyn* dyn;
  int32_t* totals;
};

static FnView fn_view(char* base, const FnLayout& L) {
  FnView v;
  base = (char*)align_up((size_t)base, 256);
  size_t o = 0;
  carve_rays(base + o, L.nr, &v.R); o += L.rays;
  carve_samples(base + o, L.ns, &v.S); o += L.samples;
  v.blocks = (uint32_t*)(base + o); o += L.blocks;
  v.batch = (int32_t*)(base + o); o += L.batch;
  v.dyn = (BatchDyn*)(base + o); o += L.dyn;
  v.totals = (int32_t*)(base + o); o += L.totals;
  v.S.act = L.act ? (float*)(base + o) : nullptr;
  return v;
}

static romap_status fn_setup(romap_ctx* ctx, const float* params, float* grad, const float half[3], uint64_t seed,
                             uint32_t step, const uint64_t* occ, const float* origin, const float* dir,
                             const float* bg, int64_t n, uint32_t flags, char* ws, size_t ws_bytes, FnView* out_v,
                             BatchDesc* out_b, bool upload) {
  if (!params || !half || !origin || !dir || !bg || !ws) return fail(ROMAP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > (int64_t)1 << 24) return fail(ROMAP_ERR_INVALID_ARG, "n must be in 1..2^24");
  if (flags & ~(ROMAP_JITTER | ROMAP_STORE_ACT)) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  for (int a = 0; a < 3; ++a)
    if (!(half[a] > 0.f)) return fail(ROMAP_ERR_INVALID_ARG, "half_size must be positive");
  FnLayout L = fn_layout(ctx->g, n, (flags & ROMAP_STORE_ACT) != 0);
  if (ws_bytes < L.total) return fail(ROMAP_ERR_INVALID_ARG, "workspace of %zu bytes is smaller than %zu", ws_bytes, L.total);
  FnView v = fn_view(ws, L);
  HostBatch hb;
  build_batch(std::vector<int32_t>{0}, std::vector<int32_t>{(int32_t)n}, &hb);
  if (upload)
    CUDA_TRY(cudaMemcpyAsync(v.batch, hb.arr.data(), sizeof(int32_t) * hb.arr.size(), cudaMemcpyHostToDevice,
                             ctx->stream));
  ObjectDev d{};
  d.params = const_cast<float*>(params);
  d.grad = grad;
  d.occ = occ;
  for (int a = 0; a < 3; ++a) {
    d.half[a] = half[a];
    d.inv_ext[a] = 1.0f / (half[a] - (-half[a]));
  }
  d.key0 = (uint32_t)seed;
  d.key1 = (uint32_t)(seed >> 32);
  d.n_rays = (int32_t)n;
  set_object_step(d, step, ctx->cfg.beta1, ctx->cfg.beta2);
  ObjectDev* od = ctx->fn_obj_dev;
  CUDA_TRY(cudaMemcpyAsync(od, &d, sizeof(d), cudaMemcpyHostToDevice, ctx->stream));
  BatchDesc b = desc_from(hb, v.batch, od);
  b.explicit_rays = 1;
  b.explicit_step = step;
  b.jitter = (flags & ROMAP_JITTER) ? 1 : 0;
  b.ex_o = origin;
  b.ex_d = dir;
  b.ex_bg = bg;
  *out_v = v;
  *out_b = b;
  return ROMAP_OK;
}

romap_status romap_fn_workspace_size(romap_ctx* ctx, int64_t n, uint32_t flags, size_t* bytes) {
  if (!ctx || !bytes) return fail(ROMAP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > (int64_t)1 << 24) return fail(ROMAP_ERR_INVALID_ARG, "n must be in 1..2^24");
  if (flags & ~(ROMAP_JITTER | ROMAP_STORE_ACT)) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  *bytes = fn_layout(ctx->g, n, (flags & ROMAP_STORE_ACT) != 0).total;
  return ROMAP_OK;
}

romap_status romap_fn_forward(romap_ctx* ctx, const float* params, const float half_size[3], uint64_t seed,
                              uint32_t step, const uint64_t* occupancy, const float* origin, const float* dir,
                              const float* bg, int64_t n, uint32_t flags, void* workspace, size_t ws_bytes,
                              float* out_ray, float* out_samples) {
  ROMAP_TRY(check_ctx(ctx));
  if (!out_ray) return fail(ROMAP_ERR_INVALID_ARG, "out_ray is NULL");
  FnView v;
  BatchDesc b;
  ROMAP_TRY(fn_setup(ctx, params, nullptr, half_size, seed, step, occupancy, origin, dir, bg, n, flags,
                     (char*)workspace, ws_bytes, &v, &b, true));
  ROMAP_TRY(run_sampling(ctx, b, v.R, v.S, v.blocks, v.dyn, v.totals, false));
  launch_tile_mlp(0, ctx->g, b, v.dyn, v.totals, v.R, v.S, tile_ctas(ctx), ctx->stream);
  launch_composite(0, ctx->g, b, v.R, v.S, v.dyn, nullptr, ctx->stream);
  ctx->launches += 2;
  CUDA_TRY(cudaMemcpyAsync(out_ray, v.R.out, sizeof(float) * 6 * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (out_samples) {  // per slot: t, delta, x, y, z, sigma (zeros for missed or culled slots)
    CUDA_TRY(cudaMemsetAsync(out_samples, 0, sizeof(float) * 6 * n * ctx->g.n_samples, ctx->stream));
    launch_sample_slots(ctx->g, n, v.R, v.S, out_samples, ctx->stream);
    ctx->launches += 1;
  }
  CUDA_TRY(cudaGetLastError());
  return ROMAP_OK;
}

romap_status romap_fn_backward(romap_ctx* ctx, const float* params, const float half_size[3], uint64_t seed,
                               uint32_t step, const uint64_t* occupancy, const float* origin, const float* dir,
                               const float* bg, int64_t n, uint32_t flags, void* workspace, size_t ws_bytes,
                               const float* grad_ray, float* grad_params, float* out_dsigma) {
  ROMAP_TRY(check_ctx(ctx));
  if (!grad_ray || !grad_params) return fail(ROMAP_ERR_INVALID_ARG, "grad_ray and grad_params are required");
  if (reinterpret_cast<uintptr_t>(grad_params) % 16 != 0)
    return fail(ROMAP_ERR_INVALID_ARG, "grad_params must be 16-byte aligned");
  FnView v;
  BatchDesc b;
  ROMAP_TRY(fn_setup(ctx, params, grad_params, half_size, seed, step, occupancy, origin, dir, bg, n, flags,
                     (char*)workspace, ws_bytes, &v, &b, false));
  v.R.gout = grad_ray;
  GridParams g = ctx->g;
  g.det = 0;  // the caller's gradient buffer is FP32: floating-point atomics
  launch_composite(2, g, b, v.R, v.S, v.dyn, nullptr, ctx->stream);
  launch_tile_mlp(1, g, b, v.dyn, v.totals, v.R, v.S, tile_ctas(ctx), ctx->stream);
  ctx->launches += 2;
  if (out_dsigma) {
    CUDA_TRY(cudaMemsetAsync(out_dsigma, 0, sizeof(float) * n * ctx->g.n_samples, ctx->stream));
    launch_scatter_slots(ctx->g, n, v.R, v.S, v.S.dsigma, 1, out_dsigma, 1, ctx->stream);
    ctx->launches += 1;
  }
  CUDA_TRY(cudaGetLastError());
  return ROMAP_OK;
}

romap_status romap_render(romap_ctx* ctx, int32_t id, const float* origin, const float* dir, int64_t n,
                          const float bg[3], float* out_rgb, float* out_depth, float* out_opacity, uint32_t flags) {
  ROMAP_TRY(check_ctx(ctx));
  ROMAP_TRY(check_id(ctx, id));
  if (!origin || !dir || !bg || n < 1) return fail(ROMAP_ERR_INVALID_ARG, "origin, dir, bg required and n >= 1");
  if (flags & ~(ROMAP_DEVICE_PTR | ROMAP_OBJECT_FRAME)) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  bool dev = flags & ROMAP_DEVICE_PTR;
  Object& o = ctx->objs[id];
  FnLayout L = fn_layout(ctx->g, n);
  size_t extra = align_up(sizeof(float) * 9 * n, 256) + align_up(sizeof(float) * 6 * (size_t)n, 256) +
                 align_up(sizeof(float) * 6 * (size_t)n, 256) + 1024;
  ROMAP_TRY(grow(ctx, ctx->ws_stage, L.total + extra));
  char* base = (char*)ctx->ws_stage.p;
  char* xb = base + align_up(L.total, 256);
  float* o_obj = (float*)xb;
  float* d_obj = o_obj + 3 * n;
  float* bgs = d_obj + 3 * n;
  float* scratch_rgb = (float*)(xb + align_up(sizeof(float) * 9 * n, 256));
  float* scratch_dep = scratch_rgb + 3 * n;
  uint8_t* scratch_cls = (uint8_t*)(scratch_dep + n);
  const float* so = origin;
  const float* sd = dir;
  float* st = (float*)(xb + align_up(sizeof(float) * 9 * n, 256) + align_up(sizeof(float) * 6 * (size_t)n, 256));
  if (!dev) {
    CUDA_TRY(cudaMemcpyAsync(st, origin, 12 * n, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(st + 3 * n, dir, 12 * n, cudaMemcpyHostToDevice, ctx->stream));
    so = st;
    sd = st + 3 * n;
  }
  std::vector<float> hbg(3 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    hbg[3 * i] = bg[0]; hbg[3 * i + 1] = bg[1]; hbg[3 * i + 2] = bg[2];
  }
  CUDA_TRY(cudaMemcpyAsync(bgs, hbg.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
  float cz = (float)std::cos(o.desc.yaw), sz = (float)std::sin(o.desc.yaw);
  launch_transform_rays(so, sd, nullptr, nullptr, nullptr, n, (flags & ROMAP_OBJECT_FRAME) ? 1 : 0, o.desc.t[0],
                        o.desc.t[1], o.desc.t[2], cz, sz, o_obj, d_obj, scratch_rgb, scratch_dep, scratch_cls,
                        ctx->stream);
  FnView v;
  BatchDesc b;
  ROMAP_TRY(fn_setup(ctx, o.params, nullptr, o.desc.half_size, o.desc.seed, 0, o.occ, o_obj, d_obj, bgs, n, 0, base,
                     L.total, &v, &b, true));
  ROMAP_TRY(run_sampling(ctx, b, v.R, v.S, v.blocks, v.dyn, v.totals, false));
  launch_tile_mlp(0, ctx->g, b, v.dyn, v.totals, v.R, v.S, tile_ctas(ctx), ctx->stream);
  launch_composite(0, ctx->g, b, v.R, v.S, v.dyn, nullptr, ctx->stream);
  ctx->launches += 3;
  CUDA_TRY(cudaGetLastError());
  float* outs = st;  // staging area is free again: rgb [3n], depth [n], opacity [n]
  launch_split_outputs(v.R.out, n, outs, outs + 3 * n, outs + 4 * n, ctx->stream);
  ctx->launches += 1;
  CUDA_TRY(cudaGetLastError());
  cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (out_rgb) CUDA_TRY(cudaMemcpyAsync(out_rgb, outs, sizeof(float) * 3 * n, k, ctx->stream));
  if (out_depth) CUDA_TRY(cudaMemcpyAsync(out_depth, outs + 3 * n, sizeof(float) * n, k, ctx->stream));
  if (out_opacity) CUDA_TRY(cudaMemcpyAsync(out_opacity, outs + 4 * n, sizeof(float) * n, k, ctx->stream));
  if (!dev) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ROMAP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Functional forward that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// render: a plugin inside a host framework that owns every byte of device
// memory and hands out no allocator, or a real-time mapping loop that must
// not call cudaMalloc/cudaFree (which may synchronise the whole device and
// stall the frame).  romap_fn_forward needs a caller workspace, which such a
// caller cannot provide.  This variant keeps its scratch (ray records,
// compacted samples, scan totals, the object record) in one file-scope device
// array of kNoAllocScratchBytes: a device reserves those bytes when the
// library's device code is first loaded there (under lazy module loading that
// may be the first call) and holds them until the process exits.
//
// Set-up: the first call on each device, with that device current, looks up
// the array's device address with cudaGetSymbolAddress (host code cannot use
// the array's name as a device address) and caches it.  The caller's stream
// must belong to the current device (the cached address is that device's).  The object record and the
// batch arrays reach the array through a set-up kernel's by-value parameters,
// never through a copy from host memory.  All calls on a device share the one array and
// it keeps the last call's contents: every scratch word the kernels read is
// written earlier in the same call, so nothing needs clearing, but calls that
// overlap on the GPU (two streams, two threads) race on the array and must be
// serialised by the caller.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Writes the one-object record and the one-entry batch arrays (slot 0; rays 0..n; blocks 0..nb; no tiles; every
// block in entry 0) into the static scratch.  Everything arrives by value in the launch parameters, so nothing is
// copied from host memory that may be gone when the kernel runs.
__global__ void k_noalloc_setup(ObjectDev d, ObjectDev* od, int32_t* batch, int32_t n, int32_t nb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *od = d;
    batch[0] = 0;                     // slot[1]
    batch[1] = 0; batch[2] = n;       // ray_base[2]
    batch[3] = 0; batch[4] = nb;      // block_base[2]
    batch[5] = 0; batch[6] = 0;       // tile_base[2]
  }
  if (i < nb) batch[7 + i] = 0;       // block_obj[nb]
}

romap_status noalloc_scratch(int dev, char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(ROMAP_ERR_UNSUPPORTED, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(ROMAP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = (char*)g_noalloc_ptr[dev];
  return ROMAP_OK;
}
}  // namespace

extern "C" romap_status romap_fn_forward_noalloc(const romap_config* cfg, void* cuda_stream, const float* params,
                                                 const float half_size[3], uint64_t seed, uint32_t step,
                                                 const uint64_t* occupancy, const float* origin, const float* dir,
                                                 const float* bg, int64_t n, uint32_t flags, float* out_ray) {
  GridParams g;
  ROMAP_TRY(make_grid(cfg, &g));
  if (!params || !half_size || !origin || !dir || !bg || !out_ray) return fail(ROMAP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > (int64_t)1 << 24) return fail(ROMAP_ERR_INVALID_ARG, "n must be in 1..2^24");
  if (flags & ~(ROMAP_JITTER)) return fail(ROMAP_ERR_INVALID_ARG, "bad flags");
  for (int a = 0; a < 3; ++a)
    if (!(half_size[a] > 0.f)) return fail(ROMAP_ERR_INVALID_ARG, "half_size must be positive");
  const size_t rec = align_up(sizeof(ObjectDev), 256);
  FnLayout L = fn_layout(g, n);
  if (rec + L.total > kNoAllocScratchBytes) {
    int64_t max_n = 0;
    for (int64_t lo = 1, hi = n; lo <= hi;) {  // largest n that fits, for the message
      int64_t mid = lo + (hi - lo) / 2;
      if (rec + fn_layout(g, mid).total <= kNoAllocScratchBytes) { max_n = mid; lo = mid + 1; } else hi = mid - 1;
    }
    return fail(ROMAP_ERR_CAPACITY,
                "romap_fn_forward_noalloc: %lld rays of %d samples need %zu bytes of scratch, more than the %zu-byte "
                "static scratch; at most %lld rays fit",
                (long long)n, g.n_samples, rec + L.total, kNoAllocScratchBytes, (long long)max_n);
  }
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int stream_dev = dev;
  CUDA_TRY(cudaStreamGetDevice(stream, &stream_dev));
  if (stream_dev != dev)
    return fail(ROMAP_ERR_INVALID_ARG, "the stream belongs to device %d but device %d is current", stream_dev, dev);
  char* base = nullptr;
  ROMAP_TRY(noalloc_scratch(dev, &base));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ObjectDev* od = (ObjectDev*)base;
  FnView v = fn_view(base + rec, L);
  HostBatch hb;  // host description only (counts and offsets); its arrays are written on the device below
  build_batch(std::vector<int32_t>{0}, std::vector<int32_t>{(int32_t)n}, &hb);
  ObjectDev d{};
  d.params = const_cast<float*>(params);
  d.occ = occupancy;
  for (int a = 0; a < 3; ++a) {
    d.half[a] = half_size[a];
    d.inv_ext[a] = 1.0f / (half_size[a] - (-half_size[a]));
  }
  d.key0 = (uint32_t)seed;
  d.key1 = (uint32_t)(seed >> 32);
  d.n_rays = (int32_t)n;
  d.step = step;  // the forward reads the step as the RNG counter only
  k_noalloc_setup<<<(unsigned)((hb.n_blocks + 255) / 256), 256, 0, stream>>>(d, od, v.batch, (int32_t)n,
                                                                               hb.n_blocks);
  BatchDesc b = desc_from(hb, v.batch, od);
  b.explicit_rays = 1;
  b.explicit_step = step;
  b.jitter = (flags & ROMAP_JITTER) ? 1 : 0;
  b.ex_o = origin;
  b.ex_d = dir;
  b.ex_bg = bg;
  launch_ray_setup(g, b, v.R, v.blocks, stream);
  launch_scan(g, b, v.blocks, v.dyn, v.totals, v.S, nullptr, stream);
  launch_write_samples(g, b, v.R, v.blocks, v.dyn, v.S, stream);
  launch_tile_mlp(0, g, b, v.dyn, v.totals, v.R, v.S, sms > 0 ? sms : 1, stream);
  launch_composite(0, g, b, v.R, v.S, v.dyn, nullptr, stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(out_ray, v.R.out, sizeof(float) * 6 * n, cudaMemcpyDeviceToDevice, stream));
  return ROMAP_OK;
}
