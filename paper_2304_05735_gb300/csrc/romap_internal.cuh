// Internal declarations shared by the CUDA translation units of libromap.
//
// Data layout in HBM (one context):
//  * per object (slot k of max_objects): parameters, gradient, Adam m and v as
//    FP32 arrays of n_params_pad floats (hash table first, level-major, entry
//    x F; then the five MLP layers row-major [out][in]); an FP16 copy of the
//    hash table for the mixed-precision path; the ray pool as structure of
//    arrays (object-frame origin and unit direction, target rgb, depth,
//    class); an optional 64^3 occupancy bitgrid.
//  * per step (workspace): ray records and compacted sample records, both
//    structure of arrays; every object's samples start on a 128-sample tile
//    boundary so that a tile belongs to one object.  The mixed-precision path
//    keeps no sample records: it packs whole rays into tiles by their number
//    of live samples (the tile plan below) and forms the samples in-kernel.
#pragma once
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace romap {

constexpr int kH = 64;          // MLP hidden width (Sec. VI: hidden size 64)
constexpr int kGeo = 15;        // geometry features passed from the density to the colour net
constexpr int kDOut = 16;       // density-net outputs: log-density + 15 geometry features
constexpr int kMaxL = 16;       // maximum levels
constexpr int kTile = 128;      // samples per tile of the MLP kernels
constexpr int kOC = 20;         // rows of the density-output/colour-input buffer (1 + 15 + 3 + pad)
constexpr int kCinPad = 20;     // colour-net first-layer input width as stored (cin <= 18, zero padded)
constexpr int kC3Rows = 4;      // colour-net last layer rows as stored (3, zero padded)
constexpr int kAS = 132;        // row stride (floats) of the per-tile activation buffers in shared memory
constexpr int kThreads = 256;   // threads of the tile kernel
constexpr uint32_t kNoRay = 0xffffffffu;

enum : uint32_t { kPurposeRay = 1, kPurposeBg = 2, kPurposeJitter = 3, kPurposeInitHash = 4, kPurposeInitMlp = 5 };
enum : int { kClsObject = 0, kClsBackground = 1, kClsOccluder = 2 };

// Grid and network shape, passed by value to kernels.
struct GridParams {
  int L, F, LF;
  uint32_t T;
  int res[kMaxL];
  uint32_t off[kMaxL];     // first entry of level l
  int dense[kMaxL];
  int64_t n_hash;          // hash parameters (entries * F)
  int64_t mlp_off[7];      // absolute parameter offsets of the MLP layers (5, 6: single-network hidden layers 2, 3)
  int64_t n_params;
  int64_t n_params_pad;    // n_params rounded up to a multiple of 4
  int dir_dims, cin;       // cin = 15 + dir_dims
  int n_samples;           // N
  float lambda1, lambda2;
  float lr, beta1, beta2, eps;
  int bg_random;
  float bg_const[3];
  int accuracy;            // FP64 transmittance log-sum and weights in the FP32 compositing kernel
  int fp8;                 // mixed path: hidden 64x64 forward GEMM in FP8 E4M3
  int f16;                 // mixed path: MLP operands in FP16 instead of BF16 (backward gradient operands scaled by B)
  int single_net;          // colour logits = density-net outputs 1..3; the colour net is skipped
  int extra;               // single-network hidden layers after the first (0..2), 64x64 each
  int det;                 // FP32 path: gradients and losses accumulated in 64-bit fixed point (bit-reproducible)
  int adam_dense;          // 1: Adam updates every chunk (no skip of never-touched chunks; same results)
  int32_t* status;         // device status word of the context (bounds checks of the ROMAP_CHECKED build), or null
};

// Deterministic accumulation (the `deterministic` configuration): every gradient contribution is rounded once to a
// 64-bit fixed-point integer with kFixBits fractional bits and added with an integer atomic.  Integer addition is
// associative, so a sum has the same bits whatever order its atomics land in.  Range per accumulator +-2^(63 -
// kFixBits); a single contribution beyond +-kFixMaxContribution (or NaN) is not added and sets a status bit.
constexpr int kFixBits = 46;
constexpr float kFixMaxContribution = 1024.0f;
constexpr int kFixLossBits = 32;   // per-object loss sums (B L and its four components): range +-2^31
constexpr float kFixLossMaxContribution = 1048576.0f;  // per ray
// Adam skips chunks of kAdamChunk parameters that were never touched (see k_adam).
constexpr int kAdamChunk = 256;

// One live object as the kernels see it (device-resident, indexed by slot).
struct ObjectDev {
  float* params;
  float* grad;
  float* m;
  float* v;
  uint16_t* table_h;       // FP16 copy of the hash table (mixed precision)
  const float* pool_o;     // [3n] object frame
  const float* pool_d;     // [3n] unit
  const float* pool_rgb;   // [3n]
  const float* pool_depth; // [n]
  const uint8_t* pool_cls; // [n]
  int64_t pool_n;
  const uint64_t* occ;     // 4096 words or null
  float half[3];
  float inv_ext[3];        // 1 / (2 half), FP32
  uint32_t key0, key1;     // Philox key
  int32_t n_rays;          // rays per step B = min(rays_per_step, pool_n)
  int32_t whole_pool;      // 1 if the whole pool is used in order
  uint32_t step;           // Adam step about to run (1-based); advanced after the Adam kernel
  float bc1, bc2;          // Adam bias corrections of that step: 1 / (1 - beta1^step), 1 / (1 - beta2^step)
  float bc1_prev, bc2_prev; // those of the step before (the update that runs after the counter has advanced)
  int32_t pad_;
  unsigned long long* gfix; // deterministic mode: fixed-point gradient accumulator [n_params_pad], else null
  uint8_t* touched;        // per chunk of kAdamChunk parameters: 1 once any gradient entry was non-zero (or null:
                           // every chunk counts as touched)
};

// Adam bias corrections of step t (Kingma & Ba, Algorithm 1), evaluated in FP64 and rounded once to FP32.
__host__ __device__ inline void adam_bias_corrections(float beta1, float beta2, uint32_t t, float* c1, float* c2) {
  *c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)t)));
  *c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)t)));
}
__host__ __device__ inline void set_object_step(ObjectDev& d, uint32_t t, float beta1, float beta2) {
  d.step = t;
  adam_bias_corrections(beta1, beta2, t, &d.bc1, &d.bc2);
  if (t >= 2) {
    adam_bias_corrections(beta1, beta2, t - 1u, &d.bc1_prev, &d.bc2_prev);
  } else {
    d.bc1_prev = d.bc2_prev = 1.0f;
  }
}

// Per-batch-object values written on the device during a step.
struct BatchDyn {
  int64_t sample_base;     // first sample (tile aligned)
  int32_t n_samples;       // live samples
  int32_t tile_base;
  int32_t n_tiles;
  int32_t pad_;
  float loss[5];           // B*L, then rgb, rr, depth, density sums (unscaled)
  float pad2_[3];
  unsigned long long loss_fix[5];  // deterministic mode: the same sums in fixed point (kFixLossBits)
  int64_t pad3_;
};

// Tile plan of the mixed-precision path: whole rays packed into tiles of kTile sample slots, each ray's live samples
// in consecutive slots, the rays of a tile one after another from slot 0.  Rays are grouped by their exact live count
// c (1..kPlanMaxCount); per object, tile *patterns* are formed greedily from the count histogram (first fit
// decreasing over the histogram: the largest remaining count opens a tile, then the largest counts that still fit
// fill it, as many copies of each as fit) and every pattern is repeated as often as its counts allow.  Each pattern
// repetition exhausts the rarest of its counts relative to its multiplicity, so the histogram empties in a bounded
// number of patterns; past kPlanMaxPat - kPlanMaxCount - 1 patterns or kPlanSegsPerCount segments of one count, the
// remaining rays of each count go into single-count tiles of floor(128 / c) rays.  Rays with c = 0 take no slot.
constexpr int kPlanMaxCount = 128;           // N <= 128 candidates per ray in the mixed path
constexpr int kPlanCounts = kPlanMaxCount + 1;
constexpr int kPlanMaxPat = 512;             // patterns per object
constexpr int kPlanSegsPerCount = 32;        // patterns one count may appear in
// Per pattern (two int4): {first tile (object-relative), tiles, rays per full tile, first perm index
// (object-relative)} and {rays, used slots of a full tile, the count of a single-count pattern (else 0), 0}; the last
// tile of a single-count pattern may hold fewer rays.
// Per segment (count c in pattern p, two int4): {first rank among the object's rays of count c, first tile, copies
// per tile a, tiles} and {slot of the first copy in a tile, its position in the tile's ray list, rays per full
// tile, first perm index of the pattern}.
// Tile record (int4): {batch entry, tile index, rays | used slots << 8, first perm index}.

// Batch description (device): object slots and the ray/block prefix sums.
struct BatchDesc {
  const int32_t* slot;       // [n] object slot of batch entry i
  const int32_t* ray_base;   // [n+1]
  const int32_t* block_base; // [n+1] blocks of 256 rays
  const int32_t* block_obj;  // [n_blocks] batch entry of each ray block
  const int32_t* tile_base;  // [n+1] first fused-kernel tile of each entry (slots of P per ray, 128 per tile)
  int32_t n;
  int32_t n_blocks;
  int32_t n_rays;
  int32_t explicit_rays;     // functional API: rays given, slot r = ray r, no pool draw
  uint32_t explicit_step;    // RNG step of the functional API
  int32_t jitter;            // stratified jitter (training) vs midpoints (render)
  const float* ex_o;         // explicit rays, object frame [3n]
  const float* ex_d;
  const float* ex_bg;        // [3n]
  ObjectDev* objs;           // device array indexed by slot
  // tile plan (mixed-precision path only; plan == 0 elsewhere)
  int32_t plan;
  uint32_t* plan_hist;       // [n * kPlanCounts] rays of each live count per entry (zero between steps)
  uint32_t* plan_bcnt;       // [n_blocks * kPlanCounts] each ray block's offset within each live count of its entry
  int4* plan_pat;            // [n * kPlanMaxPat * 2] patterns of each entry (two int4 each)
  int32_t* plan_npat;        // [n] patterns of each entry
  int4* plan_seg;            // [n * kPlanCounts * kPlanSegsPerCount * 2] segments of each entry and count
  int32_t* plan_nseg;        // [n * kPlanCounts] segments of each entry and count
  int32_t* plan_ent;         // [n] first tile of each entry
  int32_t* plan_perm;        // [n_rays] ray indices in tile order (rays with live samples only)
  int32_t* plan_rstart;      // [n_rays] first slot (in its tile) of the ray at each perm position
  int2* plan_slot;           // [max tiles * kTile] {ray, live-sample index} of each used slot
  int4* plan_tiles;          // [max tiles] tile records
  int32_t* plan_npairs;      // [1] number of tile pairs
  int32_t* status;           // device status word (deterministic accumulation range), or null
  int32_t plan_cap_tiles;    // capacity of plan_tiles (bounds checks)
};

// Per-step ray records (structure of arrays, capacity R).
struct RayBuf {
  float* o;        // [3R] object frame
  float* d;        // [3R]
  float* tn;       // [R]
  float* tf;       // [R]
  float* bg;       // [3R]
  float* rgb;      // [3R] target
  float* depth;    // [R]
  uint8_t* cls;    // [R]
  int64_t* pool_idx; // [R]
  uint32_t* count; // [R] live samples
  uint32_t* mask;  // [4R] live candidates of the ray (bit i of word i / 32), mixed-precision path
  uint32_t* off;   // [R] local offset in its block, then global sample offset
  int32_t* obj;    // [R] batch entry
  float* out;      // [6R] C_hat(3), D_hat, A, sum sigma
  const float* gout; // [6R] upstream gradient (functional API), or null
};

// Per-step compacted samples (structure of arrays, capacity S).
struct SampleBuf {
  float* x;        // [3S] (x, y, z interleaved)
  float* t;        // [S]
  float* dt;       // [S]
  uint32_t* ray;   // [S] ray index or kNoRay
  uint32_t* cand;  // [S] candidate index within the ray
  float* sigma;    // [S]
  float* rgb;      // [3S]
  float* dsigma;   // [S] dL/dsigma including the direct density term
  float* drgb;     // [3S]
  float* act;      // stored activations [tiles][act_rows][128] (functional API, ROMAP_STORE_ACT), or null
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the Philox S-box with
// multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,
// 0xBB67AE85.  u01(x) = (x >> 8) * 2^-24.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}
__host__ __device__ inline uint32_t u4_word(const U4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ inline float u01(uint32_t x) { return __fmul_rn((float)(x >> 8), 5.9604644775390625e-08f); }

// Launchers (defined in the .cu files), all on `stream`.
void launch_init_params(const GridParams& g, float* params, uint32_t key0, uint32_t key1, cudaStream_t stream);
void launch_transform_rays(const float* o_in, const float* d_in, const float* rgb_in, const float* depth_in,
                           const uint8_t* cls_in, int64_t n, int object_frame, float tx, float ty, float tz, float cz,
                           float sz, float* o_out, float* d_out, float* rgb_out, float* depth_out, uint8_t* cls_out,
                           cudaStream_t stream);
// One object's range of a multi-object ray append: its rays [first, first + count) of the concatenated inputs go to
// its pool arrays (already offset to the append position), moved to the object frame with translation t and
// yaw (cos cz, sin sz).
struct XformObj {
  int64_t first;
  float t[3];
  float cz, sz;
  float *o_out, *d_out, *rgb_out, *depth_out;
  uint8_t* cls_out;
};
void launch_transform_rays_multi(const float* o_in, const float* d_in, const float* rgb_in, const float* depth_in,
                                 const uint8_t* cls_in, int64_t n, int object_frame, const XformObj* xo, int n_obj,
                                 cudaStream_t stream);
void launch_ray_setup(const GridParams& g, const BatchDesc& b, RayBuf r, uint32_t* block_sums, cudaStream_t stream);
void launch_scan(const GridParams& g, const BatchDesc& b, uint32_t* block_sums, BatchDyn* dyn, int32_t* totals,
                 SampleBuf s, unsigned long long* live_counter, cudaStream_t stream);
void launch_write_samples(const GridParams& g, const BatchDesc& b, RayBuf r, const uint32_t* block_sums,
                          const BatchDyn* dyn, SampleBuf s, cudaStream_t stream);
// mode: 0 forward (sigma, rgb out), 1 backward (recompute + adjoint + gradients)
void launch_tile_mlp(int mode, const GridParams& g, const BatchDesc& b, const BatchDyn* dyn, const int32_t* totals,
                     RayBuf r, SampleBuf s, int n_ctas, cudaStream_t stream);
// mode: 0 render (outputs only), 1 training loss + adjoint, 2 upstream gradient + adjoint
void launch_composite(int mode, const GridParams& g, const BatchDesc& b, RayBuf r, SampleBuf s, BatchDyn* dyn,
                      int32_t* status, cudaStream_t stream);
void launch_adam(const GridParams& g, const BatchDesc& b, int write_half, cudaStream_t stream);
// the two halves of launch_adam: the update (prev: of the step before the object's current step counter) and the
// step-counter advance
void launch_adam_update(const GridParams& g, const BatchDesc& b, int write_half, int prev, cudaStream_t stream);
void launch_advance_step(const GridParams& g, const BatchDesc& b, cudaStream_t stream);
// Deterministic mode, after the backward: adds each object's fixed-point gradient into its FP32 gradient (entries
// with a zero accumulator are left alone), zeroes the accumulator, and converts the fixed-point loss sums.
void launch_fix_finish(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, cudaStream_t stream);
// Sets each chunk's Adam touched flag from its moments (1 where any m or v entry is non-zero): after a state load.
void launch_touched_from_moments(const GridParams& g, const float* m, const float* v, uint8_t* touched,
                                 cudaStream_t stream);
void launch_final_losses(const BatchDyn* dyn, const BatchDesc& b, float* out, cudaStream_t stream);
void launch_scatter_slots(const GridParams& g, int64_t n_rays, const RayBuf r, const SampleBuf s, const float* src,
                          int src_stride, float* dst, int dst_stride, cudaStream_t stream);
void launch_sample_slots(const GridParams& g, int64_t n_rays, const RayBuf r, const SampleBuf s, float* dst,
                         cudaStream_t stream);
void launch_split_outputs(const float* ray_out, int64_t n, float* rgb, float* depth, float* opacity,
                          cudaStream_t stream);
int tile_kernel_smem_bytes(int LF);
// Rows of one tile's stored activations (ROMAP_STORE_ACT): encoding (L F padded to 16 or 32), the density hidden
// layer, the 16 density-net outputs and the two colour hidden layers (or the single-network hidden layers 2, 3).
int act_rows_for(int LF);
// Mixed precision: fused forward + compositing + backward on tensor cores; P slots per ray (power of two <= 128).
// Marching cubes: at most kMcMaxTri triangles per cube; the case table is built by construction (mc_table.cu).
constexpr int kMcMaxTri = 5;
int build_mc_table(int8_t table[256][3 * kMcMaxTri + 1], uint8_t counts[256]);
size_t mc_workspace_bytes();
int mc_lattice_points();
void launch_lattice_density(const GridParams& g, const ObjectDev* objs, int slot, float* dens, cudaStream_t stream);
int launch_mc(const GridParams& g, const ObjectDev* objs, int slot, float iso, char* ws, int emit, int64_t cap_v,
              float* verts, int64_t cap_t, int32_t* tris, uint32_t* totals_out, const int8_t* table,
              const uint8_t* counts, cudaStream_t stream);
void launch_occ_update(const GridParams& g, const ObjectDev* objs, int slot, float decay, float threshold, int reset,
                       float* dens, uint64_t* bits, cudaStream_t stream);
void launch_plan_rays(const GridParams& g, const BatchDesc& b, RayBuf r, BatchDyn* dyn, cudaStream_t stream);
// Tile patterns of every batch entry (after the ray setup, before the scan writes the tile records).
void launch_plan_patterns(const BatchDesc& b, cudaStream_t stream);
// interleave: CTA c takes every n_ctas-th tile pair (tile) from c instead of a contiguous range, so that all CTAs
// work on the same few objects at a time (their tables and gradients then stay in L2).
void launch_tile_tc(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                    int total_tiles, int n_ctas, int interleave, cudaStream_t stream);
// launch_tile_tc with one tile per CTA and two CTAs per SM (BF16 or FP16 operands, two-network model only)
void launch_tile_tc1(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                     int max_tiles, int n_ctas, int interleave, cudaStream_t stream);
// launch_tile_tc with the two warpgroups of a tile pair decoupled (BF16 or FP16 operands, two-network model only)
void launch_tile_tcd(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                     int max_tiles, int n_ctas, int interleave, cudaStream_t stream);
// the FP16-operand instances of launch_tile_tc
void launch_tile_tc_f16(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                        int total_tiles, int n_ctas, int interleave, cudaStream_t stream);
void launch_to_half(const float* params, uint16_t* table_h, int64_t n_hash, cudaStream_t stream);
// Warp-specialized variant of launch_tile_tc (same results): compute warps run the MMA chain of one tile while
// memory warps gather the next tile and scatter the previous one.
void launch_tile_ws(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                    int total_tiles, int n_ctas, int interleave, cudaStream_t stream);
// Dynamic shared-memory opt-in of a kernel above 48 KB.  The attribute belongs to a device context, so it is set
// once per device (one bit of `done` per device index below 64; devices beyond that set it on every launch).  A
// failed call stays in the runtime's last error, which the caller's launch check reports.
template <class K>
inline void set_smem_attr(K* kernel, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess && bit)
    done.fetch_or(bit, std::memory_order_acq_rel);
}

template <class K>
inline void set_func_attr(K* kernel, cudaFuncAttribute attr, int value, std::atomic<uint64_t>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  if (cudaFuncSetAttribute(kernel, attr, value) == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
}

// status word bits written by the kernels
constexpr int32_t kStatusNonfinite = 1, kStatusTimeout = 2, kStatusFixRange = 4, kStatusBounds = 8;

// ROMAP_CHECKED build (compiled with -DROMAP_CHECKED into libromap_checked.so): device indices into pools, tables,
// ray and sample records and the tile plan are checked against their logical sizes; a failed check sets
// kStatusBounds in the status word and the access goes to a safe in-range index (or is skipped), never a trap.
#ifdef ROMAP_CHECKED
__device__ __forceinline__ bool bounds_ok(bool ok, int32_t* status) {
  if (!ok && status) atomicOr(status, kStatusBounds);
  return ok;
}
#define ROMAP_IN_BOUNDS(cond, status) ::romap::bounds_ok((cond), (status))
#else
#define ROMAP_IN_BOUNDS(cond, status) true
#endif
void launch_selftest_wait(int32_t* status, int limit, cudaStream_t stream);

}  // namespace romap
