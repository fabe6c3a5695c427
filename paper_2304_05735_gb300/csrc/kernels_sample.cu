// Ray sampling stage of the training step (Sec. V-B): ray draw, world ->
// object frame, ray/box slab test, stratified samples, occupancy culling and
// compaction; plus parameter initialisation.
//
// The FP32 arithmetic of this stage is written operation by operation with
// round-to-nearest intrinsics (no contraction into FMA) in one fixed order,
// so that sample positions and hash indices are reproducible bit for bit.
#include "device_common.cuh"
#include "romap_internal.cuh"

namespace romap {

__device__ inline uint32_t philox_word(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       int w) {
  return u4_word(philox(c0, c1, c2, c3, k0, k1), w);
}

// ---------------------------------------------------------------------------
// Parameter initialisation: hash entries U(-1e-4, 1e-4) (counter (k>>2, 0,
// INIT_HASH, 0), word k&3); MLP layer l (0..4, and 5..6 for the single-network
// model's extra hidden layers) Glorot-uniform with limit sqrt(6/(fan_in+fan_out))
// (counter (k>>2, l, INIT_MLP, 0), word k&3).
// ---------------------------------------------------------------------------
__global__ void k_init_params(GridParams g, float* params, uint32_t key0, uint32_t key1, float lim0, float lim1,
                              float lim2, float lim3, float lim4) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < g.n_params_pad; i += stride) {
    if (i >= g.n_params) { params[i] = 0.0f; continue; }
    uint32_t ctr1 = 0, purpose = kPurposeInitHash;
    int64_t k = i;
    float lim = 1e-4f;
    if (i >= g.n_hash) {
      int layer = 0;
#pragma unroll
      for (int l = 1; l < 7; ++l)
        if (i >= g.mlp_off[l]) layer = l;  // (layers 5, 6 exist only below n_params)
      k = i - g.mlp_off[layer];
      ctr1 = (uint32_t)layer;
      purpose = kPurposeInitMlp;
      // layers 3, 5 and 6 are all 64 x 64
      lim = layer == 0 ? lim0 : layer == 1 ? lim1 : layer == 2 ? lim2 : layer == 4 ? lim4 : lim3;
    }
    uint32_t x = philox_word((uint32_t)(k >> 2), ctr1, purpose, 0u, key0, key1, (int)(k & 3));
    float u = u01(x);
    params[i] = __fmul_rn(__fsub_rn(__fmul_rn(2.0f, u), 1.0f), lim);
  }
}

void launch_init_params(const GridParams& g, float* params, uint32_t key0, uint32_t key1, cudaStream_t stream) {
  int dims[5][2] = {{kH, g.LF}, {kDOut, kH}, {kH, g.cin}, {kH, kH}, {3, kH}};
  float lim[5];
  for (int l = 0; l < 5; ++l) lim[l] = (float)sqrt(6.0 / (double)(dims[l][0] + dims[l][1]));
  int blocks = (int)((g.n_params_pad + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_init_params<<<blocks, 256, 0, stream>>>(g, params, key0, key1, lim[0], lim[1], lim[2], lim[3], lim[4]);
}

// ---------------------------------------------------------------------------
// World -> object frame (Sec. IV-B pose: translation t, yaw about z):
// x_o = R_z^T (x_w - t), d_o = R_z^T d_w / |R_z^T d_w|.
// ---------------------------------------------------------------------------
// Ray r of the inputs -> ray w of the outputs.
__device__ __forceinline__ void transform_ray(const float* __restrict__ o_in, const float* __restrict__ d_in,
                                              const float* __restrict__ rgb_in, const float* __restrict__ depth_in,
                                              const uint8_t* __restrict__ cls_in, int64_t r, int object_frame,
                                              float tx, float ty, float tz, float cz, float sz, float* o_out,
                                              float* d_out, float* rgb_out, float* depth_out, uint8_t* cls_out,
                                              int64_t w) {
  float ox = o_in[3 * r], oy = o_in[3 * r + 1], oz = o_in[3 * r + 2];
  float dx = d_in[3 * r], dy = d_in[3 * r + 1], dz = d_in[3 * r + 2];
  float rx = dx, ry = dy, rz = dz;
  if (!object_frame) {
    float px = __fsub_rn(ox, tx), py = __fsub_rn(oy, ty), pz = __fsub_rn(oz, tz);
    ox = __fadd_rn(__fmul_rn(cz, px), __fmul_rn(sz, py));
    oy = __fsub_rn(__fmul_rn(cz, py), __fmul_rn(sz, px));
    oz = pz;
    rx = __fadd_rn(__fmul_rn(cz, dx), __fmul_rn(sz, dy));
    ry = __fsub_rn(__fmul_rn(cz, dy), __fmul_rn(sz, dx));
    rz = dz;
  }
  float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)), __fmul_rn(rz, rz)));
  o_out[3 * w] = ox; o_out[3 * w + 1] = oy; o_out[3 * w + 2] = oz;
  d_out[3 * w] = __fdiv_rn(rx, len);
  d_out[3 * w + 1] = __fdiv_rn(ry, len);
  d_out[3 * w + 2] = __fdiv_rn(rz, len);
  rgb_out[3 * w] = rgb_in ? rgb_in[3 * r] : 0.0f;
  rgb_out[3 * w + 1] = rgb_in ? rgb_in[3 * r + 1] : 0.0f;
  rgb_out[3 * w + 2] = rgb_in ? rgb_in[3 * r + 2] : 0.0f;
  depth_out[w] = depth_in ? depth_in[r] : __int_as_float(0x7fc00000);
  cls_out[w] = cls_in ? cls_in[r] : (uint8_t)kClsObject;
}

__global__ void k_transform_rays(const float* __restrict__ o_in, const float* __restrict__ d_in,
                                 const float* __restrict__ rgb_in, const float* __restrict__ depth_in,
                                 const uint8_t* __restrict__ cls_in, int64_t n, int object_frame, float tx, float ty,
                                 float tz, float cz, float sz, float* o_out, float* d_out, float* rgb_out,
                                 float* depth_out, uint8_t* cls_out) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  transform_ray(o_in, d_in, rgb_in, depth_in, cls_in, r, object_frame, tx, ty, tz, cz, sz, o_out, d_out, rgb_out,
                depth_out, cls_out, r);
}

// Several objects' rays, concatenated in the inputs: xo[k] (sorted by first, no empty ranges) says where object k's
// range starts, its pose and where its rays go in its pool.
__global__ void k_transform_rays_multi(const float* __restrict__ o_in, const float* __restrict__ d_in,
                                       const float* __restrict__ rgb_in, const float* __restrict__ depth_in,
                                       const uint8_t* __restrict__ cls_in, int64_t n, int object_frame,
                                       const XformObj* __restrict__ xo, int n_obj) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int lo = 0, hi = n_obj - 1;  // the last k with xo[k].first <= r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (xo[mid].first <= r) lo = mid;
    else hi = mid - 1;
  }
  const XformObj& x = xo[lo];
  transform_ray(o_in, d_in, rgb_in, depth_in, cls_in, r, object_frame, x.t[0], x.t[1], x.t[2], x.cz, x.sz, x.o_out,
                x.d_out, x.rgb_out, x.depth_out, x.cls_out, r - x.first);
}

void launch_transform_rays(const float* o_in, const float* d_in, const float* rgb_in, const float* depth_in,
                           const uint8_t* cls_in, int64_t n, int object_frame, float tx, float ty, float tz, float cz,
                           float sz, float* o_out, float* d_out, float* rgb_out, float* depth_out, uint8_t* cls_out,
                           cudaStream_t stream) {
  if (n <= 0) return;
  int64_t blocks = (n + 255) / 256;
  k_transform_rays<<<(unsigned)blocks, 256, 0, stream>>>(o_in, d_in, rgb_in, depth_in, cls_in, n, object_frame, tx,
                                                         ty, tz, cz, sz, o_out, d_out, rgb_out, depth_out, cls_out);
}

void launch_transform_rays_multi(const float* o_in, const float* d_in, const float* rgb_in, const float* depth_in,
                                 const uint8_t* cls_in, int64_t n, int object_frame, const XformObj* xo, int n_obj,
                                 cudaStream_t stream) {
  if (n <= 0 || n_obj <= 0) return;
  int64_t blocks = (n + 255) / 256;
  k_transform_rays_multi<<<(unsigned)blocks, 256, 0, stream>>>(o_in, d_in, rgb_in, depth_in, cls_in, n, object_frame,
                                                               xo, n_obj);
}

// Block-wide exclusive scan of 256 values.
__device__ inline uint32_t block_excl_scan256(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[8];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint32_t base = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < w) base += warp_tot[i];
    tot += warp_tot[i];
  }
  *total = tot;
  __syncthreads();
  return base + incl - v;
}

struct RayCtx {
  int bi, rl, r;
  bool valid;
};

__device__ inline RayCtx ray_of_thread(const BatchDesc& b) {
  RayCtx c;
  c.bi = b.block_obj[blockIdx.x];
  int local_block = blockIdx.x - b.block_base[c.bi];
  c.rl = local_block * 256 + threadIdx.x;
  int n = b.ray_base[c.bi + 1] - b.ray_base[c.bi];
  c.valid = c.rl < n;
  c.r = b.ray_base[c.bi] + c.rl;
  return c;
}

// ---------------------------------------------------------------------------
// Ray draw + slab + live-sample count.  One block of 256 ray slots of one
// batch object.  Draw: slot s of an object takes pool index s when the whole
// pool is used, else mulhi32(Philox(step, s, RAY, 0).x, pool size); its
// background is u01 of Philox(step, s, BG, 0) words 0..2 when random.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_ray_setup(GridParams g, BatchDesc b, RayBuf R, uint32_t* block_sums) {
  __shared__ uint32_t s_cnt[kPlanCounts];
  if (b.plan && threadIdx.x < kPlanCounts) s_cnt[threadIdx.x] = 0u;
  RayCtx c = ray_of_thread(b);
  const ObjectDev& ob = b.objs[b.slot[c.bi]];
  uint32_t count = 0;
  uint32_t m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;  // live candidates (tile plan of the mixed-precision path, N <= 128)
  if (c.valid) {
    float o[3], d[3], bg[3];
    uint32_t step = b.explicit_rays ? b.explicit_step : ob.step;
    if (b.explicit_rays) {
      for (int a = 0; a < 3; ++a) {
        o[a] = b.ex_o[3 * c.r + a];
        d[a] = b.ex_d[3 * c.r + a];
        bg[a] = b.ex_bg[3 * c.r + a];
      }
      R.rgb[3 * c.r] = R.rgb[3 * c.r + 1] = R.rgb[3 * c.r + 2] = 0.0f;
      R.depth[c.r] = __int_as_float(0x7fc00000);
      R.cls[c.r] = kClsObject;
      R.pool_idx[c.r] = c.rl;
    } else {
      int64_t p;
      if (ob.whole_pool) {
        p = c.rl;
      } else {
        uint32_t x = philox(step, (uint32_t)c.rl, kPurposeRay, 0u, ob.key0, ob.key1).x;
        p = (int64_t)(((uint64_t)x * (uint64_t)ob.pool_n) >> 32);
      }
      if (!ROMAP_IN_BOUNDS(p >= 0 && p < ob.pool_n, g.status)) p = 0;
      for (int a = 0; a < 3; ++a) {
        o[a] = ob.pool_o[3 * p + a];
        d[a] = ob.pool_d[3 * p + a];
        R.rgb[3 * c.r + a] = ob.pool_rgb[3 * p + a];
      }
      R.depth[c.r] = ob.pool_depth[p];
      R.cls[c.r] = ob.pool_cls[p];
      R.pool_idx[c.r] = p;
      if (g.bg_random) {
        U4 w = philox(step, (uint32_t)c.rl, kPurposeBg, 0u, ob.key0, ob.key1);
        bg[0] = u01(w.x); bg[1] = u01(w.y); bg[2] = u01(w.z);
      } else {
        bg[0] = g.bg_const[0]; bg[1] = g.bg_const[1]; bg[2] = g.bg_const[2];
      }
    }
    float tn, tf;
    bool hit = slab(o, d, ob.half, tn, tf);
    if (hit) {
      if (!ob.occ) {
        count = (uint32_t)g.n_samples;
        if (b.plan) {
          auto first = [&](int lo) {
            return g.n_samples >= lo + 32 ? 0xffffffffu : (g.n_samples > lo ? (1u << (g.n_samples - lo)) - 1u : 0u);
          };
          m0 = first(0); m1 = first(32); m2 = first(64); m3 = first(96);
        }
      } else {
        for_candidates(o, d, tn, tf, g.n_samples, ob.key0, ob.key1, step, (uint32_t)c.rl, b.jitter, ob.occ, ob.half,
                       ob.inv_ext, [&](int i, float, float, float, float, float, bool live) {
                         if (live) {
                           ++count;
                           if (b.plan) {
                             const uint32_t bit = 1u << (i & 31);
                             const int wd = i >> 5;
                             m0 |= wd == 0 ? bit : 0u; m1 |= wd == 1 ? bit : 0u;
                             m2 |= wd == 2 ? bit : 0u; m3 |= wd == 3 ? bit : 0u;
                           }
                         }
                       });
      }
    }
    for (int a = 0; a < 3; ++a) {
      R.o[3 * c.r + a] = o[a];
      R.d[3 * c.r + a] = d[a];
      R.bg[3 * c.r + a] = bg[a];
    }
    R.tn[c.r] = tn;
    R.tf[c.r] = hit ? tf : tn;
    R.count[c.r] = count;
    R.obj[c.r] = c.bi;
    if (b.plan) *reinterpret_cast<uint4*>(R.mask + 4 * c.r) = make_uint4(m0, m1, m2, m3);
  }
  if (b.plan) {  // rays of each live count in this block, added to the entry's histogram; the block's offset within
                 // each count is the histogram value it found (the order of the blocks within a count is arbitrary)
    __syncthreads();
    if (c.valid) atomicAdd(&s_cnt[count], 1u);
    __syncthreads();
    if (threadIdx.x < kPlanCounts) {
      const uint32_t v = s_cnt[threadIdx.x];
      b.plan_bcnt[blockIdx.x * kPlanCounts + threadIdx.x] =
          v ? atomicAdd(&b.plan_hist[(size_t)c.bi * kPlanCounts + threadIdx.x], v) : 0u;
    }
  }
  uint32_t total;
  uint32_t excl = block_excl_scan256(count, &total);
  if (c.valid) R.off[c.r] = excl;
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

void launch_ray_setup(const GridParams& g, const BatchDesc& b, RayBuf r, uint32_t* block_sums, cudaStream_t stream) {
  if (b.n_blocks <= 0) return;
  k_ray_setup<<<b.n_blocks, 256, 0, stream>>>(g, b, r, block_sums);
}

// ---------------------------------------------------------------------------
// Per-object offsets: each warp scans the block totals of its objects; one
// block-wide scan over tile counts places every object on a tile boundary.
// Padding samples up to the tile boundary get ray = kNoRay.
// ---------------------------------------------------------------------------
constexpr int kMaxBatch = 1024;

// Largest c <= lim whose bit is set in the 160-bit mask m (bit c of word c / 32), or -1.
__device__ __forceinline__ int highest_set_at_most(const uint32_t m[5], int lim) {
  if (lim < 0) return -1;
  int q = lim >> 5;
  const int bit = lim & 31;
  uint32_t x = m[q] & (bit == 31 ? 0xffffffffu : ((2u << bit) - 1u));
  while (x == 0u && q > 0) x = m[--q];
  return x ? 32 * q + 31 - __clz(x) : -1;
}

// Tile plan (mixed-precision path), run by the single block of k_scan.  Per batch entry (one warp each): the block
// offsets of every live count within the entry (in place in plan_bcnt) and the count histogram; then the patterns
// (greedy over the histogram, see kPlanMaxCount) with their segments.  The warp computes every pattern in lockstep
// (all lanes read the same shared values); lane 0 writes the records.  Then the entries' even tile counts are
// scanned into first tiles and every tile record is written.  s_tiles and s_wsum are scratch.
// Tile patterns of one batch entry (one warp per block, one block per entry): the entry's count histogram (then
// reset for the next step), the greedy patterns (see kPlanMaxCount) and their segments.  Lane l keeps the state of
// counts c = 32 k + l (k = 0..4) in registers: rays not placed yet, rays placed so far (the next segment's first
// rank) and its segment count.  Every lane builds the same pattern (uniform values, shuffles from the owner lanes);
// then each owner lane writes the segment of its count and lane 0 the pattern record.
__device__ __forceinline__ int pick5(const int v[5], int k) {
  return k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : k == 3 ? v[3] : v[4];
}

__global__ void __launch_bounds__(32) k_plan_patterns(BatchDesc b) {
  __shared__ int8_t item_of[160];                   // item of the pattern being built holding count c, or -1
  __shared__ uint8_t ia[kPlanMaxCount];             // copies of each item
  __shared__ uint8_t io_slot[kPlanMaxCount], io_perm[kPlanMaxCount];  // slot / ray offset of its first copy
  const int lane = threadIdx.x, i = blockIdx.x;
  int h[5], cons[5], ns[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int c = 32 * k + lane;
    h[k] = 0;
    if (c < kPlanCounts) {
      uint32_t* hp = b.plan_hist + (size_t)i * kPlanCounts + c;
      h[k] = c >= 1 ? (int)*hp : 0;
      *hp = 0u;
    }
    cons[k] = 0;
    ns[k] = 0;
    item_of[c] = -1;
  }
  __syncwarp();
  int4* pat = b.plan_pat + (size_t)i * kPlanMaxPat * 2;
  int4* seg = b.plan_seg + (size_t)i * kPlanCounts * kPlanSegsPerCount * 2;
  int npat = 0, T = 0, PB = 0;
  bool fallback = false;
  for (;;) {
    uint32_t m[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) m[k] = __ballot_sync(0xffffffffu, h[k] > 0);
    if (!(m[0] | m[1] | m[2] | m[3] | m[4])) break;
    if (npat >= kPlanMaxPat - kPlanCounts - 1) {
      fallback = true;
      break;
    }
    // one pattern: the largest remaining count opens the tile, then the largest counts that still fit
    int rem = kTile, lim = kPlanMaxCount, ni = 0, nrays = 0, rep = 0x7fffffff;
    bool seg_full = false;
    for (;;) {
      const int c = highest_set_at_most(m, rem < lim ? rem : lim);
      if (c <= 0) break;
      const int k = c >> 5, src = c & 31;
      const int hv = __shfl_sync(0xffffffffu, pick5(h, k), src);
      const int nsv = __shfl_sync(0xffffffffu, pick5(ns, k), src);
      const int a = hv < rem / c ? hv : rem / c;
      if (lane == 0) {
        item_of[c] = (int8_t)ni;
        ia[ni] = (uint8_t)a;
        io_slot[ni] = (uint8_t)(kTile - rem);
        io_perm[ni] = (uint8_t)nrays;
      }
      rep = min(rep, hv / a);
      seg_full = seg_full || nsv >= kPlanSegsPerCount - 1;  // keep one segment per count for the fallback
      ++ni;
      nrays += a;
      rem -= a * c;
      lim = c - 1;
    }
    __syncwarp();
    if (seg_full) {
#pragma unroll
      for (int k = 0; k < 5; ++k) item_of[32 * k + lane] = -1;
      __syncwarp();
      fallback = true;
      break;
    }
    // segments: each count's owner lane; the pattern record: lane 0
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int c = 32 * k + lane;
      const int q = item_of[c];
      if (q >= 0) {
        const int a = ia[q];
        int4* sg = seg + ((size_t)c * kPlanSegsPerCount + ns[k]) * 2;
        sg[0] = make_int4(cons[k], T, a, rep);
        sg[1] = make_int4(io_slot[q], io_perm[q], nrays, PB);
        ns[k] += 1;
        cons[k] += rep * a;
        h[k] -= rep * a;
        item_of[c] = -1;
      }
    }
    if (lane == 0) {
      pat[2 * npat] = make_int4(T, rep, nrays, PB);
      pat[2 * npat + 1] = make_int4(rep * nrays, kTile - rem, 0, 0);
    }
    __syncwarp();
    T += rep;
    PB += rep * nrays;
    ++npat;
  }
  if (fallback) {  // every count left in tiles of its own: floor(128 / c) rays of count c per tile
    for (int c = kPlanMaxCount; c >= 1; --c) {
      const int k = c >> 5, src = c & 31;
      const int rays = __shfl_sync(0xffffffffu, pick5(h, k), src);
      if (rays <= 0) continue;
      const int a = kTile / c, tiles = (rays + a - 1) / a;
      if (lane == src) {
        int4* sg = seg + ((size_t)c * kPlanSegsPerCount + pick5(ns, k)) * 2;
        sg[0] = make_int4(pick5(cons, k), T, a, tiles);
        sg[1] = make_int4(0, 0, a, PB);
#pragma unroll
        for (int kk = 0; kk < 5; ++kk)
          if (kk == k) {
            ns[kk] += 1;
            cons[kk] += rays;
            h[kk] = 0;
          }
      }
      if (lane == 0) {
        pat[2 * npat] = make_int4(T, tiles, a, PB);
        pat[2 * npat + 1] = make_int4(rays, a * c, c, 0);
      }
      T += tiles;
      PB += rays;
      ++npat;
    }
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int c = 32 * k + lane;
    if (c < kPlanCounts) b.plan_nseg[(size_t)i * kPlanCounts + c] = ns[k];
  }
  if (lane == 0) {
    b.plan_npat[i] = npat;
    b.plan_ent[i] = (T + 1) & ~1;  // even: a pair never mixes entries (the scan turns it into the first tile)
  }
}

// Tile plan (mixed-precision path), run by the single block of k_scan after k_plan_patterns: the entries' even tile
// counts are scanned into first tiles and every tile record is written.  s_tiles and s_wsum are scratch.
__device__ void plan_tiles_of_batch(const BatchDesc& b, uint32_t* s_tiles, uint32_t* s_wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (threadIdx.x < (unsigned)b.n) s_tiles[threadIdx.x] = (uint32_t)b.plan_ent[threadIdx.x];
  __syncthreads();
  // exclusive scan of the entries' tile counts
  const uint32_t v = threadIdx.x < (unsigned)b.n ? s_tiles[threadIdx.x] : 0u;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) s_wsum[w] = incl;
  __syncthreads();
  uint32_t base = 0, all = 0;
  for (int k = 0; k < 32; ++k) {
    if (k < w) base += s_wsum[k];
    all += s_wsum[k];
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)b.n) {
    s_tiles[threadIdx.x] = base + incl - v;  // first tile of entry i
    b.plan_ent[threadIdx.x] = (int32_t)(base + incl - v);
  }
  if (threadIdx.x == 0) b.plan_npairs[0] = (int32_t)(all / 2);
  __syncthreads();
  for (int i = w; i < b.n; i += 32) {
    const int4* pat = b.plan_pat + (size_t)i * kPlanMaxPat * 2;
    const int npat = b.plan_npat[i];
    const int t0 = (int)s_tiles[i];
    const int nt = (int)((i + 1 < b.n ? s_tiles[i + 1] : all) - s_tiles[i]);
    for (int t = lane; t < nt; t += 32) {
      int lo = 0, hi = npat - 1, p = -1;  // the last pattern whose first tile is at or before t
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (pat[2 * mid].x <= t) { p = mid; lo = mid + 1; } else { hi = mid - 1; }
      }
      int4 rec = make_int4(i, t0 + t, 0, b.ray_base[i]);  // padding tile: no rays, no used slots
      if (p >= 0) {
        const int4 P0 = pat[2 * p], P1 = pat[2 * p + 1];
        const int q = t - P0.x;
        if (q < P0.y) {
          const int nr = min(P0.z, P1.x - q * P0.z);
          const int used = P1.z > 0 ? nr * P1.z : P1.y;
          rec = make_int4(i, t0 + t, nr | (used << 8), b.ray_base[i] + P0.w + q * P0.z);
        }
      }
      b.plan_tiles[t0 + t] = rec;
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan(BatchDesc b, uint32_t* block_sums, BatchDyn* dyn, int32_t* totals,
                                               SampleBuf S, unsigned long long* live_counter) {
  __shared__ uint32_t s_count[kMaxBatch];
  __shared__ uint32_t s_tiles[kMaxBatch];
  __shared__ uint32_t s_wsum[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = w; i < b.n; i += 32) {
    int bb = b.block_base[i], nb = b.block_base[i + 1] - bb;
    uint32_t carry = 0;
    for (int c = 0; c < nb; c += 32) {
      uint32_t v = (c + lane < nb) ? block_sums[bb + c + lane] : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
      }
      if (c + lane < nb) block_sums[bb + c + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      s_count[i] = carry;
      s_tiles[i] = (carry + kTile - 1) / kTile;
    }
  }
  __syncthreads();
  // exclusive scan of s_tiles over batch entries (n <= 1024)
  uint32_t v = threadIdx.x < (unsigned)b.n ? s_tiles[threadIdx.x] : 0u;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) s_wsum[w] = incl;
  __syncthreads();
  uint32_t base = 0, all = 0;
  for (int i = 0; i < 32; ++i) {
    if (i < w) base += s_wsum[i];
    all += s_wsum[i];
  }
  uint32_t tile_base = base + incl - v;
  if (threadIdx.x < (unsigned)b.n) {
    int i = threadIdx.x;
    BatchDyn dd;
    dd.tile_base = (int32_t)tile_base;
    dd.n_tiles = (int32_t)v;
    dd.sample_base = (int64_t)tile_base * kTile;
    dd.n_samples = (int32_t)s_count[i];
    dd.pad_ = 0;
    for (int k = 0; k < 5; ++k) {
      dd.loss[k] = 0.0f;
      dd.loss_fix[k] = 0ull;
    }
    dd.pad2_[0] = dd.pad2_[1] = dd.pad2_[2] = 0.0f;
    dd.pad3_ = 0;
    dyn[i] = dd;
  }
  if (threadIdx.x < (unsigned)b.n) s_tiles[threadIdx.x] = tile_base;  // now the first tile of entry i
  __syncthreads();
  // padding samples of every entry up to its tile boundary
  for (int i = w; i < b.n; i += 32) {
    uint32_t cnt = s_count[i];
    uint32_t n_tiles = (cnt + kTile - 1) / kTile;
    uint32_t pad = n_tiles * kTile - cnt;
    int64_t start = (int64_t)s_tiles[i] * kTile + cnt;
    if (S.ray)
      for (uint32_t j = lane; j < pad; j += 32) S.ray[start + j] = kNoRay;
  }
  if (threadIdx.x == 0) {
    totals[0] = (int32_t)all;
    uint64_t tot = 0;
    for (int i = 0; i < b.n; ++i) tot += s_count[i];
    totals[1] = (int32_t)tot;
    if (live_counter) atomicAdd(live_counter, (unsigned long long)tot);
  }
  if (b.plan) plan_tiles_of_batch(b, s_tiles, s_wsum);
}

void launch_plan_patterns(const BatchDesc& b, cudaStream_t stream) {
  if (b.n <= 0) return;
  k_plan_patterns<<<b.n, 32, 0, stream>>>(b);
}

void launch_scan(const GridParams&, const BatchDesc& b, uint32_t* block_sums, BatchDyn* dyn, int32_t* totals,
                 SampleBuf s, unsigned long long* live_counter, cudaStream_t stream) {
  k_scan<<<1, 1024, 0, stream>>>(b, block_sums, dyn, totals, s, live_counter);
}

// ---------------------------------------------------------------------------
// Write the live samples of every ray at its compacted offset.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_write_samples(GridParams g, BatchDesc b, RayBuf R, const uint32_t* block_sums,
                                                       const BatchDyn* dyn, SampleBuf S) {
  RayCtx c = ray_of_thread(b);
  if (!c.valid) return;
  const ObjectDev& ob = b.objs[b.slot[c.bi]];
  uint32_t off = (uint32_t)(dyn[c.bi].sample_base + block_sums[blockIdx.x] + R.off[c.r]);
  R.off[c.r] = off;
  uint32_t count = R.count[c.r];
  if (count == 0) return;
  float o[3] = {R.o[3 * c.r], R.o[3 * c.r + 1], R.o[3 * c.r + 2]};
  float d[3] = {R.d[3 * c.r], R.d[3 * c.r + 1], R.d[3 * c.r + 2]};
  uint32_t step = b.explicit_rays ? b.explicit_step : ob.step;
  uint32_t j = off;
  for_candidates(o, d, R.tn[c.r], R.tf[c.r], g.n_samples, ob.key0, ob.key1, step, (uint32_t)c.rl, b.jitter, ob.occ,
                 ob.half, ob.inv_ext, [&](int i, float t, float dt, float x, float y, float z, bool live) {
                   if (!live) return;
                   S.x[3 * (size_t)j] = x;
                   S.x[3 * (size_t)j + 1] = y;
                   S.x[3 * (size_t)j + 2] = z;
                   S.t[j] = t;
                   S.dt[j] = dt;
                   S.ray[j] = (uint32_t)c.r;
                   S.cand[j] = (uint32_t)i;
                   ++j;
                 });
}

void launch_write_samples(const GridParams& g, const BatchDesc& b, RayBuf r, const uint32_t* block_sums,
                          const BatchDyn* dyn, SampleBuf s, cudaStream_t stream) {
  if (b.n_blocks <= 0) return;
  k_write_samples<<<b.n_blocks, 256, 0, stream>>>(g, b, r, block_sums, dyn, s);
}

// ---------------------------------------------------------------------------
// Scatter per-sample values into per-slot arrays [ray * N + candidate].
// ---------------------------------------------------------------------------
__global__ void k_scatter_slots(int n_samples_per_ray, int64_t n_rays, RayBuf R, SampleBuf S, const float* src,
                                int src_stride, float* dst, int dst_stride) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  uint32_t cnt = R.count[r], off = R.off[r];
  for (uint32_t j = 0; j < cnt; ++j) {
    uint32_t s = off + j;
    int64_t slot = r * n_samples_per_ray + S.cand[s];
    for (int k = 0; k < dst_stride; ++k) dst[slot * dst_stride + k] = src[(int64_t)s * src_stride + k];
  }
}

void launch_scatter_slots(const GridParams& g, int64_t n_rays, const RayBuf r, const SampleBuf s, const float* src,
                          int src_stride, float* dst, int dst_stride, cudaStream_t stream) {
  if (n_rays <= 0) return;
  k_scatter_slots<<<(unsigned)((n_rays + 255) / 256), 256, 0, stream>>>(g.n_samples, n_rays, r, s, src, src_stride,
                                                                        dst, dst_stride);
}

// Per slot [ray * N + candidate] x 6: t, delta, x, y, z, sigma.
__global__ void k_sample_slots(int n_samples_per_ray, int64_t n_rays, RayBuf R, SampleBuf S, float* dst) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  uint32_t cnt = R.count[r], off = R.off[r];
  for (uint32_t j = 0; j < cnt; ++j) {
    uint32_t s = off + j;
    float* o = dst + (r * n_samples_per_ray + S.cand[s]) * 6;
    o[0] = S.t[s]; o[1] = S.dt[s];
    o[2] = S.x[3 * (size_t)s]; o[3] = S.x[3 * (size_t)s + 1]; o[4] = S.x[3 * (size_t)s + 2];
    o[5] = S.sigma[s];
  }
}

void launch_sample_slots(const GridParams& g, int64_t n_rays, const RayBuf r, const SampleBuf s, float* dst,
                         cudaStream_t stream) {
  if (n_rays <= 0) return;
  k_sample_slots<<<(unsigned)((n_rays + 255) / 256), 256, 0, stream>>>(g.n_samples, n_rays, r, s, dst);
}

}  // namespace romap
