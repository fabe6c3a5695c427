// Warp-specialized variant of the mixed-precision fused tile kernel (same arithmetic as kernels_tc.cu; see the
// operand layouts there).  The per-tile work splits into two roles that run concurrently in one CTA of 256 threads:
//   * compute warps 0-3 (thread s <-> sample slot s <-> TMEM lane s): the ten tcgen05.mma groups of the forward and
//     backward MLP with their epilogues, volume rendering, losses and adjoint, and the weight-gradient accumulation
//     in TMEM; thread 0 issues every MMA of the CTA, so accumulations into the shared TMEM columns stay in order;
//   * memory warps 4-7: the sample positions and FP16 hash gathers of the next tile, and the hash-gradient scatter
//     (vector REDs) of the tile finished before, reading dL/dencoding from a shared-memory staging row.
// Two tile slots in shared memory hand tiles from one role to the other: full[slot] (memory -> compute, 128
// arrivals after the encoding rows are written and fenced for the async proxy) and empty[slot] (compute -> memory,
// 128 arrivals after the encoding gradient is staged).  The random-access work of the memory warps, bound by L1/L2
// request throughput, overlaps the latency-bound chain of MMA round trips of the compute warps.
// Every wait is bounded; on time-out the kernel records ROMAP_ERR_TIMEOUT, lets its MMAs drain (bounded), frees its
// tensor memory and returns.
#include <cstddef>

#include "tc_common.cuh"

namespace romap {
namespace {
using namespace tc;

constexpr int kWsThreads = 256;  // 4 compute warps + 4 memory warps
constexpr int kCompute = 128;

template <int LFP>
struct WsSlot {
  // activation buffers: contiguous and in this order (the MN-major A operands of the weight-gradient GEMMs, 64
  // features with M padded to 128, read up to 1 KB past their buffer into the next one of the slot)
  __align__(128) unsigned char E[kT * LFP * 2];
  __align__(128) unsigned char H1[kT * kH * 2];
  __align__(128) unsigned char CIN[kT * 32 * 2];
  __align__(128) unsigned char H2[kT * kH * 2];
  __align__(128) unsigned char H3[kT * kH * 2];
  __align__(128) unsigned char DL[kT * 16 * 2];
  float px[3][kT];
  float t[kT];
  float dt[kT];
  float sig[kT];
  float o0[kT];
  float rgb[3][kT];
  float dsig[kT];
  float drgb[3][kT];
  int valid[kT];
  int ray[kT];            // global ray index of the slot (-1 outside the tile's rays)
  __align__(16) float dE[kT][LFP + 4];  // dL/dencoding staged for the scatter (padded rows: float4 access)
  int pfirst, nrays, bi;  // first plan_perm index, rays and batch entry of the tile
};

template <int LFP>
struct WsSmem {
  __align__(128) unsigned char w1[kH * LFP * 2];
  __align__(128) unsigned char w2[16 * kH * 2];
  __align__(128) unsigned char w3[kH * 32 * 2];
  __align__(128) unsigned char w4[kH * kH * 2];
  __align__(128) unsigned char w5[16 * kH * 2];
  WsSlot<LFP> slot[2];
  __align__(8) uint64_t mma_bar;
  __align__(8) uint64_t full_bar[2];
  __align__(8) uint64_t empty_bar[2];
  uint32_t tmem_base;
  int fail;    // set by any thread whose bounded wait gave up
  int c_stop;  // the compute warps' copy of fail: written by compute thread 0 before a compute barrier only
};

__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, %0;" ::"n"(kCompute) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epi_relu64(uint32_t taddr, unsigned char* buf, int row, bool f16) {
  float v[64];
#pragma unroll
  for (int c = 0; c < 4; ++c) tmem_ld16(taddr + 16 * c, v + 16 * c);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 64; ++j) v[j] = fmaxf(v[j], 0.f);
#pragma unroll
  for (int c = 0; c < 8; ++c) store8(buf, row, c, kH, v + 8 * c, f16);
}
__device__ __forceinline__ void epi_mask64(uint32_t taddr, unsigned char* buf, int row, bool f16) {
  float v[64];
#pragma unroll
  for (int c = 0; c < 4; ++c) tmem_ld16(taddr + 16 * c, v + 16 * c);
  tmem_wait_ld();
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float h[8];
    load8(buf, row, c, kH, h, f16);
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = h[j] > 0.f ? v[8 * c + j] : 0.f;
    store8(buf, row, c, kH, h, f16);
  }
}

// ---------------------------------------------------------------------------------------------------------------
// memory warps: scatter the tile that left a slot, then gather the next tile into it
// ---------------------------------------------------------------------------------------------------------------
template <int LFP, bool F16>
__device__ void memory_role(WsSmem<LFP>& sm, const GridParams& g, const BatchDesc& b, const RayBuf& R,
                            const WorkOrder& wo, int n) {
  const int s = threadIdx.x - kCompute;
  constexpr int LMAX = LFP / 2;
  constexpr bool f16 = F16;
  for (int k = 0; k < n + 2; ++k) {
    if (sm.fail) break;
    const int slot = k & 1;
    WsSlot<LFP>& sl = sm.slot[slot];
    if (k >= 2) {
      if (!mbar_wait(&sm.empty_bar[slot], ((k - 2) >> 1) & 1)) {
        sm.fail = 1;
        break;
      }
      if (sl.valid[s]) {
        const ObjectDev* ob = &b.objs[b.slot[b.plan_tiles[wo.item(k - 2)].x]];
        const float p[3] = {sl.px[0][s], sl.px[1][s], sl.px[2][s]};
        float2* gt = reinterpret_cast<float2*>(ob->grad);
        float de[LFP];
#pragma unroll
        for (int c = 0; c < LFP / 4; ++c) {
          const float4 q = *reinterpret_cast<const float4*>(&sl.dE[s][4 * c]);
          de[4 * c] = q.x; de[4 * c + 1] = q.y; de[4 * c + 2] = q.z; de[4 * c + 3] = q.w;
        }
#pragma unroll
        for (int l = 0; l < LMAX; ++l) {
          const float d0 = de[2 * l], d1 = de[2 * l + 1];
          if (l >= g.L || (d0 == 0.f && d1 == 0.f)) continue;
          Corners c;
          level_corners(g, l, p, ob->half, ob->inv_ext, c);
          scatter_corners(gt + g.off[l], c.idx, c.w, d0, d1);
        }
      }
    }
    if (k < n) {
      const int4 ti = b.plan_tiles[wo.item(k)];
      const ObjectDev* ob = &b.objs[b.slot[ti.x]];
      const SlotSample q = plan_sample(g, b, R, ob, ti.x, ti, s);
      if (s == 0) {
        sl.pfirst = ti.w;
        sl.nrays = ti.z & 255;
        sl.bi = ti.x;
      }
      sl.ray[s] = q.ray;
      sl.valid[s] = q.valid;
      sl.px[0][s] = q.x; sl.px[1][s] = q.y; sl.px[2][s] = q.z;
      sl.t[s] = q.t;
      sl.dt[s] = q.dt;
      float e[LFP];
#pragma unroll
      for (int c = 0; c < LFP; ++c) e[c] = 0.f;
      if (q.valid) {
        const float p[3] = {q.x, q.y, q.z};
        gather_levels<LFP, 0, LMAX>(g, ob, p, e);
      }
#pragma unroll
      for (int c = 0; c < LFP / 8; ++c) store8(sl.E, s, c, LFP, e + 8 * c, f16);
      fence_async_smem();
      mbar_arrive(&sm.full_bar[slot]);
    }
  }
}

// ---------------------------------------------------------------------------------------------------------------
// compute warps: forward, compositing, backward of one tile at a time
// ---------------------------------------------------------------------------------------------------------------
template <int LFP, bool F16>
__device__ void compute_role(WsSmem<LFP>& sm, const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf R,
                             int32_t* status, int n, uint32_t& phase, bool& pending) {
  const int s = threadIdx.x, warp = s >> 5;
  const uint32_t tm = sm.tmem_base;
  // FP16 operands: gradient operands scaled by the object's batch size B, FP32 results unscaled (as the lockstep
  // kernel)
  constexpr bool f16 = F16;
  auto unscale_of = [&](int bi_) { return f16 ? 1.0f / (float)(b.ray_base[bi_ + 1] - b.ray_base[bi_]) : 1.0f; };
  const uint32_t tmp = tm + ((uint32_t)(32 * warp) << 16) + kColTmp;
  const uint32_t dtmp = tm + kColTmp;
  auto sync_then_issue = [&]() {
    fence_async_smem();
    tc_before();
    bar_compute();
    tc_after();
  };
  // Every stop decision of the compute warps reads c_stop after a compute barrier, so that all of them take the
  // same branch (fail itself may change at any time).
  auto wait_mma = [&]() -> bool {
    if (s == 0) {
      if (!mbar_wait(&sm.mma_bar, phase)) sm.fail = 1;
      sm.c_stop = sm.fail;
    }
    phase ^= 1u;
    bar_compute();
    tc_after();
    pending = sm.c_stop != 0;
    return sm.c_stop == 0;
  };
  int bi = -1;
  const ObjectDev* ob = nullptr;
  uint32_t acc_dw = 0;
  for (int k = 0; k < n; ++k) {
    const int slot = k & 1;
    WsSlot<LFP>& sl = sm.slot[slot];
    if (s == 0) {
      if (!mbar_wait(&sm.full_bar[slot], (k >> 1) & 1)) sm.fail = 1;
      sm.c_stop = sm.fail;
    }
    bar_compute();
    if (sm.c_stop) break;
    const int nbi = sl.bi;
    if (nbi != bi) {
      if (bi >= 0) flush_dw<LFP>(tm, g, ob->grad, unscale_of(bi), kCompute);
      bi = nbi;
      ob = &b.objs[b.slot[bi]];
      load_weights<LFP, 20>(sm, g, ob->params, s, kCompute);
      acc_dw = 0;
    }
    const int n_rays_obj = b.ray_base[bi + 1] - b.ray_base[bi];
    const float invB = 1.0f / (float)n_rays_obj;
    const float gscale = f16 ? (float)n_rays_obj : 1.0f, gunscale = f16 ? invB : 1.0f;
    sync_then_issue();
    // ---- forward ----
    if (s == 0) {
      pending = true;
#pragma unroll
      for (int kk = 0; kk < LFP / 16; ++kk)
        mma(dtmp, desc_k(sl.E, LFP, kk), desc_k(sm.w1, LFP, kk), idesc(64, 0, 0, f16), kk > 0);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    epi_relu64(tmp, sl.H1, s, f16);
    sync_then_issue();
    if (s == 0) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma(dtmp, desc_k(sl.H1, kH, kk), desc_k(sm.w2, kH, kk), idesc(16, 0, 0, f16), kk > 0);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    {
      float v[16];
      tmem_ld16(tmp, v);
      tmem_wait_ld();
      const float o0 = v[0];
      sl.o0[s] = o0;
      sl.sig[s] = expf(fminf(fmaxf(o0, -15.f), 15.f));
      float cin[32];
#pragma unroll
      for (int j = 0; j < 15; ++j) cin[j] = v[1 + j];
      float d0 = 0.f, d1 = 0.f, d2 = 0.f;
      if (g.dir_dims == 3 && sl.valid[s]) {
        const int64_t r = sl.ray[s];
        d0 = R.d[3 * r]; d1 = R.d[3 * r + 1]; d2 = R.d[3 * r + 2];
      }
      cin[15] = d0; cin[16] = d1; cin[17] = d2;
#pragma unroll
      for (int j = 18; j < 32; ++j) cin[j] = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) store8(sl.CIN, s, c, 32, cin + 8 * c, f16);
    }
    sync_then_issue();
    if (s == 0) {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) mma(dtmp, desc_k(sl.CIN, 32, kk), desc_k(sm.w3, 32, kk), idesc(64, 0, 0, f16), kk > 0);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    epi_relu64(tmp, sl.H2, s, f16);
    sync_then_issue();
    if (s == 0) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma(dtmp, desc_k(sl.H2, kH, kk), desc_k(sm.w4, kH, kk), idesc(64, 0, 0, f16), kk > 0);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    epi_relu64(tmp, sl.H3, s, f16);
    sync_then_issue();
    if (s == 0) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma(dtmp, desc_k(sl.H3, kH, kk), desc_k(sm.w5, kH, kk), idesc(16, 0, 0, f16), kk > 0);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    {
      float v[16];
      tmem_ld16(tmp, v);
      tmem_wait_ld();
      sl.rgb[0][s] = 1.0f / (1.0f + expf(-v[0]));
      sl.rgb[1][s] = 1.0f / (1.0f + expf(-v[1]));
      sl.rgb[2][s] = 1.0f / (1.0f + expf(-v[2]));
    }
    bar_compute();
    // ---- compositing, losses, adjoint: one warp per ray ----
    {
      auto tile_of = [&](int) -> WsSlot<LFP>& { return sl; };
      composite_rays(tile_of, sl.nrays, sl.nrays, warp, kCompute / 32, g, b, R, dyn, bi, invB, status);
    }
    bar_compute();
    // ---- backward ----
    float dpre;
    {
      const bool valid = sl.valid[s];
      float dl[16];
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) dl[k2] = 0.f;
      if (valid) {
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) {
          const float c = sl.rgb[k2][s];
          dl[k2] = sl.drgb[k2][s] * c * (1.f - c);
        }
      }
      const float o0 = sl.o0[s];
      dpre = (valid && o0 >= -15.f && o0 <= 15.f) ? sl.dsig[s] * sl.sig[s] : 0.f;
      if (f16) {  // FP16 operands: per-ray scale (undone on the FP32 results)
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) dl[k2] *= gscale;
        dpre *= gscale;
      }
      store8(sl.DL, s, 0, 16, dl, f16);
      store8(sl.DL, s, 1, 16, dl + 8, f16);
    }
    sync_then_issue();
    if (s == 0) {  // dH3 = DL W5 ; dW5^T += H3^T DL
      mma(dtmp, desc_k(sl.DL, 16, 0), desc_mn(sm.w5, kH, 0), idesc(64, 0, 1, f16), 0);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma(kColDW5 + tm, desc_mn(sl.H3, kH, kk), desc_mn(sl.DL, 16, kk), idesc(16, 1, 1, f16), kk > 0 ? 1u : acc_dw);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    epi_mask64(tmp, sl.H3, s, f16);
    sync_then_issue();
    if (s == 0) {  // dH2 = dH3 W4 ; dW4 += dH3^T H2
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma(dtmp, desc_k(sl.H3, kH, kk), desc_mn(sm.w4, kH, kk), idesc(64, 0, 1, f16), kk > 0);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma(kColDW4 + tm, desc_mn(sl.H3, kH, kk), desc_mn(sl.H2, kH, kk), idesc(64, 1, 1, f16), kk > 0 ? 1u : acc_dw);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    epi_mask64(tmp, sl.H2, s, f16);
    sync_then_issue();
    if (s == 0) {  // dCIN = dH2 W3 ; dW3 += dH2^T CIN
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma(dtmp, desc_k(sl.H2, kH, kk), desc_mn(sm.w3, 32, kk), idesc(32, 0, 1, f16), kk > 0);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma(kColDW3 + tm, desc_mn(sl.H2, kH, kk), desc_mn(sl.CIN, 32, kk), idesc(32, 1, 1, f16), kk > 0 ? 1u : acc_dw);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    {
      float v[16], d[16];
      tmem_ld16(tmp, v);
      tmem_wait_ld();
      d[0] = dpre;
#pragma unroll
      for (int j = 0; j < 15; ++j) d[1 + j] = v[j];
      store8(sl.DL, s, 0, 16, d, f16);
      store8(sl.DL, s, 1, 16, d + 8, f16);
    }
    sync_then_issue();
    if (s == 0) {  // dH1 = dOUT W2 ; dW2^T += H1^T dOUT
      mma(dtmp, desc_k(sl.DL, 16, 0), desc_mn(sm.w2, kH, 0), idesc(64, 0, 1, f16), 0);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma(kColDW2 + tm, desc_mn(sl.H1, kH, kk), desc_mn(sl.DL, 16, kk), idesc(16, 1, 1, f16), kk > 0 ? 1u : acc_dw);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    epi_mask64(tmp, sl.H1, s, f16);
    sync_then_issue();
    if (s == 0) {  // dE = dH1 W1 ; dW1 += dH1^T E
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma(dtmp, desc_k(sl.H1, kH, kk), desc_mn(sm.w1, LFP, kk), idesc(LFP, 0, 1, f16), kk > 0);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        mma(kColDW1 + tm, desc_mn(sl.H1, kH, kk), desc_mn(sl.E, LFP, kk), idesc(LFP, 1, 1, f16), kk > 0 ? 1u : acc_dw);
      mma_commit(&sm.mma_bar);
    }
    if (!wait_mma()) break;
    acc_dw = 1;
    {  // stage dL/dencoding for the memory warps
      float de[LFP];
#pragma unroll
      for (int c = 0; c < LFP / 16; ++c) tmem_ld16(tmp + 16 * c, de + 16 * c);
      tmem_wait_ld();
      if (f16) {
#pragma unroll
        for (int c = 0; c < LFP; ++c) de[c] *= gunscale;
      }
#pragma unroll
      for (int c = 0; c < LFP / 4; ++c)
        *reinterpret_cast<float4*>(&sl.dE[s][4 * c]) = make_float4(de[4 * c], de[4 * c + 1], de[4 * c + 2], de[4 * c + 3]);
    }
    mbar_arrive(&sm.empty_bar[slot]);
  }
  if (s == 0) sm.c_stop = sm.fail;
  bar_compute();
  if (!sm.c_stop && bi >= 0) flush_dw<LFP>(tm, g, ob->grad, unscale_of(bi), kCompute);
}

template <int LFP, bool F16>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_tile_ws(GridParams g, BatchDesc b, BatchDyn* dyn, RayBuf R, int32_t* status, int interleave) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WsSmem<LFP>& sm = *reinterpret_cast<WsSmem<LFP>*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  const int total_tiles = 2 * *b.plan_npairs;
  // tiles of this CTA: a contiguous range of the plan, or chunks of `interleave` tiles dealt round-robin (WorkOrder)
  const WorkOrder wo(total_tiles, (int)gridDim.x, (int)blockIdx.x, interleave);
  const int n = wo.count();
  if (n <= 0) return;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mma_bar)));
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.full_bar[i])), "r"(kCompute));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.empty_bar[i])), "r"(kCompute));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sm.fail = 0;
    sm.c_stop = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
  uint32_t phase = 0;
  bool pending = false;
  if (warp < 4) compute_role<LFP, F16>(sm, g, b, dyn, R, status, n, phase, pending);
  else memory_role<LFP, F16>(sm, g, b, R, wo, n);
  if (t == 0 && sm.fail) {
    if (status) atomicOr(status, 2);
    if (pending) mbar_wait(&sm.mma_bar, phase ^ 1u);  // bounded: let MMAs in flight finish before freeing TMEM
  }
  tc_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem_base), "r"(kTmemCols));
}

static_assert(offsetof(WsSlot<16>, dE) % 16 == 0 && offsetof(WsSlot<32>, dE) % 16 == 0, "float4 rows of dE");

template <int LFP, bool F16>
void launch_ws_t(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status, int max_tiles,
                 int n_ctas, int interleave, cudaStream_t stream) {
  int bytes = (int)sizeof(WsSmem<LFP>);
  if (bytes < 116 * 1024) bytes = 116 * 1024;  // one CTA per SM: the 512-column TMEM allocation never waits
  static std::atomic<uint64_t> attr_done{0};
  set_smem_attr(k_tile_ws<LFP, F16>, bytes, attr_done);
  // the plan's tile count is read on the device; max_tiles only bounds the grid
  int grid = n_ctas < max_tiles ? n_ctas : max_tiles;
  if (grid < 1) return;
  k_tile_ws<LFP, F16><<<grid, kWsThreads, bytes, stream>>>(g, b, dyn, r, status, interleave);
}

}  // namespace

void launch_tile_ws(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                    int max_tiles, int n_ctas, int interleave, cudaStream_t stream) {
  if (g.f16) {
    if (g.LF <= 16) launch_ws_t<16, true>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_ws_t<32, true>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else {
    if (g.LF <= 16) launch_ws_t<16, false>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_ws_t<32, false>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  }
}

}  // namespace romap
