// The fused mixed-precision tile kernel (template), included by the translation units that instantiate it: BF16
// and FP8 operands in kernels_tc.cu, FP16 operands in kernels_tc16.cu (one unit each, compiled in parallel).
//
// Mixed-precision training step on the 5th-generation tensor cores: one fused kernel over tiles of 128 sample
// slots that hold whole rays.  The tile plan packs the rays of each object by their number of live samples (rays of
// one class share a slot count P = 128 / k for k rays per tile), so culled candidates and missed rays take no slots.
//
// Per tile, in one CTA of 128 threads (thread s <-> sample slot s <-> TMEM lane s):
//   1. sample positions of the slot (same FP32 operations as the sampling kernels: bit-identical),
//   2. multiresolution hash encoding gathered from the FP16 copy of the table, interpolated in FP32,
//      stored as BF16, or FP16 when F16 (the A operand of the first layer),
//   3. the five MLP layers (Sec. V; hidden 64) as tcgen05.mma kind::f16 (BF16 x BF16 or FP16 x FP16 -> FP32
//      in TMEM), each followed by an epilogue that reads its row from TMEM, applies the activation and writes
//      the next operand row to shared memory,
//   4. volume rendering (Eq. 6), the losses of Eq. 7-11 and the compositing adjoint, one warp per ray,
//   5. the backward: per layer one GEMM for the input gradient (dX = dY W: A = dY K-major, B = W read
//      MN-major from the forward copy) and one for the weight gradient (dW = dY^T X over the 128 samples, or its
//      transpose for the 16-output layers: both operands read MN-major from the activation buffers, M padded to
//      128), the latter accumulated in TMEM across all tiles of the same object and added to the FP32 gradient once
//      per object change,
//   6. the hash-gradient scatter (FP32 vector atomics into the FP32 gradient of the table).
// The transmittance scan, the losses and every accumulation stay in FP32; Adam keeps FP32 masters and
// refreshes the FP16 table copy.  With FP16 operands the backward's gradient operands are scaled by the object's
// batch size B and the FP32 results unscaled (FP16's range; BF16 needs no scale).
//
// Shared-memory operands use the canonical no-swizzle core-matrix layout (8 rows x 16 bytes per core
// matrix): for a K-major [R rows][K] buffer, element (r, k) sits at (r/8)*(K/8)*128 + (k/8)*128 +
// (r%8)*16 + (k%8)*2 bytes; the descriptor strides are LBO = 128 (between 8-column groups along K) and
// SBO = (K/8)*128 (between 8-row groups).  The same buffer read as an MN-major operand (MN = its columns,
// K = its rows) has LBO = (K/8)*128 and SBO = 128.
//
// Every wait on an mbarrier is bounded; on time-out the kernel records ROMAP_ERR_TIMEOUT in the status
// word, waits (bounded) for its own MMAs, frees its tensor memory and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace romap {
namespace {
using namespace tc;


// A CTA processes TPC tiles in lockstep, warpgroup g on tile g: TPC = 2 (a tile pair, one CTA of 256 threads per SM,
// 512 TMEM columns) or TPC = 1 (one tile, two CTAs of 128 threads per SM, 256 TMEM columns each; the two CTAs of an
// SM pass no barrier together, so one's memory-bound phases can overlap the other's GEMMs and epilogues).

// Buffers of one tile.  The activation buffers are contiguous and in this order: the MN-major A operands of the
// weight-gradient GEMMs (64 features, M padded to 128: dH^T for dW1, dW3, dW4; H3^T and HL^T for the transposed dW5
// and dW2) read up to 1 KB past their buffer (the rows >= its feature count), which lands in the next buffer of the
// same tile and only feeds TMEM rows that are never read; DL and E are read as B operands, without overrun.
template <int LFP>
struct TileBufs {
  __align__(128) unsigned char E[2][kT * LFP * 2];  // this pair's encoding and the next pair's, alternating
  __align__(128) unsigned char H1[kT * kH * 2];
  __align__(128) unsigned char CIN[kT * 32 * 2];
  __align__(128) unsigned char H2[kT * kH * 2];
  __align__(128) unsigned char H3[kT * kH * 2];
  __align__(128) unsigned char DL[kT * 16 * 2];  // dL/dlogit, then dL/d(density outputs)
  float px[3][kT];
  float t[kT];
  float dt[kT];
  float sig[kT];
  float o0[kT];
  float rgb[3][kT];
  float dsig[kT];
  float drgb[3][kT];
  int valid[kT];
  int ray[kT];  // global ray index of the slot (-1 outside the tile's rays)
  int pfirst, nrays;  // first plan_perm index and number of the tile's rays
};

// Encoding levels [l0, l1) of one sample, interpolated in FP32 from the FP16 table, into row s of a K-major BF16
// encoding buffer; three levels per round so that 24 gathers are in flight (a gather window of 3 levels is one round).
template <int LFP, bool F16>
__device__ __forceinline__ void gather_rows(const GridParams& g, const ObjectDev* ob, const float p[3],
                                            unsigned char* E, int s, int l0, int l1) {
  const __half2* tab = reinterpret_cast<const __half2*>(ob->table_h);
  // the box in registers: the encoding stores below may alias global memory as far as the compiler knows, which would
  // make every round reload it
  const float hf[3] = {ob->half[0], ob->half[1], ob->half[2]};
  const float ie[3] = {ob->inv_ext[0], ob->inv_ext[1], ob->inv_ext[2]};
#pragma unroll 1
  for (int l = l0; l < l1; l += 3) {
    // the loads of three levels go out first; only the cells' fractions are kept while they are in flight and the
    // trilinear weights are formed from them afterwards (fewer live registers than 24 weights)
    const bool has1 = l + 1 < l1, has2 = l + 2 < l1;
    int i0[3];
    float f0[3], f1[3], f2[3];
    __half2 v0[8], v1[8], v2[8];
    level_cell(g, l, p, hf, ie, i0, f0);
#pragma unroll
    for (int k = 0; k < 8; ++k) v0[k] = __ldg(tab + g.off[l] + corner_index(g, l, i0, k));
    if (has1) {
      level_cell(g, l + 1, p, hf, ie, i0, f1);
#pragma unroll
      for (int k = 0; k < 8; ++k) v1[k] = __ldg(tab + g.off[l + 1] + corner_index(g, l + 1, i0, k));
    }
    if (has2) {
      level_cell(g, l + 2, p, hf, ie, i0, f2);
#pragma unroll
      for (int k = 0; k < 8; ++k) v2[k] = __ldg(tab + g.off[l + 2] + corner_index(g, l + 2, i0, k));
    }
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = corner_weight(f0, k);
      const float2 h = __half22float2(v0[k]);
      a0 = fmaf(w, h.x, a0); a1 = fmaf(w, h.y, a1);
    }
    *reinterpret_cast<uint32_t*>(E + kmaj(s, 2 * l, LFP)) = pack2(a0, a1, F16);
    if (has1) {
      float b0 = 0.f, b1 = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float w = corner_weight(f1, k);
        const float2 h = __half22float2(v1[k]);
        b0 = fmaf(w, h.x, b0); b1 = fmaf(w, h.y, b1);
      }
      *reinterpret_cast<uint32_t*>(E + kmaj(s, 2 * l + 2, LFP)) = pack2(b0, b1, F16);
    }
    if (has2) {
      float d0 = 0.f, d1 = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float w = corner_weight(f2, k);
        const float2 h = __half22float2(v2[k]);
        d0 = fmaf(w, h.x, d0); d1 = fmaf(w, h.y, d1);
      }
      *reinterpret_cast<uint32_t*>(E + kmaj(s, 2 * l + 4, LFP)) = pack2(d0, d1, F16);
    }
  }
}
// zero row s of an encoding buffer over the levels [l0, l1)
template <int LFP>
__device__ __forceinline__ void zero_rows(unsigned char* E, int s, int l0, int l1) {
#pragma unroll 1
  for (int l = l0; l < l1; ++l) *reinterpret_cast<uint32_t*>(E + kmaj(s, 2 * l, LFP)) = 0u;
}

// Hash-gradient scatter of levels [0, L) of a tile's slots, one warp = 32 consecutive slots: slot s at p (valid),
// its dL/dencoding (times unscale) read from TMEM columns de .. de + 2L - 1 of its lane.  Consecutive live samples
// of a ray lie close together, so on the coarse levels runs of adjacent lanes fall in the same grid cell and update
// the same eight corners.  The L1 spends about a cycle on every active lane of a reduction, same address or not, so
// where enough lanes continue a run the runs are summed first (segmented suffix sums by shuffles, as many rounds as
// the longest run needs) and only their first lanes issue the reductions; elsewhere every lane issues its own.  The
// loop reads no memory: after the reductions' memory clobbers, a read of the object's box would be reissued every
// level and wait behind the reductions already queued.
__device__ __forceinline__ void scatter_levels(const GridParams& g, const ObjectDev* ob, int s, int L, const float p[3],
                                               bool valid, uint32_t de, float unscale) {
  constexpr uint32_t kAll = 0xffffffffu;
  constexpr int kMinMerged = 4;  // lanes that must continue a run before a level is summed by shuffles
  const int lane = s & 31;
  const float hf[3] = {ob->half[0], ob->half[1], ob->half[2]};
  const float ie[3] = {ob->inv_ext[0], ob->inv_ext[1], ob->inv_ext[2]};
  float2* gt = reinterpret_cast<float2*>(ob->grad);
#pragma unroll 1
  for (int l = 0; l < L; ++l) {
    float d0, d1;
    tmem_ld2(de + 2u * (uint32_t)l, d0, d1);
    tmem_wait_ld();
    d0 = valid ? d0 * unscale : 0.f;
    d1 = valid ? d1 * unscale : 0.f;
    const bool act = d0 != 0.f || d1 != 0.f;
    if (!__any_sync(kAll, act)) continue;
    int i0[3];
    float f[3];
    level_cell(g, l, p, hf, ie, i0, f);
    // run key: the cell (21 bits per axis); a lane without a contribution gets a key no other lane has
    const unsigned long long key = act ? ((unsigned long long)(uint32_t)i0[0] |
                                          ((unsigned long long)(uint32_t)i0[1] << 21) |
                                          ((unsigned long long)(uint32_t)i0[2] << 42))
                                       : ~0ull - (unsigned long long)lane;
    const unsigned long long prev = __shfl_up_sync(kAll, key, 1);
    const bool head = lane == 0 || prev != key;
    const uint32_t heads = __ballot_sync(kAll, head);
    float a[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = corner_weight(f, k);
      a[2 * k] = w * d0;
      a[2 * k + 1] = w * d1;
    }
    const bool merge = __popc(~heads) >= kMinMerged;
    if (merge) {
      const uint32_t above = lane == 31 ? 0u : heads & ~((2u << lane) - 1u);  // run heads after this lane
      const int span = (above ? __ffs(above) - 2 : 31) - lane;                 // lanes after this one in its run
      const int max_span = (int)__reduce_max_sync(kAll, (uint32_t)span);
      for (int off = 1; off <= max_span; off <<= 1) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float o = __shfl_down_sync(kAll, a[k], off);
          if (off <= span) a[k] += o;
        }
      }
    }
    if (act && (head || !merge)) {
      uint32_t idx[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) idx[k] = corner_index(g, l, i0, k);
      scatter_sums(gt + g.off[l], idx, a);
    }
  }
}

template <int LFP, bool FP8, bool SN, int TPC>
struct TcSmem {
  // weights (B operands of the forward), K-major BF16 [out][in]; w4 holds the colour net's 64x64 layer, or the
  // single-network model's hidden layer 2, and w6() its hidden layer 3
  __align__(128) unsigned char w1[kH * LFP * 2];
  __align__(128) unsigned char w2[16 * kH * 2];
  __align__(128) unsigned char w3[kH * 32 * 2];
  __align__(128) unsigned char w4[kH * kH * 2];
  __align__(128) unsigned char w5[16 * kH * 2];
  TileBufs<LFP> tb[TPC];
  // FP8 E4M3 operands of the hidden 64x64 forward GEMM (ROMAP_PREC_MIXED_FP8): K-major W4 here, each tile's H2
  // rows in h2q(u)
  __align__(128) unsigned char w4q[FP8 ? kH * kH : 16];
  float w4_inv[kH];                    // 1 / (448 / max |W4 row n|) for each output n of the loaded object
  __align__(8) uint64_t mbar[2];  // MMA completion: [0] for the CTA, or [g] for warpgroup g when decoupled
  uint32_t tmem_base;
  int fail;
  int stop[2];  // each group's copy of fail, written by its MMA-issuing thread before a group barrier only
  int rv;       // decoupled warpgroups: rendezvous arrivals
  // the single-network model has no colour-net input: tile 0's CIN buffer holds its hidden layer 3 (a separate
  // buffer would take shared memory from the L1 cache that serves the encoding gathers)
  __device__ unsigned char* w6() { return tb[0].CIN; }
  // tile u's H2 rows in FP8 live in its H3 buffer, which is dead from the end of the backward until the epilogue of
  // the GEMM that reads them writes H3.  Keeping the kernel's shared memory at or below 195 KB leaves the SM's L1
  // cache, which serves the encoding gathers, at 60 KB instead of 28 KB.
  __device__ unsigned char* h2q(int u) { return tb[u].H3; }
};
static_assert(kT * 32 * 2 == kH * kH * 2, "a 64x64 BF16 layer fits in a CIN buffer");
static_assert(kT * kH <= kT * kH * 2, "a tile's FP8 H2 rows fit in its H3 buffer");

// 195 KB plus the 1 KB the system reserves per CTA fit the 196 KB shared-memory carveout; one byte more and the
// carveout becomes 228 KB, which leaves 28 KB of L1 (measured: the fused step 14% slower)
static_assert(sizeof(TcSmem<32, false, false, 2>) <= 195 * 1024 && sizeof(TcSmem<32, true, false, 2>) <= 195 * 1024 &&
                  sizeof(TcSmem<32, false, true, 2>) <= 195 * 1024,
              "shared memory of the fused kernel above the 196 KB carveout");
// two one-tile CTAs (plus 1 KB each reserved by the system) in the 228 KB carveout
static_assert(2 * (sizeof(TcSmem<32, false, false, 1>) + 1024) <= 228 * 1024, "two one-tile CTAs per SM");

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ uint32_t fp8x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

// The FP8 copy of W4, each output row n scaled by 448 / max |W4[n][.]| (4 consecutive threads per row; needs
// nthreads >= 4 kH and a barrier before the MMA reads it).
// The single-network model's hidden layer 3 (64 x 64) as K-major BF16.
template <class Smem>
__device__ void load_w6(Smem& sm, const GridParams& g, const float* __restrict__ P, int t, int nthreads) {
  for (int i = t; i < kH * kH; i += nthreads) {
    int o = i / kH, k = i % kH;
    *reinterpret_cast<uint16_t*>(sm.w6() + kmaj(o, k, kH)) = pack1(P[g.mlp_off[6] + i], g.f16 != 0);
  }
}

template <class Smem>
__device__ void load_w4_fp8(Smem& sm, const GridParams& g, const float* __restrict__ P, int t, int nthreads) {
  const float* W = P + g.mlp_off[3];
  for (int base = 0; base < 4 * kH; base += nthreads) {
    const int i = base + t;  // row i / 4, columns 16 (i % 4) .. + 15
    const int n = i >> 2, q = i & 3;
    float v[16];
    float m = 0.f;
    if (n < kH) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] = W[n * kH + 16 * q + j];
        m = fmaxf(m, fabsf(v[j]));
      }
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    if (n < kH) {
      const float sc = m > 0.f ? 448.f / m : 1.f;
      uint4 w;
      w.x = fp8x4(v[0] * sc, v[1] * sc, v[2] * sc, v[3] * sc);
      w.y = fp8x4(v[4] * sc, v[5] * sc, v[6] * sc, v[7] * sc);
      w.z = fp8x4(v[8] * sc, v[9] * sc, v[10] * sc, v[11] * sc);
      w.w = fp8x4(v[12] * sc, v[13] * sc, v[14] * sc, v[15] * sc);
      *reinterpret_cast<uint4*>(sm.w4q + kmaj8(n, 16 * q, kH)) = w;
      if (q == 0) sm.w4_inv[n] = 1.f / sc;
    }
  }
}

// relu(row_scale * col_scale[j] * TMEM row) -> BF16 row (the dequantising epilogue of the FP8 GEMM)
__device__ __forceinline__ void epi_relu64_scaled(uint32_t taddr, unsigned char* buf, int row, float row_scale,
                                                  const float* col_scale, bool f16) {
  float v[64];
#pragma unroll
  for (int c = 0; c < 4; ++c) tmem_ld16(taddr + 16 * c, v + 16 * c);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 64; ++j) v[j] = fmaxf(v[j] * row_scale * col_scale[j], 0.f);
#pragma unroll
  for (int c = 0; c < 8; ++c) store8(buf, row, c, kH, v + 8 * c, f16);
}

// relu(TMEM row) -> BF16 row of an activation buffer (64 columns); the four TMEM loads share one wait
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
// TMEM row masked by relu'(the forward activation stored in buf) -> written back into buf (64 columns)
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

// DEC (decoupled, with TPC = 2): the two warpgroups of the CTA run their tiles of each pair independently, each with
// its own MMA-issuing thread, mbarrier, named barrier and 256 TMEM columns (its own weight-gradient accumulators and
// temporary); they share the weights in shared memory and meet only at object changes (a bounded rendezvous), so
// that one tile's memory-bound phases (gathers, scatter) can run while the other tile's GEMMs, epilogues and
// compositing do.
template <int LFP, bool FP8, bool SN, bool F16, int TPC, bool DEC>
__global__ void __launch_bounds__(128 * TPC, 3 - TPC)
    k_tile_tc(GridParams g, BatchDesc b, BatchDyn* dyn, RayBuf R, int32_t* status, int interleave) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  static_assert(!DEC || TPC == 2, "decoupled warpgroups need a tile pair");
  constexpr int kTilesPerCta = TPC, kTcThreads = 128 * TPC;
  constexpr uint32_t kCols = TPC == 2 ? 512u : 256u;  // TMEM columns: kColTmp + 64 per tile, a power of 2
  TcSmem<LFP, FP8, SN, TPC>& sm = *reinterpret_cast<TcSmem<LFP, FP8, SN, TPC>*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  const int wg = t >> 7;          // tile of the pair
  const int s = t & (kT - 1);     // slot within the tile = TMEM lane
  TileBufs<LFP>& tb = sm.tb[wg];
  // MLP operands in FP16 instead of BF16: the backward's gradient operands are then scaled by the object's batch
  // size B (the losses are means over B rays, so the scaled values are per-ray gradients, inside FP16's range) and
  // the FP32 results unscaled
  constexpr bool f16 = F16;
  auto unscale_of = [&](int bi_) { return f16 ? 1.0f / (float)(b.ray_base[bi_ + 1] - b.ray_base[bi_]) : 1.0f; };
  // pairs of this CTA: a contiguous range of the plan, or chunks of `interleave` pairs dealt round-robin (WorkOrder)
  // work items: tile pairs, or single tiles (both tiles of a pair hold the same object; the second may be empty)
  const WorkOrder wo((TPC == 2 ? 1 : 2) * *b.plan_npairs, (int)gridDim.x, (int)blockIdx.x, interleave);
  const int n_items = wo.count();
  if (n_items <= 0) return;

  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sm.mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sm.mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sm.fail = 0;
    sm.stop[0] = sm.stop[1] = 0;
    sm.rv = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&sm.tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tm = sm.tmem_base;
  // TMEM column of tile u's temporary, and the weight-gradient accumulators the tiles of this thread's warpgroup use:
  // shared by the pair (columns 0..191), or decoupled: warpgroup g's own block of 256 columns
  auto tcol = [](int u) { return DEC ? 256u * (uint32_t)u + kColTmp : kColTmp + 64u * (uint32_t)u; };
  const uint32_t dwb = tm + (DEC ? 256u * (uint32_t)wg : 0u);
  const uint32_t tmp = tm + ((uint32_t)(32 * (warp & 3)) << 16) + tcol(wg);  // this thread's row
  uint32_t phase = 0;
  bool ok = true;
  // the MMA-issuing thread and the tiles it issues for: thread 0 for both tiles, or the first thread of each
  // decoupled warpgroup for its own tile
  const bool issuer = DEC ? (t & 127) == 0 : t == 0;
  const int u_lo = DEC ? wg : 0, u_hi = DEC ? wg + 1 : kTilesPerCta;
  uint64_t* const mbar = &sm.mbar[DEC ? wg : 0];
  auto group_sync = [&]() {  // the CTA, or this decoupled warpgroup (named barrier 1 + g)
    if constexpr (DEC) asm volatile("bar.sync %0, 128;" :: "r"(1 + wg) : "memory");
    else __syncthreads();
  };

  auto sync_then_issue = [&]() {  // every thread's shared writes and TMEM reads become visible to the MMAs
    fence_async_smem();
    tc_before();
    group_sync();
    tc_after();
  };
  // every stop decision of a group reads its stop copy after a group barrier, so that all of its threads take the
  // same branch (fail itself may be set by the other decoupled group at any time)
  const int grp = DEC ? wg : 0;
  auto wait_mma = [&]() -> bool {  // one thread polls the mbarrier; the others wait at the barrier
    if (issuer) {
      if (!mbar_wait(mbar, phase)) sm.fail = 1;
      sm.stop[grp] = *(volatile int*)&sm.fail;
    }
    phase ^= 1u;
    group_sync();
    tc_after();
    return sm.stop[grp] == 0;
  };
  auto tmp_d = [&](int u) { return tm + tcol(u); };
  // decoupled warpgroups meet at object changes: each one's first thread arrives on the shared counter and waits
  // (bounded) for the other's arrival; a time-out or the other's failure sets the failure flag
  int rv_round = 0;
  auto rendezvous = [&]() -> bool {
    fence_async_smem();  // this thread's shared-memory writes (the weights) visible to the other group's MMAs
    group_sync();
    if ((t & 127) == 0) {
      __threadfence_block();
      const int target = 2 * (++rv_round);
      atomicAdd(&sm.rv, 1);
      int it = 0;
      while (*(volatile int*)&sm.rv < target && *(volatile int*)&sm.fail == 0 && ++it < kWaitLimit) {
      }
      if (it >= kWaitLimit) sm.fail = 1;
      sm.stop[grp] = *(volatile int*)&sm.fail;
      __threadfence_block();
    }
    group_sync();
    return sm.stop[grp] == 0;
  };

  int bi = -1;
  const ObjectDev* ob = nullptr;
  uint32_t acc_dw = 0;  // 0 until the first weight-gradient GEMM of an object has run
  constexpr int LMAX = LFP / 2;
  // the sample and encoding of the next pair are computed ahead, mostly while the backward GEMMs of the current
  // pair run, and kept in registers until the current pair no longer reads the tile buffers
  int4 nx_ti = b.plan_tiles[wo.item(0) * kTilesPerCta + wg];  // both tiles of a pair belong to the same object
  int nx_bi = nx_ti.x;
  const ObjectDev* nx_ob = &b.objs[b.slot[nx_bi]];
  SlotSample nx = plan_sample(g, b, R, nx_ob, nx_bi, nx_ti, s);
  const int Lg = g.L < LMAX ? g.L : LMAX;
  // hidden layers after the first (single-network model) and their activation buffers: hid(u, 0) = H1, 1 = H2,
  // 2 = H3 of tile u; the last one feeds the density net's output layer
  const int nl = SN ? g.extra : 0;
  auto hid = [&](int u, int k) -> unsigned char* { return k == 0 ? sm.tb[u].H1 : k == 1 ? sm.tb[u].H2 : sm.tb[u].H3; };
  // level ranges of the backward windows that overlap the next pair's gather: five with the colour net; without
  // it one per hidden layer plus the output layer's
  const int nwin = SN ? 2 + nl : 5;
  auto part = [&](int k) { return k * Lg / nwin; };
  int cur = 0;  // encoding buffer of the current pair
  // columns past 2 L stay zero in both buffers
  for (int u = 0; u < 2; ++u) zero_rows<LFP>(tb.E[u], s, Lg, LMAX);
  if (nx.valid) {
    const float p[3] = {nx.x, nx.y, nx.z};
    gather_rows<LFP, F16>(g, nx_ob, p, tb.E[0], s, 0, Lg);
  } else {
    zero_rows<LFP>(tb.E[0], s, 0, Lg);
  }
  for (int it = 0; it < n_items && ok; ++it) {
    // ---- 1-2. the prepared sample and encoding of this pair -> tile buffers ---------------------------------------
    tb.valid[s] = nx.valid;
    tb.ray[s] = nx.ray;
    if (s == 0) {
      tb.pfirst = nx_ti.w;
      tb.nrays = nx_ti.z & 255;
    }
    tb.px[0][s] = nx.x; tb.px[1][s] = nx.y; tb.px[2][s] = nx.z;
    tb.t[s] = nx.t;
    tb.dt[s] = nx.dt;
    if (nx_bi != bi) {
      // the new object's weights are fetched first, so that their round trip overlaps the flush of the previous
      // object's weight gradients (warps 0, 1, 4 and 5)
      constexpr int kWB = (WeightIndex<LFP>::total + kTcThreads - 1) / kTcThreads;
      float wv[kWB];
      weights_fetch<LFP, kWB>(g, nx_ob->params, t, kTcThreads, wv);
      if constexpr (DEC) {
        // both warpgroups are done with the previous object's weights; each flushes its own accumulators
        if (!rendezvous()) {
          ok = false;
          break;
        }
        if (bi >= 0) flush_dw_group<LFP>(dwb, g, ob->grad, unscale_of(bi));
      } else {
        if (bi >= 0) flush_dw<LFP>(tm, g, ob->grad, unscale_of(bi), kTcThreads);
      }
      bi = nx_bi;
      ob = nx_ob;
      weights_store<LFP, kWB>(sm, g, t, kTcThreads, wv);
      if (FP8) load_w4_fp8(sm, g, ob->params, t, kTcThreads);
      if (SN && g.extra >= 2) load_w6(sm, g, ob->params, t, kTcThreads);
      if constexpr (DEC) {  // the new weights are in place for both warpgroups
        if (!rendezvous()) {
          ok = false;
          break;
        }
      }
      acc_dw = 0;
    }
    const int n_rays_obj = b.ray_base[bi + 1] - b.ray_base[bi];
    const float invB = 1.0f / (float)n_rays_obj;
    const float gscale = f16 ? (float)n_rays_obj : 1.0f, gunscale = f16 ? invB : 1.0f;
    const bool has_next = it + 1 < n_items;
    if (has_next) {
      nx_ti = b.plan_tiles[wo.item(it + 1) * kTilesPerCta + wg];
      nx_bi = nx_ti.x;
      nx_ob = &b.objs[b.slot[nx_bi]];
    }
    sync_then_issue();
    // ---- 3. forward ----------------------------------------------------------------------------------------------
    if (issuer) {  // L1: E W1^T
      for (int u = u_lo; u < u_hi; ++u)
#pragma unroll
        for (int kk = 0; kk < LFP / 16; ++kk)
          mma(tmp_d(u), desc_k(sm.tb[u].E[cur], LFP, kk), desc_k(sm.w1, LFP, kk), idesc(64, 0, 0, f16), kk > 0);
      mma_commit(mbar);
    }
    if (!(ok = wait_mma())) break;
    epi_relu64(tmp, tb.H1, s, f16);
    if constexpr (SN) {  // single-network hidden layers 2 and 3: hid(k + 1) = relu(hid(k) M^T), M = w4, w6
      for (int k = 0; k < nl; ++k) {
        sync_then_issue();
        if (issuer) {
          for (int u = u_lo; u < u_hi; ++u)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma(tmp_d(u), desc_k(hid(u, k), kH, kk), desc_k(k == 0 ? sm.w4 : sm.w6(), kH, kk), idesc(64, 0, 0, f16),
                  kk > 0);
          mma_commit(mbar);
        }
        if (!(ok = wait_mma())) break;
        epi_relu64(tmp, hid(wg, k + 1), s, f16);
      }
      if (!ok) break;
    }
    sync_then_issue();
    if (issuer) {  // L2: HL W2^T (16 outputs), HL = H1 unless the single network has more hidden layers
      for (int u = u_lo; u < u_hi; ++u)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma(tmp_d(u), desc_k(hid(u, nl), kH, kk), desc_k(sm.w2, kH, kk), idesc(16, 0, 0, f16), kk > 0);
      mma_commit(mbar);
    }
    if (!(ok = wait_mma())) break;
    {
      float v[16];
      tmem_ld16(tmp, v);
      tmem_wait_ld();
      const float o0 = v[0];
      tb.o0[s] = o0;
      tb.sig[s] = expf(fminf(fmaxf(o0, -15.f), 15.f));
      if constexpr (SN) {  // the colour logits are density-net outputs 1..3
#pragma unroll
        for (int k = 0; k < 3; ++k) tb.rgb[k][s] = 1.0f / (1.0f + expf(-v[1 + k]));
      } else {
        float cin[32];
#pragma unroll
        for (int j = 0; j < 15; ++j) cin[j] = v[1 + j];
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (g.dir_dims == 3 && tb.valid[s]) {
          const int64_t r = tb.ray[s];
          d0 = R.d[3 * r]; d1 = R.d[3 * r + 1]; d2 = R.d[3 * r + 2];
        }
        cin[15] = d0; cin[16] = d1; cin[17] = d2;
#pragma unroll
        for (int j = 18; j < 32; ++j) cin[j] = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) store8(tb.CIN, s, c, 32, cin + 8 * c, f16);
      }
    }
    if constexpr (!SN) {  // ---- colour net --------------------------------------------------------------------------
      sync_then_issue();
      if (issuer) {  // L3: CIN W3^T
        for (int u = u_lo; u < u_hi; ++u)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            mma(tmp_d(u), desc_k(sm.tb[u].CIN, 32, kk), desc_k(sm.w3, 32, kk), idesc(64, 0, 0, f16), kk > 0);
        mma_commit(mbar);
      }
      if (!(ok = wait_mma())) break;
      epi_relu64(tmp, tb.H2, s, f16);
      float h2_scale = 1.f;  // FP8: 448 / max of this sample's H2 row (1 when all zero)
      if (FP8) {  // this sample's H2 row in E4M3; the row scale factors out of its GEMM outputs
        float hv[64];
#pragma unroll
        for (int c = 0; c < 8; ++c) load8(tb.H2, s, c, kH, hv + 8 * c, f16);
        float m = 0.f;
#pragma unroll
        for (int j = 0; j < 64; ++j) m = fmaxf(m, hv[j]);
        const float sc = m > 0.f ? 448.f / m : 1.f;
        h2_scale = sc;
#pragma unroll
        for (int c = 0; c < 4; ++c) {  // 16 consecutive k of row s are one 16-byte core-matrix row
          const float* h = hv + 16 * c;
          uint4 q;
          q.x = fp8x4(h[0] * sc, h[1] * sc, h[2] * sc, h[3] * sc);
          q.y = fp8x4(h[4] * sc, h[5] * sc, h[6] * sc, h[7] * sc);
          q.z = fp8x4(h[8] * sc, h[9] * sc, h[10] * sc, h[11] * sc);
          q.w = fp8x4(h[12] * sc, h[13] * sc, h[14] * sc, h[15] * sc);
          *reinterpret_cast<uint4*>(sm.h2q(wg) + kmaj8(s, 16 * c, kH)) = q;
        }
      }
      sync_then_issue();
      if (issuer) {  // L4: H2 W4^T
        for (int u = u_lo; u < u_hi; ++u) {
          if (FP8) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
              mma8(tmp_d(u), desc_k8(sm.h2q(u), kH, kk), desc_k8(sm.w4q, kH, kk), idesc8(64), kk > 0);
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma(tmp_d(u), desc_k(sm.tb[u].H2, kH, kk), desc_k(sm.w4, kH, kk), idesc(64, 0, 0, f16), kk > 0);
          }
        }
        mma_commit(mbar);
      }
      if (!(ok = wait_mma())) break;
      if (FP8) epi_relu64_scaled(tmp, tb.H3, s, 1.0f / h2_scale, sm.w4_inv, f16);
      else epi_relu64(tmp, tb.H3, s, f16);
      sync_then_issue();
      if (issuer) {  // L5: H3 W5^T (3 of 16 outputs)
        for (int u = u_lo; u < u_hi; ++u)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma(tmp_d(u), desc_k(sm.tb[u].H3, kH, kk), desc_k(sm.w5, kH, kk), idesc(16, 0, 0, f16), kk > 0);
        mma_commit(mbar);
      }
      if (!(ok = wait_mma())) break;
      {
        float v[16];
        tmem_ld16(tmp, v);
        tmem_wait_ld();
        tb.rgb[0][s] = 1.0f / (1.0f + expf(-v[0]));
        tb.rgb[1][s] = 1.0f / (1.0f + expf(-v[1]));
        tb.rgb[2][s] = 1.0f / (1.0f + expf(-v[2]));
      }
    }  // colour net
    group_sync();
    // ---- 4. compositing, losses, adjoint: one warp per ray of the pair -----------------------------------------
    {
      if constexpr (DEC) {  // this warpgroup's tile, its four warps
        auto tile_of = [&](int) -> TileBufs<LFP>& { return tb; };
        composite_rays(tile_of, tb.nrays, tb.nrays, warp & 3, 4, g, b, R, dyn, bi, invB, status);
      } else {
        const int nr0 = sm.tb[0].nrays;
        int nr_all = nr0;
        if constexpr (TPC == 2) nr_all += sm.tb[1].nrays;
        auto tile_of = [&](int u) -> TileBufs<LFP>& { return sm.tb[u]; };
        composite_rays(tile_of, nr0, nr_all, warp, kTcThreads / 32, g, b, R, dyn, bi, invB, status);
      }
    }
    group_sync();
    // ---- 5. backward -----------------------------------------------------------------------------------------------
    float dpre;
    {
      const bool valid = tb.valid[s];
      float dl[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) dl[k] = 0.f;
      if (valid) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float c = tb.rgb[k][s];
          dl[k] = tb.drgb[k][s] * c * (1.f - c);
        }
      }
      const float o0 = tb.o0[s];
      dpre = (valid && o0 >= -15.f && o0 <= 15.f) ? tb.dsig[s] * tb.sig[s] : 0.f;
      if (f16) {  // FP16 operands: per-ray scale (undone on the FP32 results)
#pragma unroll
        for (int k = 0; k < 3; ++k) dl[k] *= gscale;
        dpre *= gscale;
      }
      if constexpr (SN) {  // dOUT = [dsigma * sigma, dlogit 0..2, 0 ...]
#pragma unroll
        for (int k = 15; k > 0; --k) dl[k] = k <= 3 ? dl[k - 1] : 0.f;
        dl[0] = dpre;
      }
      store8(tb.DL, s, 0, 16, dl, f16);
      store8(tb.DL, s, 1, 16, dl + 8, f16);
    }
    if constexpr (!SN) {  // ---- colour net backward ------------------------------------------------------------------
      sync_then_issue();
      if (issuer) {  // dH3 = DL W5 ; dW5^T += H3^T DL
        for (int u = u_lo; u < u_hi; ++u) {
          mma(tmp_d(u), desc_k(sm.tb[u].DL, 16, 0), desc_mn(sm.w5, kH, 0), idesc(64, 0, 1, f16), 0);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            mma(kColDW5 + dwb, desc_mn(sm.tb[u].H3, kH, kk), desc_mn(sm.tb[u].DL, 16, kk), idesc(16, 1, 1, f16),
                (u > u_lo || kk > 0) ? 1u : acc_dw);
        }
        mma_commit(mbar);
      }
      {  // while the MMAs run: the next pair's sample and part 0 of its encoding (into the other buffer)
        if (has_next) {
          nx = plan_sample(g, b, R, nx_ob, nx_bi, nx_ti, s);
          const float p[3] = {nx.x, nx.y, nx.z};
          if (nx.valid) gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(0), part(1));
          else zero_rows<LFP>(tb.E[cur ^ 1], s, 0, Lg);
        }
      }
      if (!(ok = wait_mma())) break;
      epi_mask64(tmp, tb.H3, s, f16);
      sync_then_issue();
      if (issuer) {  // dH2 = dH3 W4 ; dW4 += dH3^T H2
        for (int u = u_lo; u < u_hi; ++u) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma(tmp_d(u), desc_k(sm.tb[u].H3, kH, kk), desc_mn(sm.w4, kH, kk), idesc(64, 0, 1, f16), kk > 0);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            mma(kColDW4 + dwb, desc_mn(sm.tb[u].H3, kH, kk), desc_mn(sm.tb[u].H2, kH, kk), idesc(64, 1, 1, f16),
                (u > u_lo || kk > 0) ? 1u : acc_dw);
        }
        mma_commit(mbar);
      }
      {  // while the MMAs run: part 1 of the next pair's encoding
        if (has_next && nx.valid) {
          const float p[3] = {nx.x, nx.y, nx.z};
          gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(1), part(2));
        }
      }
      if (!(ok = wait_mma())) break;
      epi_mask64(tmp, tb.H2, s, f16);
      sync_then_issue();
      if (issuer) {  // dCIN = dH2 W3 (32 columns) ; dW3 += dH2^T CIN
        for (int u = u_lo; u < u_hi; ++u) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma(tmp_d(u), desc_k(sm.tb[u].H2, kH, kk), desc_mn(sm.w3, 32, kk), idesc(32, 0, 1, f16), kk > 0);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            mma(kColDW3 + dwb, desc_mn(sm.tb[u].H2, kH, kk), desc_mn(sm.tb[u].CIN, 32, kk), idesc(32, 1, 1, f16),
                (u > u_lo || kk > 0) ? 1u : acc_dw);
        }
        mma_commit(mbar);
      }
      {  // while the MMAs run: part 2 of the next pair's encoding
        if (has_next && nx.valid) {
          const float p[3] = {nx.x, nx.y, nx.z};
          gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(2), part(3));
        }
      }
      if (!(ok = wait_mma())) break;
      {  // dOUT = [dsigma * sigma, dCIN[0..14]] into DL
        float v[16], d[16];
        tmem_ld16(tmp, v);
        tmem_wait_ld();
        d[0] = dpre;
#pragma unroll
        for (int j = 0; j < 15; ++j) d[1 + j] = v[j];
        store8(tb.DL, s, 0, 16, d, f16);
        store8(tb.DL, s, 1, 16, d + 8, f16);
      }
    }  // colour net backward
    sync_then_issue();
    if (issuer) {  // dHL = dOUT W2 ; dW2^T += HL^T dOUT
      for (int u = u_lo; u < u_hi; ++u) {
        mma(tmp_d(u), desc_k(sm.tb[u].DL, 16, 0), desc_mn(sm.w2, kH, 0), idesc(64, 0, 1, f16), 0);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          mma(kColDW2 + dwb, desc_mn(hid(u, nl), kH, kk), desc_mn(sm.tb[u].DL, 16, kk), idesc(16, 1, 1, f16),
              (u > u_lo || kk > 0) ? 1u : acc_dw);
      }
      mma_commit(mbar);
    }
    if constexpr (SN) {  // while the MMAs run: the next pair's sample and the first half of its encoding
      if (has_next) {
        nx = plan_sample(g, b, R, nx_ob, nx_bi, nx_ti, s);
        const float p[3] = {nx.x, nx.y, nx.z};
        if (nx.valid) gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(0), part(1));
        else zero_rows<LFP>(tb.E[cur ^ 1], s, 0, Lg);
      }
    } else {  // while the MMAs run: part 3 of the next pair's encoding
      if (has_next && nx.valid) {
        const float p[3] = {nx.x, nx.y, nx.z};
        gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(3), part(4));
      }
    }
    if (!(ok = wait_mma())) break;
    epi_mask64(tmp, hid(wg, nl), s, f16);
    if constexpr (SN) {  // hidden layers 3, 2: dhid(k) = dhid(k + 1) M ; dM += dhid(k + 1)^T hid(k)
      for (int k = nl - 1; k >= 0; --k) {
        sync_then_issue();
        if (issuer) {
          const unsigned char* w = k == 0 ? sm.w4 : sm.w6();
          const uint32_t col = k == 0 ? kColDW4 : kColDW3;
          for (int u = u_lo; u < u_hi; ++u) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma(tmp_d(u), desc_k(hid(u, k + 1), kH, kk), desc_mn(w, kH, kk), idesc(64, 0, 1, f16), kk > 0);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              mma(col + dwb, desc_mn(hid(u, k + 1), kH, kk), desc_mn(hid(u, k), kH, kk), idesc(64, 1, 1, f16),
                  (u > u_lo || kk > 0) ? 1u : acc_dw);
          }
          mma_commit(mbar);
        }
        {  // while the MMAs run: the next part of the next pair's encoding
          if (has_next && nx.valid) {
            const float p[3] = {nx.x, nx.y, nx.z};
            gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(nl - k), part(nl - k + 1));
          }
        }
        if (!(ok = wait_mma())) break;
        epi_mask64(tmp, hid(wg, k), s, f16);
      }
      if (!ok) break;
    }
    sync_then_issue();
    if (issuer) {  // dE = dH1 W1 (LFP columns) ; dW1 += dH1^T E
      for (int u = u_lo; u < u_hi; ++u) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma(tmp_d(u), desc_k(sm.tb[u].H1, kH, kk), desc_mn(sm.w1, LFP, kk), idesc(LFP, 0, 1, f16), kk > 0);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          mma(kColDW1 + dwb, desc_mn(sm.tb[u].H1, kH, kk), desc_mn(sm.tb[u].E[cur], LFP, kk), idesc(LFP, 1, 1, f16),
              (u > u_lo || kk > 0) ? 1u : acc_dw);
      }
      mma_commit(mbar);
    }
    {  // while the MMAs run: the last part of the next pair's encoding
      if (has_next && nx.valid) {
        const float p[3] = {nx.x, nx.y, nx.z};
        gather_rows<LFP, F16>(g, nx_ob, p, tb.E[cur ^ 1], s, part(nwin - 1), part(nwin));
      }
    }
    if (!(ok = wait_mma())) break;
    acc_dw = 1;
    {  // ---- 6. scatter dL/dencoding into the FP32 table gradient ----
      const float p[3] = {tb.px[0][s], tb.px[1][s], tb.px[2][s]};
      scatter_levels(g, ob, s, Lg, p, tb.valid[s] != 0, tmp, gunscale);
    }
    cur ^= 1;  // the next pair's encoding is in the other buffer
    tc_before();
    group_sync();
    tc_after();
  }
  if (ok && bi >= 0) {
    if constexpr (DEC) flush_dw_group<LFP>(dwb, g, ob->grad, unscale_of(bi));
    else flush_dw<LFP>(tm, g, ob->grad, unscale_of(bi), kTcThreads);
  } else if (!ok) {
    if (issuer) {
      if (status) atomicOr(status, 2);
      mbar_wait(mbar, phase ^ 1u);  // bounded: let the MMAs still in flight finish before the columns are freed
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tm), "r"(kCols));
}

template <int LFP, bool FP8, bool SN, bool F16, int TPC, bool DEC = false>
void launch_tc_t(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                 int max_tiles, int n_ctas, int interleave, cudaStream_t stream) {
  auto kernel = k_tile_tc<LFP, FP8, SN, F16, TPC, DEC>;
  int bytes = (int)sizeof(TcSmem<LFP, FP8, SN, TPC>);
  static std::atomic<uint64_t> attr_done{0};
  if (TPC == 2) {
    // at least 116 KB of shared memory per CTA keeps one CTA per SM, so that the 512-column TMEM allocation of one
    // CTA never waits on another
    if (bytes < 116 * 1024) bytes = 116 * 1024;
    set_smem_attr(kernel, bytes, attr_done);
  } else {
    // two CTAs per SM (256 TMEM columns each): the largest shared-memory carveout
    static std::atomic<uint64_t> carve_done{0};
    set_smem_attr(kernel, bytes, attr_done);
    set_func_attr(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared,
                  carve_done);
  }
  // the plan's pair count is read on the device; max_tiles only bounds the grid
  const int max_units = TPC == 2 ? (max_tiles + 1) / 2 : max_tiles;
  const int ctas = TPC == 2 ? n_ctas : 2 * n_ctas;
  const int grid = ctas < max_units ? ctas : max_units;
  if (grid < 1) return;
  kernel<<<grid, 128 * TPC, bytes, stream>>>(g, b, dyn, r, status, interleave);
}

}  // namespace
}  // namespace romap
