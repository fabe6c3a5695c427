// tcgen05 helpers shared by the tensor-core tile kernels (instruction and shared-memory descriptors, TMEM loads,
// BF16 operand rows, weight staging, weight-gradient flush, compositing of one ray, hash gathers, slot samples).
// See kernels_tc.cu for the operand layouts.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "device_common.cuh"
#include "romap_internal.cuh"

namespace romap {
namespace tc {


constexpr int kT = 128;           // samples per tile (MMA M)
constexpr int kTmemCols = 512;
// TMEM columns: weight-gradient accumulators (shared by the tiles of a CTA), then one 64-column temporary per tile.
// dW1, dW3 and dW4 accumulate with their output rows in TMEM lanes (M = out, padded to 128) and their inputs in
// columns (dW1: LFP columns, dW3: 32, or 64 for the single network's hidden layer 3, dW4: 64), so that a lane holds a
// contiguous row of the FP32 gradient, flushed with 16-byte reductions; dW2 and dW5 (16 and 3 outputs of 64 inputs)
// accumulate transposed, inputs in lanes and 16 output columns each, flushed with reductions that are contiguous
// across lanes.  192 columns of accumulators plus 64 per tile: 256 for a one-tile CTA (two CTAs per SM), 320 of 512
// for a tile pair.
constexpr uint32_t kColDW1 = 0, kColDW3 = 32, kColDW2 = 96, kColDW4 = 112, kColDW5 = 176, kColTmp = 192;
constexpr int kWaitLimit = 1 << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// K-major operand: [rows][K] buffer; K-step kk covers columns 16 kk .. 16 kk + 15
__device__ __forceinline__ uint64_t desc_k(const void* buf, int K, int kk) {
  return make_desc(smem_u32(buf) + (uint32_t)kk * 256u, 128u, (uint32_t)(K / 8) * 128u);
}
// MN-major view of a K-major [rows][F] buffer: MN = its F columns, K = its rows; K-step kk covers rows 16 kk ..
__device__ __forceinline__ uint64_t desc_mn(const void* buf, int F, int kk) {
  return make_desc(smem_u32(buf) + (uint32_t)kk * 2u * (uint32_t)(F / 8) * 128u, (uint32_t)(F / 8) * 128u, 128u);
}
// instruction descriptor, kind::f16: A and B both BF16 (format 1) or both FP16 (format 0, f16), FP32 D
__host__ __device__ constexpr uint32_t idesc(int N, int a_mn, int b_mn, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) | ((uint32_t)a_mn << 15) |
         ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kT >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
// 8-bit operands (kind::f8f6f4, E4M3): core matrix = 8 rows x 16 elements; a K-major [rows][K] buffer holds element
// (r, k) at byte (r/8)(K/16)128 + (k/16)128 + (r%8)16 + (k%16); one MMA covers K = 32 (two 16-element groups)
__device__ __forceinline__ uint32_t kmaj8(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K >> 4) * 128 + (k >> 4) * 128 + (r & 7) * 16 + (k & 15));
}
__device__ __forceinline__ uint64_t desc_k8(const void* buf, int K, int kk) {
  return make_desc(smem_u32(buf) + (uint32_t)kk * 256u, 128u, (uint32_t)(K / 16) * 128u);
}
// instruction descriptor, kind::f8f6f4: E4M3 A and B (format 0), FP32 D, K-major operands
__host__ __device__ constexpr uint32_t idesc8(int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kT >> 4) << 24);
}
__device__ __forceinline__ void mma8(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = kWaitLimit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  }
  return done != 0;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 w .. 32 w + 31)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 2 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float& a, float& b) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
  a = __uint_as_float(r0);
  b = __uint_as_float(r1);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element (r, k) in a K-major [rows][K] BF16 buffer
__device__ __forceinline__ uint32_t kmaj(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
// MLP operands are BF16, or FP16 (f16: 3 more mantissa bits, range +-65504: values are saturated there; a NaN
// stays a NaN, so that a broken step still shows as a non-finite loss)
__device__ __forceinline__ float sat_f16(float x) { return x > 65504.f ? 65504.f : (x < -65504.f ? -65504.f : x); }
__device__ __forceinline__ uint32_t pack2(float a, float b, bool f16) {
  if (f16) {
    __half2 h = __floats2half2_rn(sat_f16(a), sat_f16(b));
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack2(uint32_t x, bool f16) {
  if (f16) return __half22float2(*reinterpret_cast<const __half2*>(&x));
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x));
}
__device__ __forceinline__ uint16_t pack1(float a, bool f16) {
  if (f16) {
    __half h = __float2half_rn(sat_f16(a));
    return *reinterpret_cast<uint16_t*>(&h);
  }
  __nv_bfloat16 h = __float2bfloat16_rn(a);
  return *reinterpret_cast<uint16_t*>(&h);
}
// row r, 8 columns starting at 8c, packed as BF16 / FP16
__device__ __forceinline__ void store8(unsigned char* buf, int r, int c, int K, const float* v, bool f16) {
  uint4 q;
  q.x = pack2(v[0], v[1], f16); q.y = pack2(v[2], v[3], f16);
  q.z = pack2(v[4], v[5], f16); q.w = pack2(v[6], v[7], f16);
  *reinterpret_cast<uint4*>(buf + kmaj(r, 8 * c, K)) = q;
}
__device__ __forceinline__ void load8(const unsigned char* buf, int r, int c, int K, float* v, bool f16) {
  const uint4 q = *reinterpret_cast<const uint4*>(buf + kmaj(r, 8 * c, K));
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = unpack2(w[i], f16);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// The five forward weight matrices of an object as K-major BF16 (FP16) operands, in one index space of padded shapes:
// [w1: kH x LFP][w2: 16 x kH][w3: kH x 32][w4: kH x kH][w5: 16 x kH] (padding reads as 0).  A thread's loads of a batch
// are all issued before its first shared-memory store, so that a batch costs one round trip to L2: under the load of
// the other CTAs' hash gathers and scatters a round trip takes a few thousand cycles, and staging the weights one
// load at a time made every object change of a CTA cost tens of microseconds.
template <int LFP>
struct WeightIndex {
  static constexpr int n1 = kH * LFP, n2 = n1 + 16 * kH, n3 = n2 + kH * 32, n4 = n3 + kH * kH, total = n4 + 16 * kH;
};
template <int LFP>
__device__ __forceinline__ float weight_fetch(const GridParams& g, const float* __restrict__ P, int64_t off4, int i) {
  using W = WeightIndex<LFP>;
  if (i < W::n1) {
    const int o = i / LFP, k = i % LFP;
    return k < g.LF ? __ldg(P + g.mlp_off[0] + o * g.LF + k) : 0.f;
  }
  if (i < W::n2) return __ldg(P + g.mlp_off[1] + (i - W::n1));
  if (i < W::n3) {
    const int j = i - W::n2, o = j / 32, k = j % 32;
    return k < g.cin ? __ldg(P + g.mlp_off[2] + o * g.cin + k) : 0.f;
  }
  if (i < W::n4) return __ldg(P + off4 + (i - W::n3));
  const int j = i - W::n4;
  return j < 3 * kH ? __ldg(P + g.mlp_off[4] + j) : 0.f;
}
template <int LFP, class Smem>
__device__ __forceinline__ unsigned char* weight_dest(Smem& sm, int i) {
  using W = WeightIndex<LFP>;
  if (i < W::n1) return sm.w1 + kmaj(i / LFP, i % LFP, LFP);
  if (i < W::n2) { const int j = i - W::n1; return sm.w2 + kmaj(j / kH, j % kH, kH); }
  if (i < W::n3) { const int j = i - W::n2; return sm.w3 + kmaj(j / 32, j % 32, 32); }
  if (i < W::n4) { const int j = i - W::n3; return sm.w4 + kmaj(j / kH, j % kH, kH); }
  const int j = i - W::n4;
  return sm.w5 + kmaj(j / kH, j % kH, kH);
}
// Weights i = t + j nthreads, j < kBatch, of the index space above: fetched into v, then stored (the split lets a
// caller overlap the fetch's round trip with other work).
template <int LFP, int kBatch>
__device__ __forceinline__ void weights_fetch(const GridParams& g, const float* __restrict__ P, int t, int nthreads,
                                              float (&v)[kBatch]) {
  const int64_t off4 = g.extra >= 1 ? g.mlp_off[5] : g.mlp_off[3];  // single network: its hidden layer 2
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const int i = t + j * nthreads;
    v[j] = i < WeightIndex<LFP>::total ? weight_fetch<LFP>(g, P, off4, i) : 0.f;
  }
}
template <int LFP, int kBatch, class Smem>
__device__ __forceinline__ void weights_store(Smem& sm, const GridParams& g, int t, int nthreads,
                                              const float (&v)[kBatch]) {
  const bool f16 = g.f16 != 0;
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const int i = t + j * nthreads;
    if (i < WeightIndex<LFP>::total) *reinterpret_cast<uint16_t*>(weight_dest<LFP>(sm, i)) = pack1(v[j], f16);
  }
}
// All weights by thread t of nthreads, kBatch loads in flight per thread.
template <int LFP, int kBatch, class Smem>
__device__ void load_weights(Smem& sm, const GridParams& g, const float* __restrict__ P, int t, int nthreads) {
  for (int base = t; base < WeightIndex<LFP>::total; base += kBatch * nthreads) {
    float v[kBatch];
    weights_fetch<LFP, kBatch>(g, P, base, nthreads, v);
    weights_store<LFP, kBatch>(sm, g, base, nthreads, v);
  }
}

__device__ __forceinline__ void red_add4f(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
// Adds TMEM columns [c0, c0 + ncols) of this thread's lane (row o of a weight gradient when valid), times scale, to
// row[0 .. in): columns in 16-column blocks, the blocks dealt to the nh flushing warps of the same lanes (half h),
// starting at block rot (mod the block count).  tcgen05.ld is warp-collective, so every lane loads and only the valid
// rows add.
__device__ __forceinline__ void flush_rows(uint32_t lane_taddr, uint32_t c0, int ncols, bool valid, float* row, int in,
                                           float scale, int h, int nh, int rot) {
  const int nblk = ncols / 16;
  for (int i = h; i < nblk; i += nh) {
    const int blk = (i + rot) % nblk;
    float v[16];
    tmem_ld16(lane_taddr + c0 + 16u * (uint32_t)blk, v);
    tmem_wait_ld();
    if (!valid) continue;
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
      const int k = 16 * blk + j;
      if (k >= in) break;
      float* a = row + k;
      if (k + 3 < in && (reinterpret_cast<uintptr_t>(a) & 15u) == 0) {
        if (v[j] != 0.f || v[j + 1] != 0.f || v[j + 2] != 0.f || v[j + 3] != 0.f)
          red_add4f(a, v[j] * scale, v[j + 1] * scale, v[j + 2] * scale, v[j + 3] * scale);
      } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (k + jj < in && v[j + jj] != 0.f) atomicAdd(a + jj, v[j + jj] * scale);
      }
    }
  }
}
// Adds TMEM columns c0 .. c0 + nout - 1 of this thread's lane (input k of a transposed weight gradient), times
// scale, to col[o * 64] for output o (col = the gradient of output 0 at input k): a warp's lanes add 32 consecutive
// floats per output.  The 16 columns are loaded once; flushing warp h of nh takes every nh-th output.
__device__ __forceinline__ void flush_cols(uint32_t lane_taddr, uint32_t c0, int nout, float* col, float scale, int h,
                                           int nh) {
  float v[16];
  tmem_ld16(lane_taddr + c0, v);
  tmem_wait_ld();
#pragma unroll
  for (int o = 0; o < 16; ++o)
    if (o < nout && o % nh == h && v[o] != 0.f) atomicAdd(col + o * kH, v[o] * scale);
}
// Adds the TMEM weight-gradient accumulators of one object, times scale (the inverse of the FP16 path's gradient
// scale, else 1), to its FP32 gradient.  Lanes 0..63 hold the rows (dW1, dW3, dW4) or the inputs (dW2, dW5), which
// warps w with w % 4 < 2 can read; with nthreads >= 256 warps 0, 1, 4 and 5 share the work (warps 4 and 5 take every
// other 16-column block or output).  Every CTA that finishes an object flushes the same few kilobytes at about the
// same time, so each CTA starts at a different matrix and column block: the reductions of different CTAs then mostly
// meet different L2 lines.  flush_dw_lanes: the matrices' rows (or inputs) 32 q .. 32 q + 31 of one lane group (lt:
// the group's TMEM lane address), flushing warp h of nh.
template <int LFP>
__device__ void flush_dw_lanes(uint32_t lt, int q, int h, int nh, const GridParams& g, float* __restrict__ grad,
                               float scale) {
  const int o = 32 * q + (threadIdx.x & 31);  // this lane's output row, or input for the transposed ones
  const int rot = (int)blockIdx.x;
  const int nmat = g.single_net ? 2 + g.extra : 5;
  for (int i = 0; i < nmat; ++i) {
    const int m = (i + rot) % nmat;
    if (m == 0) {  // first layer [64][LF]
      flush_rows(lt, kColDW1, LFP, true, grad + g.mlp_off[0] + o * g.LF, g.LF, scale, h, nh, rot);
    } else if (m == 1) {  // density output layer [16][64], transposed (fed by H1 or the last hidden layer)
      flush_cols(lt, kColDW2, 16, grad + g.mlp_off[1] + o, scale, h, nh);
    } else if (g.single_net) {  // hidden layers 2 and 3 [64][64] in the DW4 and DW3 columns
      const int x = m - 2;
      flush_rows(lt, x == 0 ? kColDW4 : kColDW3, kH, true, grad + g.mlp_off[5 + x] + o * kH, kH, scale, h, nh, rot);
    } else if (m == 2) {  // colour input [64][cin]
      flush_rows(lt, kColDW3, 32, true, grad + g.mlp_off[2] + o * g.cin, g.cin, scale, h, nh, rot);
    } else if (m == 3) {  // [64][64]
      flush_rows(lt, kColDW4, kH, true, grad + g.mlp_off[3] + o * kH, kH, scale, h, nh, rot);
    } else {  // colour output [3][64], transposed
      flush_cols(lt, kColDW5, 3, grad + g.mlp_off[4] + o, scale, h, nh);
    }
  }
}
template <int LFP>
__device__ void flush_dw(uint32_t tm, const GridParams& g, float* __restrict__ grad, float scale, int nthreads) {
  const int w = threadIdx.x >> 5;
  if ((w & 3) >= 2 || w >= nthreads / 32) return;
  const int q = w & 1;                     // lanes 32 q .. 32 q + 31
  const int nh = nthreads >= 256 ? 2 : 1;  // flushing warps per lane group
  flush_dw_lanes<LFP>(tm + ((uint32_t)(32 * q) << 16), q, (w >> 2) & (nh - 1), nh, g, grad, scale);
}
// The accumulators at TMEM column base dwb of one warpgroup, flushed by that warpgroup's warps 0 and 1.
template <int LFP>
__device__ void flush_dw_group(uint32_t dwb, const GridParams& g, float* __restrict__ grad, float scale) {
  const int q = (threadIdx.x >> 5) & 3;
  if (q >= 2) return;
  flush_dw_lanes<LFP>(dwb + ((uint32_t)(32 * q) << 16), q, 0, 1, g, grad, scale);
}

__device__ __forceinline__ float warp_incl_prefix(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}
__device__ __forceinline__ float warp_incl_suffix(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float n = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += n;
  }
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-ray inputs of the losses of Eq. 7-11: background colour (the random colour of Eq. 8), target colour, sparse
// depth (NaN without one) and class.
struct RayTarget {
  float bg0, bg1, bg2, t0, t1, t2, dep;
  int cls;
};
__device__ __forceinline__ RayTarget ray_target(const RayBuf& R, int64_t r) {
  RayTarget q;
  q.bg0 = R.bg[3 * r]; q.bg1 = R.bg[3 * r + 1]; q.bg2 = R.bg[3 * r + 2];
  q.t0 = R.rgb[3 * r]; q.t1 = R.rgb[3 * r + 1]; q.t2 = R.rgb[3 * r + 2];
  q.dep = R.depth[r];
  q.cls = R.cls[r];
  return q;
}

// Losses of Eq. 7-11 of one ray from its rendered colour and depth (every term divided by the batch size B through
// invB in the gradients; the sums are accumulated unscaled).
struct RayLoss {
  float loss, l_rgb, l_rr, l_dep, l_den;
  float gC0, gC1, gC2, gD, gdir;
};
__device__ __forceinline__ RayLoss ray_loss(const GridParams& g, const RayTarget& tg, float Ch0, float Ch1, float Ch2,
                                            float Dh, float ssum, float invB) {
  RayLoss q{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int cls = tg.cls;
  if (cls != kClsOccluder) {
    const float t0 = cls == kClsObject ? tg.t0 : tg.bg0;
    const float t1 = cls == kClsObject ? tg.t1 : tg.bg1;
    const float t2 = cls == kClsObject ? tg.t2 : tg.bg2;
    const float e0 = Ch0 - t0, e1 = Ch1 - t1, e2 = Ch2 - t2;
    const float sq = e0 * e0 + e1 * e1 + e2 * e2;
    q.loss += sq;
    if (cls == kClsObject) q.l_rgb = sq; else q.l_rr = sq;
    q.gC0 = 2.f * e0 * invB; q.gC1 = 2.f * e1 * invB; q.gC2 = 2.f * e2 * invB;
    const float dep = tg.dep;
    if (isfinite(dep)) {
      const float e = Dh - dep;
      q.loss += g.lambda1 * fabsf(e);
      q.l_dep = fabsf(e);
      q.gD = g.lambda1 * (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) * invB;
    }
    if (cls == kClsBackground) {
      q.loss += g.lambda2 * ssum;
      q.l_den = ssum;
      q.gdir = g.lambda2 * invB;
    }
  }
  return q;
}
__device__ __forceinline__ void add_ray_loss(BatchDyn* dyn, int bi, const RayLoss& q, int32_t* status) {
  float* L = dyn[bi].loss;
  atomicAdd(L + 0, q.loss);
  if (q.l_rgb != 0.f) atomicAdd(L + 1, q.l_rgb);
  if (q.l_rr != 0.f) atomicAdd(L + 2, q.l_rr);
  if (q.l_dep != 0.f) atomicAdd(L + 3, q.l_dep);
  if (q.l_den != 0.f) atomicAdd(L + 4, q.l_den);
  if (!isfinite(q.loss) && status) atomicOr(status, 1);
}

// Eq. 6 + Eq. 7-11 + adjoint for one ray whose samples occupy slots [base, base + P) of the tile.
template <class Bufs>
__device__ RayLoss composite_ray(Bufs& sm, const GridParams& g, RayBuf R, int64_t r, int base, int P,
                                 const RayTarget& tg, float invB) {
  const int lane = threadIdx.x & 31;
  const float bg0 = tg.bg0, bg1 = tg.bg1, bg2 = tg.bg2;
  float carry = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Dh = 0.f, ssum = 0.f;
  for (int c = 0; c < P; c += 32) {
    const int j = c + lane;
    const bool in = j < P && sm.valid[base + j];
    const int s = base + (j < P ? j : 0);
    const float sg = in ? sm.sig[s] : 0.f, dt = in ? sm.dt[s] : 0.f, tt = in ? sm.t[s] : 0.f;
    const float sd = sg * dt;
    const float incl = warp_incl_prefix(sd, lane);
    float excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.f;
    const float Pf = carry + excl;
    const float w = expf(-Pf) * (-expm1f(-sd));
    if (in) {
      C0 = fmaf(w, sm.rgb[0][s], C0);
      C1 = fmaf(w, sm.rgb[1][s], C1);
      C2 = fmaf(w, sm.rgb[2][s], C2);
      Dh = fmaf(w, tt, Dh);
      ssum += sg;
    }
    if (j < P) sm.dsig[s] = Pf;  // exclusive prefix, consumed by the adjoint below
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  C0 = warp_sum(C0); C1 = warp_sum(C1); C2 = warp_sum(C2); Dh = warp_sum(Dh); ssum = warp_sum(ssum);
  const float Tend = expf(-carry);
  const float Ch0 = fmaf(Tend, bg0, C0), Ch1 = fmaf(Tend, bg1, C1), Ch2 = fmaf(Tend, bg2, C2);
  if (lane == 0) {
    float* o = R.out + 6 * r;
    o[0] = Ch0; o[1] = Ch1; o[2] = Ch2; o[3] = Dh; o[4] = -expm1f(-carry); o[5] = ssum;
  }
  // losses of Eq. 7-11 (every term divided by the batch size B)
  const RayLoss q = ray_loss(g, tg, Ch0, Ch1, Ch2, Dh, ssum, invB);
  const float gC0 = q.gC0, gC1 = q.gC1, gC2 = q.gC2, gD = q.gD, gdir = q.gdir;
  // adjoint, chunks in reverse order
  float SC0 = 0.f, SC1 = 0.f, SC2 = 0.f, SD = 0.f;
  const float bgterm = Tend * (gC0 * bg0 + gC1 * bg1 + gC2 * bg2);
  for (int c = ((P - 1) / 32) * 32; c >= 0; c -= 32) {
    const int j = c + lane;
    const bool in = j < P && sm.valid[base + j];
    const int s = base + (j < P ? j : 0);
    const float sg = in ? sm.sig[s] : 0.f, dt = in ? sm.dt[s] : 0.f, tt = in ? sm.t[s] : 0.f;
    const float Pf = (j < P) ? sm.dsig[s] : 0.f;
    const float c0 = in ? sm.rgb[0][s] : 0.f, c1 = in ? sm.rgb[1][s] : 0.f, c2 = in ? sm.rgb[2][s] : 0.f;
    const float sd = sg * dt;
    const float Tn = expf(-(Pf + sd));
    const float w = in ? expf(-Pf) * (-expm1f(-sd)) : 0.f;
    float s0 = warp_incl_suffix(w * c0, lane), s1 = warp_incl_suffix(w * c1, lane);
    float s2 = warp_incl_suffix(w * c2, lane), s3 = warp_incl_suffix(w * tt, lane);
    float e0 = __shfl_down_sync(0xffffffffu, s0, 1), e1 = __shfl_down_sync(0xffffffffu, s1, 1);
    float e2 = __shfl_down_sync(0xffffffffu, s2, 1), e3 = __shfl_down_sync(0xffffffffu, s3, 1);
    if (lane == 31) e0 = e1 = e2 = e3 = 0.f;
    float gs = gC0 * (Tn * c0 - (SC0 + e0)) + gC1 * (Tn * c1 - (SC1 + e1)) + gC2 * (Tn * c2 - (SC2 + e2)) - bgterm;
    gs += gD * (Tn * tt - (SD + e3));
    gs = dt * gs + gdir;
    if (j < P) {
      sm.dsig[s] = in ? gs : 0.f;
      sm.drgb[0][s] = in ? gC0 * w : 0.f;
      sm.drgb[1][s] = in ? gC1 * w : 0.f;
      sm.drgb[2][s] = in ? gC2 * w : 0.f;
    }
    SC0 += __shfl_sync(0xffffffffu, s0, 0);
    SC1 += __shfl_sync(0xffffffffu, s1, 0);
    SC2 += __shfl_sync(0xffffffffu, s2, 0);
    SD += __shfl_sync(0xffffffffu, s3, 0);
  }
  return q;
}

// Compositing, losses and adjoint of the rays of up to two tiles (rays j < nr0 in tile_of(0), the others in
// tile_of(1)), ray j by warp j mod nwarps.  Lane k of a warp first fetches the plan entry and targets of the warp's
// k-th ray, so that all of a warp's fetches are in flight together instead of three dependent round trips per ray;
// the warp's loss terms go to the object's sums in one set of atomics.
template <class TileOf>
__device__ __forceinline__ void composite_rays(TileOf tile_of, int nr0, int nr_all, int warp, int nwarps,
                                               const GridParams& g, const BatchDesc& b, RayBuf R, BatchDyn* dyn,
                                               int bi, float invB, int32_t* status) {
  constexpr uint32_t kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  RayLoss sum{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // this warp's loss terms, added once at the end
  for (int k0 = 0; warp + nwarps * k0 < nr_all; k0 += 32) {
    const int j = warp + nwarps * (k0 + lane);
    int u = 0, r = 0, base = 0, P = 0;
    RayTarget tg{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, kClsOccluder};
    if (j < nr_all) {
      u = j < nr0 ? 0 : 1;
      const int pi = tile_of(u).pfirst + (j < nr0 ? j : j - nr0);
      r = b.plan_perm[pi];
      base = b.plan_rstart[pi];
      P = (int)R.count[r];
      tg = ray_target(R, r);
    }
    const int rem = (nr_all - 1 - warp) / nwarps + 1 - k0;  // this warp's rays from k0 on
    const int n = rem < 32 ? rem : 32;
    for (int k = 0; k < n; ++k) {
      const int uk = __shfl_sync(kAll, u, k), rk = __shfl_sync(kAll, r, k);
      const int bk = __shfl_sync(kAll, base, k), pk = __shfl_sync(kAll, P, k);
      RayTarget tk;
      tk.bg0 = __shfl_sync(kAll, tg.bg0, k); tk.bg1 = __shfl_sync(kAll, tg.bg1, k);
      tk.bg2 = __shfl_sync(kAll, tg.bg2, k); tk.t0 = __shfl_sync(kAll, tg.t0, k);
      tk.t1 = __shfl_sync(kAll, tg.t1, k); tk.t2 = __shfl_sync(kAll, tg.t2, k);
      tk.dep = __shfl_sync(kAll, tg.dep, k); tk.cls = __shfl_sync(kAll, tg.cls, k);
      const RayLoss q = composite_ray(tile_of(uk), g, R, rk, bk, pk, tk, invB);
      sum.loss += q.loss; sum.l_rgb += q.l_rgb; sum.l_rr += q.l_rr; sum.l_dep += q.l_dep; sum.l_den += q.l_den;
    }
  }
  if (lane == 0 && warp < nr_all) add_ray_loss(dyn, bi, sum, status);
}

// Hash encoding of levels [L0, L1) of one sample from the FP16 table, two levels per round so that 16 gathers are
// in flight; e holds the LFP features (levels outside [L0, L1) are left untouched).
template <int LFP, int L0, int L1>
__device__ __forceinline__ void gather_levels(const GridParams& g, const ObjectDev* ob, const float p[3], float* e) {
  const __half2* tab = reinterpret_cast<const __half2*>(ob->table_h);
  const float hf[3] = {ob->half[0], ob->half[1], ob->half[2]};
  const float ie[3] = {ob->inv_ext[0], ob->inv_ext[1], ob->inv_ext[2]};
#pragma unroll
  for (int l = L0; l < L1; l += 2) {
    const bool has0 = l < g.L, has1 = (l + 1 < L1) && (l + 1 < g.L);
    Corners c0, c1;
    if (has0) level_corners(g, l, p, hf, ie, c0);
    if (has1) level_corners(g, l + 1, p, hf, ie, c1);
    __half2 v0[8], v1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v0[k] = has0 ? __ldg(tab + g.off[l] + c0.idx[k]) : __half2{};
      v1[k] = has1 ? __ldg(tab + g.off[l + 1] + c1.idx[k]) : __half2{};
    }
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 f0 = __half22float2(v0[k]), f1 = __half22float2(v1[k]);
      if (has0) { a0 = fmaf(c0.w[k], f0.x, a0); a1 = fmaf(c0.w[k], f0.y, a1); }
      if (has1) { b0 = fmaf(c1.w[k], f1.x, b0); b1 = fmaf(c1.w[k], f1.y, b1); }
    }
    e[2 * l] = a0; e[2 * l + 1] = a1;
    if (l + 1 < L1) { e[2 * l + 2] = b0; e[2 * l + 3] = b1; }
  }
}

// The sample of one slot: candidate i of ray rl of the object (same FP32 operations as the sampling kernels).
// Work items (tile pairs, or tiles) of CTA c of a grid: a contiguous range of the plan (chunk = 0), or chunks of
// `chunk` consecutive items dealt round-robin over the CTAs (CTA c takes items [c chunk, c chunk + chunk), then
// [(c + grid) chunk, ...)), so that all CTAs work on the same few objects at a time and those objects' tables and
// gradients stay in L2; larger chunks give each CTA longer runs of one object (fewer weight reloads and
// weight-gradient flushes).
struct WorkOrder {
  int total, grid, c, chunk, lo, hi;
  __device__ WorkOrder(int total_, int grid_, int c_, int chunk_) : total(total_), grid(grid_), c(c_), chunk(chunk_) {
    lo = chunk ? 0 : (int)((int64_t)total * c / grid);
    hi = chunk ? 0 : (int)((int64_t)total * (c + 1) / grid);
  }
  __device__ int count() const {
    if (!chunk) return hi - lo;
    const int round = grid * chunk, full = total / round, rem = total - full * round;
    const int extra = rem - c * chunk;
    return full * chunk + (extra < 0 ? 0 : (extra > chunk ? chunk : extra));
  }
  __device__ int item(int it) const { return chunk ? (it / chunk) * grid * chunk + c * chunk + it % chunk : lo + it; }
};

struct SlotSample {
  float x, y, z, t, dt;
  int valid;
  int ray;  // global ray index of the slot, or -1 for a slot outside the tile's rays
};

// Position of the (j+1)-th set bit of x (j < popc(x)), by halving popcounts.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int j) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const int c = __popc(x & ((1u << w) - 1u));
    if (j >= c) {
      j -= c;
      x >>= w;
      pos += w;
    }
  }
  return pos;
}

// The sample of slot s of a planned tile (see kPlanMaxCount): the slot table gives its ray and the index j of its
// live sample; the j-th live candidate i is found in the ray's live-candidate mask; same FP32 operations as the
// sampling kernels.  Slots past the tile's used ones hold no sample.
__device__ __forceinline__ SlotSample plan_sample(const GridParams& g, const BatchDesc& b, const RayBuf& R,
                                                  const ObjectDev* ob, int bi, int4 tile, int s) {
  SlotSample q{0.f, 0.f, 0.f, 0.f, 0.f, 0, -1};
  if (s >= (tile.z >> 8)) return q;
  const int2 e = b.plan_slot[(int64_t)tile.y * kTile + s];
  const int r = e.x;
  if (!ROMAP_IN_BOUNDS(r >= b.ray_base[bi] && r < b.ray_base[bi + 1] && e.y >= 0, g.status)) return q;
  q.ray = r;
  // everything the sample needs from the ray, loaded at once (one round trip after the slot's)
  const uint4 m4 = *reinterpret_cast<const uint4*>(R.mask + 4 * (int64_t)r);
  const uint32_t cnt = R.count[r];
  const float tn = R.tn[r], tf = R.tf[r];
  const float o0 = R.o[3 * r], o1 = R.o[3 * r + 1], o2 = R.o[3 * r + 2];
  const float d0 = R.d[3 * r], d1 = R.d[3 * r + 1], d2 = R.d[3 * r + 2];
  int j = e.y;
  if ((uint32_t)j >= cnt) return q;
  // candidate index of the j-th live candidate: its mask word, then its bit
  uint32_t m = m4.x;
  int wd = 0;
  if (j >= __popc(m)) {
    j -= __popc(m); m = m4.y; wd = 1;
    if (j >= __popc(m)) {
      j -= __popc(m); m = m4.z; wd = 2;
      if (j >= __popc(m)) { j -= __popc(m); m = m4.w; wd = 3; }
    }
  }
  const int i = 32 * wd + nth_set_bit(m, j);
  const int N = g.n_samples;
  const int rl = r - b.ray_base[bi];
  const float step_len = __fdiv_rn(__fsub_rn(tf, tn), (float)N);
  const uint32_t step = ob->step;
  q.t = candidate_t(tn, step_len, i, ob->key0, ob->key1, step, (uint32_t)rl, 1);
  const float tnext = (i + 1 < N) ? candidate_t(tn, step_len, i + 1, ob->key0, ob->key1, step, (uint32_t)rl, 1) : tf;
  q.dt = __fsub_rn(tnext, q.t);
  q.x = __fadd_rn(o0, __fmul_rn(q.t, d0));
  q.y = __fadd_rn(o1, __fmul_rn(q.t, d1));
  q.z = __fadd_rn(o2, __fmul_rn(q.t, d2));
  q.valid = 1;
  return q;
}

}  // namespace tc
}  // namespace romap
