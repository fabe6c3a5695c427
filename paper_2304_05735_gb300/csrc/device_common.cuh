// Device helpers shared by the sampling, FP32 tile and tensor-core tile kernels: the ray/box slab test, the
// occupancy lookup, stratified sample positions and hash-grid corners.  The FP32 arithmetic of the slab test, the
// sample positions and the corner selection is written with round-to-nearest intrinsics in one fixed order (no
// contraction into FMA), so that every kernel and the oracle produce the same bits.
#pragma once
#include "romap_internal.cuh"

namespace romap {

// ---------------------------------------------------------------------------
// Ray/box slab test (box [-half, half]); returns hit.
// ---------------------------------------------------------------------------
__device__ inline bool slab(const float o[3], const float d[3], const float half[3], float& tn, float& tf) {
  float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float lo = -half[a], hi = half[a];
    float inv = __fdiv_rn(1.0f, d[a]);
    float ta = __fmul_rn(__fsub_rn(lo, o[a]), inv);
    float tb = __fmul_rn(__fsub_rn(hi, o[a]), inv);
    float mn = fminf(ta, tb), mx = fmaxf(ta, tb);
    t0 = (a == 0) ? mn : fmaxf(t0, mn);
    t1 = (a == 0) ? mx : fminf(t1, mx);
  }
  tn = fmaxf(t0, 0.0f);
  tf = t1;
  return t1 > tn;
}

__device__ inline bool occupied(const uint64_t* occ, float x, float y, float z, const float half[3],
                                const float inv_ext[3]) {
  if (!occ) return true;
  float p[3] = {x, y, z};
  uint32_t c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u = fminf(fmaxf(__fmul_rn(__fsub_rn(p[a], -half[a]), inv_ext[a]), 0.0f), 1.0f);
    int ci = (int)__fmul_rn(u, 64.0f);
    c[a] = (uint32_t)(ci > 63 ? 63 : ci);
  }
  uint32_t bit = c[0] + 64u * c[1] + 4096u * c[2];
  return (__ldg(occ + (bit >> 6)) >> (bit & 63u)) & 1ull;
}

// Stratified candidates t_i = t_near + (i + u_i) dt_N, delta_i = t_{i+1} - t_i
// (last: t_far - t_{N-1}), x_i = o + t_i d; f(i, t, delta, x, y, z, live).
// u_i is word i mod 4 of the Philox draw (step, slot, jitter, i / 4), or 1/2 without jitter.  The candidates are
// walked in blocks of 16 whose four draws are independent of one another, so that their rounds overlap instead of
// running back to back; the next block's first draw comes with them (delta of the block's last candidate).
template <class Fn>
__device__ inline void for_candidates(const float o[3], const float d[3], float tn, float tf, int N, uint32_t k0,
                                      uint32_t k1, uint32_t step, uint32_t slot, int jitter, const uint64_t* occ,
                                      const float half[3], const float inv_ext[3], Fn f) {
  const float step_len = __fdiv_rn(__fsub_rn(tf, tn), (float)N);
  auto t_at = [&](int i, float u) { return __fadd_rn(tn, __fmul_rn(__fadd_rn((float)i, u), step_len)); };
  auto draw = [&](int q) -> U4 {
    if (!jitter || 4 * q >= N) return U4{0u, 0u, 0u, 0u};  // not needed
    return philox(step, slot, kPurposeJitter, (uint32_t)q, k0, k1);
  };
  auto u_of = [&](const U4& r, int w) { return jitter ? u01(u4_word(r, w)) : 0.5f; };
  U4 r0 = draw(0);
  float t_cur = t_at(0, u_of(r0, 0));
  for (int b0 = 0; b0 < N; b0 += 16) {
    const int q = b0 >> 2;
    const U4 r1 = draw(q + 1), r2 = draw(q + 2), r3 = draw(q + 3), rn = draw(q + 4);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int i = b0 + j;
      if (i >= N) break;
      const int jn = j + 1;
      const float u_next = jn < 4 ? u_of(r0, jn & 3) : jn < 8 ? u_of(r1, jn & 3) : jn < 12 ? u_of(r2, jn & 3)
                           : jn < 16 ? u_of(r3, jn & 3) : u_of(rn, 0);
      const float t_next = i + 1 < N ? t_at(i + 1, u_next) : tf;
      float dt = __fsub_rn(t_next, t_cur);
      float x = __fadd_rn(o[0], __fmul_rn(t_cur, d[0]));
      float y = __fadd_rn(o[1], __fmul_rn(t_cur, d[1]));
      float z = __fadd_rn(o[2], __fmul_rn(t_cur, d[2]));
      f(i, t_cur, dt, x, y, z, occupied(occ, x, y, z, half, inv_ext));
      t_cur = t_next;
    }
    r0 = rn;
  }
}

// Non-returning vector atomic add of two floats (red.global.add.v2.f32): the scatter never reads the old value.
__device__ __forceinline__ void red_add2(float2* addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}
// 16-byte aligned addr
__device__ __forceinline__ void red_add4(float2* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
// Scatter of one level: the 8 corner gradients a[2k], a[2k+1] (features 0, 1 of corner k) added into the FP32
// gradient of the level (gt points at the level's first entry, 16-byte aligned since levels start at multiples of 8
// entries).  Corners k and k+1 differ by one step in x; when their entries form an aligned pair {2m, 2m+1} (x even on
// a hashed level, an even index on a dense one) one 16-byte vector add covers both, which saves one L1->L2 request.
__device__ __forceinline__ void scatter_sums(float2* gt, const uint32_t idx[8], const float a[16]) {
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    const uint32_t i0 = idx[k], i1 = idx[k + 1];
    if ((i0 ^ i1) == 1u) {
      if (i0 < i1) red_add4(gt + i0, a[2 * k], a[2 * k + 1], a[2 * k + 2], a[2 * k + 3]);
      else red_add4(gt + i1, a[2 * k + 2], a[2 * k + 3], a[2 * k], a[2 * k + 1]);
    } else {
      red_add2(gt + i0, a[2 * k], a[2 * k + 1]);
      red_add2(gt + i1, a[2 * k + 2], a[2 * k + 3]);
    }
  }
}
// The same for one sample: corner k receives (w_k d0, w_k d1).
__device__ __forceinline__ void scatter_corners(float2* gt, const uint32_t idx[8], const float w[8], float d0,
                                                float d1) {
  float a[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[2 * k] = w[k] * d0;
    a[2 * k + 1] = w[k] * d1;
  }
  scatter_sums(gt, idx, a);
}

// Deterministic mode: one contribution added to a 64-bit fixed-point accumulator (kFixBits fractional bits), rounded
// once to nearest.  Zero is skipped; a NaN or a contribution beyond kFixMaxContribution is not added and sets
// kStatusFixRange (NaN also kStatusNonfinite) so that the step reports it.
__device__ __forceinline__ void red_add_fix(unsigned long long* addr, float v, int32_t* status, int bits = kFixBits,
                                            float max_abs = kFixMaxContribution) {
  if (v == 0.0f) return;
  if (!(fabsf(v) <= max_abs)) {
    if (status) atomicOr(status, (v != v) ? (kStatusFixRange | kStatusNonfinite) : kStatusFixRange);
    return;
  }
  const long long q = __double2ll_rn(ldexp((double)v, bits));
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(addr), "l"((unsigned long long)q) : "memory");
}
// Fixed-point scatter of one level (gt points at the level's first entry, F = 2 accumulators per entry).
__device__ __forceinline__ void scatter_corners_fix(unsigned long long* gt, const uint32_t idx[8], const float w[8],
                                                    float d0, float d1, int32_t* status) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    red_add_fix(gt + 2 * (size_t)idx[k], w[k] * d0, status);
    red_add_fix(gt + 2 * (size_t)idx[k] + 1, w[k] * d1, status);
  }
}

// Position of candidate i of a ray (same operations as for_candidates).
__device__ inline float candidate_t(float tn, float step_len, int i, uint32_t k0, uint32_t k1, uint32_t step,
                                    uint32_t slot, int jitter) {
  float u = 0.5f;
  if (jitter) u = u01(u4_word(philox(step, slot, kPurposeJitter, (uint32_t)i >> 2, k0, k1), i & 3));
  return __fadd_rn(tn, __fmul_rn(__fadd_rn((float)i, u), step_len));
}

// ---------------------------------------------------------------------------
// Hash-grid corners of one level for an object-frame point (FP32, fixed
// order): u = clamp((x + half) inv_ext, 0, 1), pos = u N_l, i0 =
// min(floor(pos), N_l - 1), f = pos - i0; dense index x + y(N+1) + z(N+1)^2
// or spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861) mod T.
// ---------------------------------------------------------------------------
struct Corners {
  uint32_t idx[8];
  float w[8];
};

// Cell of level l holding p: its lower corner i0 and the fractions f within it.
__device__ __forceinline__ void level_cell(const GridParams& g, int l, const float p[3], const float half[3],
                                           const float inv_ext[3], int i0[3], float f[3]) {
  const int N = g.res[l];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u = fminf(fmaxf(__fmul_rn(__fsub_rn(p[a], -half[a]), inv_ext[a]), 0.0f), 1.0f);
    float pos = __fmul_rn(u, (float)N);
    int i = (int)floorf(pos);
    i = i > N - 1 ? N - 1 : i;
    i0[a] = i;
    f[a] = __fsub_rn(pos, (float)i);
  }
}
// Table index of corner k (bits x, y, z) of the cell with lower corner i0 (T = 2^log2_table_size, so the modulo of
// the spatial hash is a mask).
__device__ __forceinline__ uint32_t corner_index(const GridParams& g, int l, const int i0[3], int k) {
  const uint32_t n1 = (uint32_t)g.res[l] + 1u;
  const uint32_t cx = (uint32_t)(i0[0] + (k & 1));
  const uint32_t cy = (uint32_t)(i0[1] + ((k >> 1) & 1));
  const uint32_t cz = (uint32_t)(i0[2] + ((k >> 2) & 1));
  const uint32_t idx =
      g.dense[l] ? (cx + cy * n1 + cz * n1 * n1) : (((cx * 1u) ^ (cy * 2654435761u) ^ (cz * 805459861u)) & (g.T - 1u));
  if (!ROMAP_IN_BOUNDS(idx < (g.dense[l] ? n1 * n1 * n1 : g.T), g.status)) return 0u;
  return idx;
}
// Trilinear weight of corner k for the fractions f.
__device__ __forceinline__ float corner_weight(const float f[3], int k) {
  const float wx = (k & 1) ? f[0] : 1.0f - f[0];
  const float wy = ((k >> 1) & 1) ? f[1] : 1.0f - f[1];
  const float wz = ((k >> 2) & 1) ? f[2] : 1.0f - f[2];
  return wx * wy * wz;
}

__device__ inline void level_corners(const GridParams& g, int l, const float p[3], const float half[3],
                                     const float inv_ext[3], Corners& c) {
  int i0[3];
  float f[3];
  level_cell(g, l, p, half, inv_ext, i0, f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c.idx[k] = corner_index(g, l, i0, k);
    c.w[k] = corner_weight(f, k);
  }
}

}  // namespace romap
