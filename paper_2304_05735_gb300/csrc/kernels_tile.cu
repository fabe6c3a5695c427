// FP32 tile kernel: multiresolution hash encoding (Mueller et al. 2022, the
// encoding of Sec. V) and the tiny density/colour MLP (Sec. V, hidden 64),
// forward and backward, on tiles of 128 samples of one object.
//
// One persistent CTA per SM walks a contiguous range of tiles, so that it
// touches one or two objects and keeps that object's weights in shared
// memory.  Within a tile every layer is a small GEMM over the 128 samples,
// computed with register blocking from activations staged in shared memory
// as [feature][sample] rows (row stride kAS floats, padded for conflict-free
// float4 access).  The backward pass recomputes the forward activations
// (no per-sample activation traffic to HBM), forms the input gradients layer
// by layer, accumulates the weight gradients of every tile of the same
// object in registers and flushes them with one atomic add per weight per
// object change, and scatters the encoding gradient into the hash-table
// gradient with vector atomics (red.global.add.v2.f32).
#include "device_common.cuh"
#include "romap_internal.cuh"

namespace romap {

constexpr int kW6S = kH + 4;  // row stride of w6: float4-aligned rows, conflict-free column reads

template <int LFP>
struct TileSmem {
  // weights: row-major [out][in] (backward input gradients) and transposed (forward)
  float w1[kH * LFP];
  float w1t[LFP * kH];
  float w2[kDOut * kH];
  float w2t[kH * kDOut];
  float w3[kH * kCinPad];
  float w3t[kCinPad * kH];
  float w4[kH * kH];
  float w4t[kH * kH];
  float w5[kC3Rows * kH];
  float w6[kH * kW6S];    // single-network hidden layer 3, [out][in] only (its forward reads it transposed)
  // activations [feature][sample]
  float E[LFP * kAS];     // encoding, then dL/dencoding
  float H1[kH * kAS];     // density hidden, then its gradient
  float OC[kOC * kAS];    // row 0 log-density, rows 1..15 geometry, rows 16..18 direction; then dL/dout
  float H2[kH * kAS];
  float H3[kH * kAS];
  float DL[kC3Rows * kAS];
  float sig[kTile];
  float rgb[3][kTile];
  float px[3][kTile];
  uint32_t ray[kTile];
  int cur_obj;
};

static_assert(sizeof(TileSmem<32>) <= 227 * 1024, "tile kernel shared memory above the per-CTA limit");

int tile_kernel_smem_bytes(int LF) {
  return LF <= 16 ? (int)sizeof(TileSmem<16>) : (int)sizeof(TileSmem<32>);
}

// ---------------------------------------------------------------------------
// C[m][n] = sum_k A[k][m] B[k][n] for the 128 samples m and N = 16*TN
// outputs.  Thread t owns rows {4 mg + j, 64 + 4 mg + j} (mg = t % 16) and
// columns {TN ng + j} (ng = t / 16).
// ---------------------------------------------------------------------------
template <int TN>
__device__ inline void gemm_tile(const float* __restrict__ A, int K, const float* __restrict__ B, int ldb,
                                 float (&acc)[8][TN]) {
  const int t = threadIdx.x, mg = t & 15, ng = t >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;
  const float* a = A + 4 * mg;
  const float* b = B + TN * ng;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float4 x0 = *reinterpret_cast<const float4*>(a + k * kAS);
    float4 x1 = *reinterpret_cast<const float4*>(a + k * kAS + 64);
    float bv[TN];
    if constexpr (TN == 4) {
      float4 q = *reinterpret_cast<const float4*>(b + k * ldb);
      bv[0] = q.x; bv[1] = q.y; bv[2] = q.z; bv[3] = q.w;
    } else if constexpr (TN == 2) {
      float2 q = *reinterpret_cast<const float2*>(b + k * ldb);
      bv[0] = q.x; bv[1] = q.y;
    } else {
      bv[0] = b[k * ldb];
    }
    float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(xs[i], bv[j], acc[i][j]);
  }
}

// The same product with B given transposed: B[k][n] = BT[n * ldbt + k].
template <int TN>
__device__ inline void gemm_tile_bt(const float* __restrict__ A, int K, const float* __restrict__ BT, int ldbt,
                                    float (&acc)[8][TN]) {
  const int t = threadIdx.x, mg = t & 15, ng = t >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;
  const float* a = A + 4 * mg;
  const float* b = BT + TN * ng * ldbt;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float4 x0 = *reinterpret_cast<const float4*>(a + k * kAS);
    float4 x1 = *reinterpret_cast<const float4*>(a + k * kAS + 64);
    float bv[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) bv[j] = b[j * ldbt + k];
    float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(xs[i], bv[j], acc[i][j]);
  }
}

// Store acc to C[n][m] (row stride kAS) through epi(value, n, m) -> value.
template <int TN, class Epi>
__device__ inline void store_tile(float* C, const float (&acc)[8][TN], Epi epi) {
  const int t = threadIdx.x, mg = t & 15, ng = t >> 4;
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    int n = TN * ng + j;
    float4 v0, v1;
    v0.x = epi(acc[0][j], n, 4 * mg + 0);
    v0.y = epi(acc[1][j], n, 4 * mg + 1);
    v0.z = epi(acc[2][j], n, 4 * mg + 2);
    v0.w = epi(acc[3][j], n, 4 * mg + 3);
    v1.x = epi(acc[4][j], n, 64 + 4 * mg + 0);
    v1.y = epi(acc[5][j], n, 64 + 4 * mg + 1);
    v1.z = epi(acc[6][j], n, 64 + 4 * mg + 2);
    v1.w = epi(acc[7][j], n, 64 + 4 * mg + 3);
    *reinterpret_cast<float4*>(C + n * kAS + 4 * mg) = v0;
    *reinterpret_cast<float4*>(C + n * kAS + 64 + 4 * mg) = v1;
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of one tile: G[o][k] += sum_m D[o][m] X[k][m] for
// o < NO, k < NK.  Thread t owns o = og + (NO/TO) i, k = kg + (NK/TK) j with
// og = t / (NK/TK), kg = t % (NK/TK).
// ---------------------------------------------------------------------------
template <int NO, int NK, int TO, int TK>
__device__ inline void wgrad_tile(const float* __restrict__ D, const float* __restrict__ X, float (&g)[TO][TK]) {
  static_assert((NO / TO) * (NK / TK) == kThreads, "wgrad tiling must cover the block");
  const int t = threadIdx.x, og = t / (NK / TK), kg = t % (NK / TK);
#pragma unroll 2
  for (int m = 0; m < kTile; m += 4) {
    float4 dv[TO], xv[TK];
#pragma unroll
    for (int i = 0; i < TO; ++i) dv[i] = *reinterpret_cast<const float4*>(D + (og + (NO / TO) * i) * kAS + m);
#pragma unroll
    for (int j = 0; j < TK; ++j) xv[j] = *reinterpret_cast<const float4*>(X + (kg + (NK / TK) * j) * kAS + m);
#pragma unroll
    for (int i = 0; i < TO; ++i)
#pragma unroll
      for (int j = 0; j < TK; ++j) {
        float a = g[i][j];
        a = fmaf(dv[i].x, xv[j].x, a);
        a = fmaf(dv[i].y, xv[j].y, a);
        a = fmaf(dv[i].z, xv[j].z, a);
        a = fmaf(dv[i].w, xv[j].w, a);
        g[i][j] = a;
      }
  }
}

template <int NO, int NK, int TO, int TK>
__device__ inline void wgrad_flush(float* __restrict__ dst, int rows, int cols, float (&g)[TO][TK]) {
  const int t = threadIdx.x, og = t / (NK / TK), kg = t % (NK / TK);
#pragma unroll
  for (int i = 0; i < TO; ++i)
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      int o = og + (NO / TO) * i, k = kg + (NK / TK) * j;
      if (o < rows && k < cols && g[i][j] != 0.0f) atomicAdd(dst + o * cols + k, g[i][j]);
      g[i][j] = 0.0f;
    }
}

// Deterministic mode: the same flush into the fixed-point accumulator (called after every tile, so each flushed sum
// covers one tile, whose samples and their order do not depend on the launch: the sums are reproducible).
template <int NO, int NK, int TO, int TK>
__device__ inline void wgrad_flush_fix(unsigned long long* __restrict__ dst, int rows, int cols, float (&g)[TO][TK],
                                       int32_t* status) {
  const int t = threadIdx.x, og = t / (NK / TK), kg = t % (NK / TK);
#pragma unroll
  for (int i = 0; i < TO; ++i)
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      int o = og + (NO / TO) * i, k = kg + (NK / TK) * j;
      if (o < rows && k < cols) red_add_fix(dst + o * cols + k, g[i][j], status);
      g[i][j] = 0.0f;
    }
}

// Stored activations of one tile (ACT): rows [encoding (LFP) | H1 (64) | density-net outputs 0..15 | H2 (64) |
// H3 (64)] x 128 samples, copied as float4 between shared memory and the workspace (to_global: smem -> act).
__host__ __device__ constexpr int act_rows(int lfp) { return lfp + kH + kDOut + kH + kH; }

template <int LFP, bool TO_GLOBAL>
__device__ inline void act_copy(TileSmem<LFP>& sm, float* __restrict__ act) {
  constexpr int kRows = act_rows(LFP), kQ = kTile / 4;
  for (int i = threadIdx.x; i < kRows * kQ; i += kThreads) {
    const int r = i / kQ, q = i % kQ;
    float* row = r < LFP ? sm.E + r * kAS
                 : r < LFP + kH ? sm.H1 + (r - LFP) * kAS
                 : r < LFP + kH + kDOut ? sm.OC + (r - LFP - kH) * kAS
                 : r < LFP + 2 * kH + kDOut ? sm.H2 + (r - LFP - kH - kDOut) * kAS
                 : sm.H3 + (r - LFP - 2 * kH - kDOut) * kAS;
    float4* gp = reinterpret_cast<float4*>(act + (size_t)r * kTile) + q;
    float4* sp = reinterpret_cast<float4*>(row) + q;
    if (TO_GLOBAL) *gp = *sp; else *sp = *gp;
  }
}

template <int TO, int TK>
__device__ inline void zero2(float (&g)[TO][TK]) {
#pragma unroll
  for (int i = 0; i < TO; ++i)
#pragma unroll
    for (int j = 0; j < TK; ++j) g[i][j] = 0.0f;
}

// ---------------------------------------------------------------------------
// The kernel.  MODE 0: forward only (writes sigma and rgb per sample).
// MODE 1: recompute forward, then backward from dL/dsigma and dL/drgb.
// DET (MODE 1 only): gradients go to the object's fixed-point accumulator,
// the weight gradients flushed after every tile.
// ACT (stored activations): MODE 0 also writes the tile's activations (the
// encoding, every hidden layer and the density-net outputs) to S.act; MODE 1
// reads them back instead of gathering and recomputing the forward.
// ---------------------------------------------------------------------------
template <int LFP, int MODE, bool DET = false, bool ACT = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_tile_mlp(GridParams g, BatchDesc b, const BatchDyn* __restrict__ dyn, const int32_t* __restrict__ totals,
               RayBuf R, SampleBuf S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<LFP>& sm = *reinterpret_cast<TileSmem<LFP>*>(smem_raw);
  const int t = threadIdx.x;
  const int64_t total_tiles = totals[0];
  const int64_t tile_lo = total_tiles * blockIdx.x / gridDim.x;
  const int64_t tile_hi = total_tiles * (blockIdx.x + 1) / gridDim.x;
  const int cin = g.cin;

  // weight-gradient accumulators (per object, flushed on object change); the single-network model keeps its
  // hidden layers 2 and 3 in g4 and g6
  constexpr int TO1 = 2, TK1 = LFP / 8;   // dW1: 64 x LFP
  float g1[TO1][TK1], g2[1][4], g3[1][5], g4[4][4], g5[1][1], g6[4][4];
  zero2(g1); zero2(g2); zero2(g3); zero2(g4); zero2(g5); zero2(g6);
  auto flush_fix = [&](unsigned long long* gm) {
    wgrad_flush_fix<kH, LFP, TO1, TK1>(gm + g.mlp_off[0], kH, g.LF, g1, b.status);
    wgrad_flush_fix<kDOut, kH, 1, 4>(gm + g.mlp_off[1], kDOut, kH, g2, b.status);
    if (!g.single_net) {
      wgrad_flush_fix<kH, kCinPad, 1, 5>(gm + g.mlp_off[2], kH, cin, g3, b.status);
      wgrad_flush_fix<kH, kH, 4, 4>(gm + g.mlp_off[3], kH, kH, g4, b.status);
      wgrad_flush_fix<kC3Rows, kH, 1, 1>(gm + g.mlp_off[4], 3, kH, g5, b.status);
    } else {
      if (g.extra >= 1) wgrad_flush_fix<kH, kH, 4, 4>(gm + g.mlp_off[5], kH, kH, g4, b.status);
      if (g.extra >= 2) wgrad_flush_fix<kH, kH, 4, 4>(gm + g.mlp_off[6], kH, kH, g6, b.status);
    }
  };
  auto flush = [&](float* gm) {
    wgrad_flush<kH, LFP, TO1, TK1>(gm + g.mlp_off[0], kH, g.LF, g1);
    wgrad_flush<kDOut, kH, 1, 4>(gm + g.mlp_off[1], kDOut, kH, g2);
    if (!g.single_net) {
      wgrad_flush<kH, kCinPad, 1, 5>(gm + g.mlp_off[2], kH, cin, g3);
      wgrad_flush<kH, kH, 4, 4>(gm + g.mlp_off[3], kH, kH, g4);
      wgrad_flush<kC3Rows, kH, 1, 1>(gm + g.mlp_off[4], 3, kH, g5);
    } else {
      if (g.extra >= 1) wgrad_flush<kH, kH, 4, 4>(gm + g.mlp_off[5], kH, kH, g4);
      if (g.extra >= 2) wgrad_flush<kH, kH, 4, 4>(gm + g.mlp_off[6], kH, kH, g6);
    }
  };

  int bi = -1;
  const ObjectDev* ob = nullptr;
  for (int64_t tile = tile_lo; tile < tile_hi; ++tile) {
    // ---- object of this tile --------------------------------------------
    int nbi = bi < 0 ? 0 : bi;
    while (nbi + 1 < b.n && tile >= dyn[nbi].tile_base + dyn[nbi].n_tiles) ++nbi;
    if (nbi != bi) {
      if (MODE == 1 && !DET && bi >= 0) flush(ob->grad);
      bi = nbi;
      ob = &b.objs[b.slot[bi]];
      __syncthreads();
      const float* P = ob->params;
      for (int i = t; i < kH * LFP; i += kThreads) {
        int o = i / LFP, k = i % LFP;
        float v = k < g.LF ? P[g.mlp_off[0] + o * g.LF + k] : 0.0f;
        sm.w1[o * LFP + k] = v;
        sm.w1t[k * kH + o] = v;
      }
      for (int i = t; i < kDOut * kH; i += kThreads) {
        int o = i / kH, k = i % kH;
        float v = P[g.mlp_off[1] + i];
        sm.w2[i] = v;
        sm.w2t[k * kDOut + o] = v;
      }
      for (int i = t; i < kH * kCinPad; i += kThreads) {
        int o = i / kCinPad, k = i % kCinPad;
        float v = k < cin ? P[g.mlp_off[2] + o * cin + k] : 0.0f;
        sm.w3[i] = v;
        sm.w3t[k * kH + o] = v;
      }
      // the colour net's 64 x 64 layer, or the single-network model's hidden layer 2
      const int64_t off4 = g.extra >= 1 ? g.mlp_off[5] : g.mlp_off[3];
      for (int i = t; i < kH * kH; i += kThreads) {
        int o = i / kH, k = i % kH;
        float v = P[off4 + i];
        sm.w4[i] = v;
        sm.w4t[k * kH + o] = v;
      }
      for (int i = t; i < kC3Rows * kH; i += kThreads) sm.w5[i] = i < 3 * kH ? P[g.mlp_off[4] + i] : 0.0f;
      if (g.extra >= 2)
        for (int i = t; i < kH * kH; i += kThreads) sm.w6[(i / kH) * kW6S + i % kH] = P[g.mlp_off[6] + i];
      __syncthreads();
    }
    const int64_t s0 = (int64_t)tile * kTile;

    // ---- per-sample inputs ----------------------------------------------
    if (t < kTile) {
      uint32_t r = S.ray[s0 + t];
      if (r != kNoRay && !ROMAP_IN_BOUNDS(r < (uint32_t)b.n_rays, g.status)) r = kNoRay;
      sm.ray[t] = r;
      float x = 0.f, y = 0.f, z = 0.f;
      if (r != kNoRay) {
        x = S.x[3 * (s0 + t)]; y = S.x[3 * (s0 + t) + 1]; z = S.x[3 * (s0 + t) + 2];
      }
      sm.px[0][t] = x; sm.px[1][t] = y; sm.px[2][t] = z;
      // colour-net direction inputs (rows 16..18) and zero pad row 19
      float dx = 0.f, dy = 0.f, dz = 0.f;
      if (r != kNoRay && g.dir_dims == 3) { dx = R.d[3 * r]; dy = R.d[3 * r + 1]; dz = R.d[3 * r + 2]; }
      sm.OC[16 * kAS + t] = dx; sm.OC[17 * kAS + t] = dy; sm.OC[18 * kAS + t] = dz; sm.OC[19 * kAS + t] = 0.f;
    }
    __syncthreads();

    float* HL = sm.H1;  // the hidden layer that feeds the density net's output layer
    if (g.extra >= 1) HL = g.extra >= 2 ? sm.H3 : sm.H2;
    float* const act = ACT ? S.act + (size_t)tile * act_rows(LFP) * kTile : nullptr;
    if (MODE == 1 && ACT) {  // stored activations of this tile instead of the gather and the forward GEMMs
      act_copy<LFP, false>(sm, act);
      __syncthreads();
    } else {
    // ---- hash encoding (gather): thread -> (sample, half of the levels) --
    {
      const int s = t & (kTile - 1), h = t >> 7;
      const bool valid = sm.ray[s] != kNoRay;
      const float p[3] = {sm.px[0][s], sm.px[1][s], sm.px[2][s]};
      const int l0 = h * (g.L / 2), l1 = (h + 1) * (g.L / 2) + (h == 1 ? (g.L & 1) : 0);
      for (int l = l0; l < l1; ++l) {
        float e0 = 0.f, e1 = 0.f;
        if (valid) {
          Corners c;
          level_corners(g, l, p, ob->half, ob->inv_ext, c);
          const float2* tab = reinterpret_cast<const float2*>(ob->params) + g.off[l];
          float2 v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = __ldg(tab + c.idx[k]);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            e0 = fmaf(c.w[k], v[k].x, e0);
            e1 = fmaf(c.w[k], v[k].y, e1);
          }
        }
        sm.E[(2 * l) * kAS + s] = e0;
        sm.E[(2 * l + 1) * kAS + s] = e1;
      }
      for (int r = 2 * g.L + h; r < LFP; r += 2) sm.E[r * kAS + s] = 0.f;  // padded features
    }
    __syncthreads();

    // ---- forward ---------------------------------------------------------
    {  // H1 = relu(E W1^T)
      float acc[8][4];
      gemm_tile<4>(sm.E, LFP, sm.w1t, kH, acc);
      store_tile<4>(sm.H1, acc, [](float v, int, int) { return fmaxf(v, 0.0f); });
    }
    __syncthreads();
    if (g.extra >= 1) {  // single-network hidden layer 2: H2 = relu(H1 M1^T)
      float acc[8][4];
      gemm_tile<4>(sm.H1, kH, sm.w4t, kH, acc);
      store_tile<4>(sm.H2, acc, [](float v, int, int) { return fmaxf(v, 0.0f); });
      __syncthreads();
      if (g.extra >= 2) {  // hidden layer 3: H3 = relu(H2 M2^T)
        gemm_tile_bt<4>(sm.H2, kH, sm.w6, kW6S, acc);
        store_tile<4>(sm.H3, acc, [](float v, int, int) { return fmaxf(v, 0.0f); });
        __syncthreads();
      }
    }
    {  // OC[0..15] = HL W2^T
      float acc[8][1];
      gemm_tile<1>(HL, kH, sm.w2t, kDOut, acc);
      store_tile<1>(sm.OC, acc, [](float v, int, int) { return v; });
    }
    __syncthreads();
    if (!g.single_net) {
      {  // H2 = relu(CIN W3^T), CIN = OC rows 1..cin
        float acc[8][4];
        gemm_tile<4>(sm.OC + kAS, cin, sm.w3t, kH, acc);
        store_tile<4>(sm.H2, acc, [](float v, int, int) { return fmaxf(v, 0.0f); });
      }
      __syncthreads();
      {  // H3 = relu(H2 W4^T)
        float acc[8][4];
        gemm_tile<4>(sm.H2, kH, sm.w4t, kH, acc);
        store_tile<4>(sm.H3, acc, [](float v, int, int) { return fmaxf(v, 0.0f); });
      }
      __syncthreads();
    }
    }  // gather and forward
    if (MODE == 0 && ACT) act_copy<LFP, true>(sm, act);  // (reads rows the logits below do not write)
    if (t < kTile) {  // logits, sigmoid, density
      float l0 = 0.f, l1 = 0.f, l2 = 0.f;
      if (g.single_net) {  // the colour logits are density-net outputs 1..3
        l0 = sm.OC[kAS + t];
        l1 = sm.OC[2 * kAS + t];
        l2 = sm.OC[3 * kAS + t];
      } else {
#pragma unroll 8
        for (int k = 0; k < kH; ++k) {
          float h = sm.H3[k * kAS + t];
          l0 = fmaf(sm.w5[k], h, l0);
          l1 = fmaf(sm.w5[kH + k], h, l1);
          l2 = fmaf(sm.w5[2 * kH + k], h, l2);
        }
      }
      float c0 = 1.0f / (1.0f + __expf(-l0));
      float c1 = 1.0f / (1.0f + __expf(-l1));
      float c2 = 1.0f / (1.0f + __expf(-l2));
      float o0 = sm.OC[t];
      float sg = expf(fminf(fmaxf(o0, -15.0f), 15.0f));
      sm.sig[t] = sg;
      sm.rgb[0][t] = c0; sm.rgb[1][t] = c1; sm.rgb[2][t] = c2;
      if (MODE == 0 && sm.ray[t] != kNoRay) {
        S.sigma[s0 + t] = sg;
        S.rgb[3 * (s0 + t)] = c0;
        S.rgb[3 * (s0 + t) + 1] = c1;
        S.rgb[3 * (s0 + t) + 2] = c2;
      }
    }
    if (MODE == 0) {
      __syncthreads();
      continue;
    }

    // ---- backward ----------------------------------------------------------
    __syncthreads();
    if (g.single_net) {  // dOUT = [dsigma * sigma, dlogit 0..2, 0 ...]
      if (t < kTile) {
        const bool valid = sm.ray[t] != kNoRay;
        float ds = valid ? S.dsigma[s0 + t] : 0.f;
        float o0 = sm.OC[t];
        sm.OC[t] = (o0 >= -15.0f && o0 <= 15.0f) ? ds * sm.sig[t] : 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          float c = sm.rgb[j][t];
          float dc = valid ? S.drgb[3 * (s0 + t) + j] : 0.f;
          sm.OC[(1 + j) * kAS + t] = dc * c * (1.0f - c);
        }
        for (int j = 4; j < kDOut; ++j) sm.OC[j * kAS + t] = 0.0f;
      }
    } else {
      if (t < kTile) {
        const bool valid = sm.ray[t] != kNoRay;
        float ds = valid ? S.dsigma[s0 + t] : 0.f;
        float o0 = sm.OC[t];
        float dpre = (o0 >= -15.0f && o0 <= 15.0f) ? ds * sm.sig[t] : 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          float c = sm.rgb[j][t];
          float dc = valid ? S.drgb[3 * (s0 + t) + j] : 0.f;
          sm.DL[j * kAS + t] = dc * c * (1.0f - c);
        }
        sm.DL[3 * kAS + t] = 0.0f;
        sm.sig[t] = dpre;  // reuse: dL/d(out_0)
      }
      __syncthreads();
      wgrad_tile<kC3Rows, kH, 1, 1>(sm.DL, sm.H3, g5);  // dW5 += DL^T H3
      __syncthreads();
      {  // dH3 = (DL W5) * [H3 > 0], in place
        float acc[8][4];
        gemm_tile<4>(sm.DL, kC3Rows, sm.w5, kH, acc);
        const float* H3 = sm.H3;
        store_tile<4>(sm.H3, acc, [H3](float v, int n, int m) { return H3[n * kAS + m] > 0.f ? v : 0.f; });
      }
      __syncthreads();
      wgrad_tile<kH, kH, 4, 4>(sm.H3, sm.H2, g4);  // dW4 += dH3^T H2
      __syncthreads();
      {  // dH2 = (dH3 W4) * [H2 > 0], in place
        float acc[8][4];
        gemm_tile<4>(sm.H3, kH, sm.w4, kH, acc);
        const float* H2 = sm.H2;
        store_tile<4>(sm.H2, acc, [H2](float v, int n, int m) { return H2[n * kAS + m] > 0.f ? v : 0.f; });
      }
      __syncthreads();
      wgrad_tile<kH, kCinPad, 1, 5>(sm.H2, sm.OC + kAS, g3);  // dW3 += dH2^T CIN
      __syncthreads();
      {  // dOUT[1..15] = (dH2 W3)[0..14]; dOUT[0] = dsigma * sigma (clamp mask)
        float acc[8][1];
        gemm_tile<1>(sm.H2, kH, sm.w3, kCinPad, acc);
        store_tile<1>(sm.OC + kAS, acc, [](float v, int, int) { return v; });  // writes rows 1..16
      }
      __syncthreads();
      if (t < kTile) sm.OC[t] = sm.sig[t];
    }  // colour net
    __syncthreads();
    wgrad_tile<kDOut, kH, 1, 4>(sm.OC, HL, g2);  // dW2 += dOUT^T HL
    __syncthreads();
    {  // dHL = (dOUT W2) * [HL > 0], in place
      float acc[8][4];
      gemm_tile<4>(sm.OC, kDOut, sm.w2, kH, acc);
      const float* Hf = HL;
      store_tile<4>(HL, acc, [Hf](float v, int n, int m) { return Hf[n * kAS + m] > 0.f ? v : 0.f; });
    }
    __syncthreads();
    if (g.extra >= 2) {  // hidden layer 3: dM2 += dH3^T H2; dH2 = (dH3 M2) * [H2 > 0], in place
      wgrad_tile<kH, kH, 4, 4>(sm.H3, sm.H2, g6);
      __syncthreads();
      float acc[8][4];
      gemm_tile<4>(sm.H3, kH, sm.w6, kW6S, acc);
      const float* H2 = sm.H2;
      store_tile<4>(sm.H2, acc, [H2](float v, int n, int m) { return H2[n * kAS + m] > 0.f ? v : 0.f; });
      __syncthreads();
    }
    if (g.extra >= 1) {  // hidden layer 2: dM1 += dH2^T H1; dH1 = (dH2 M1) * [H1 > 0], in place
      wgrad_tile<kH, kH, 4, 4>(sm.H2, sm.H1, g4);
      __syncthreads();
      float acc[8][4];
      gemm_tile<4>(sm.H2, kH, sm.w4, kH, acc);
      const float* H1 = sm.H1;
      store_tile<4>(sm.H1, acc, [H1](float v, int n, int m) { return H1[n * kAS + m] > 0.f ? v : 0.f; });
      __syncthreads();
    }
    wgrad_tile<kH, LFP, TO1, TK1>(sm.H1, sm.E, g1);  // dW1 += dH1^T E
    __syncthreads();
    {  // dE = dH1 W1, into E
      float acc[8][LFP / 16];
      gemm_tile<LFP / 16>(sm.H1, kH, sm.w1, LFP, acc);
      store_tile<LFP / 16>(sm.E, acc, [](float v, int, int) { return v; });
    }
    __syncthreads();
    {  // scatter dE into the hash-table gradient
      const int s = t & (kTile - 1), h = t >> 7;
      if (sm.ray[s] != kNoRay) {
        const float p[3] = {sm.px[0][s], sm.px[1][s], sm.px[2][s]};
        const int l0 = h * (g.L / 2), l1 = (h + 1) * (g.L / 2) + (h == 1 ? (g.L & 1) : 0);
        for (int l = l0; l < l1; ++l) {
          float d0 = sm.E[(2 * l) * kAS + s], d1 = sm.E[(2 * l + 1) * kAS + s];
          if (d0 == 0.f && d1 == 0.f) continue;
          Corners c;
          level_corners(g, l, p, ob->half, ob->inv_ext, c);
          if (DET) {
            scatter_corners_fix(ob->gfix + 2 * (size_t)g.off[l], c.idx, c.w, d0, d1, b.status);
          } else {
            float2* gt = reinterpret_cast<float2*>(ob->grad) + g.off[l];
            scatter_corners(gt, c.idx, c.w, d0, d1);
          }
        }
      }
    }
    if (DET) flush_fix(ob->gfix);  // this tile's weight gradients
    __syncthreads();
  }
  if (MODE == 1 && !DET && bi >= 0) flush(ob->grad);
}

template <int LFP, int MODE, bool DET, bool ACT>
static void launch_tile_t(const GridParams& g, const BatchDesc& b, const BatchDyn* dyn, const int32_t* totals,
                          RayBuf r, SampleBuf s, int n_ctas, cudaStream_t stream) {
  static std::atomic<uint64_t> attr_done{0};
  int bytes = (int)sizeof(TileSmem<LFP>);
  set_smem_attr(k_tile_mlp<LFP, MODE, DET, ACT>, bytes, attr_done);
  k_tile_mlp<LFP, MODE, DET, ACT><<<n_ctas, kThreads, bytes, stream>>>(g, b, dyn, totals, r, s);
}

template <int LFP>
static void launch_tile_l(int mode, const GridParams& g, const BatchDesc& b, const BatchDyn* dyn,
                          const int32_t* totals, RayBuf r, SampleBuf s, int n_ctas, cudaStream_t stream) {
  const bool act = s.act != nullptr;  // stored activations (the deterministic mode keeps recomputing)
  if (mode == 0) {
    if (act) launch_tile_t<LFP, 0, false, true>(g, b, dyn, totals, r, s, n_ctas, stream);
    else launch_tile_t<LFP, 0, false, false>(g, b, dyn, totals, r, s, n_ctas, stream);
  } else if (g.det) {
    launch_tile_t<LFP, 1, true, false>(g, b, dyn, totals, r, s, n_ctas, stream);
  } else if (act) {
    launch_tile_t<LFP, 1, false, true>(g, b, dyn, totals, r, s, n_ctas, stream);
  } else {
    launch_tile_t<LFP, 1, false, false>(g, b, dyn, totals, r, s, n_ctas, stream);
  }
}

void launch_tile_mlp(int mode, const GridParams& g, const BatchDesc& b, const BatchDyn* dyn, const int32_t* totals,
                     RayBuf r, SampleBuf s, int n_ctas, cudaStream_t stream) {
  if (g.LF <= 16) launch_tile_l<16>(mode, g, b, dyn, totals, r, s, n_ctas, stream);
  else launch_tile_l<32>(mode, g, b, dyn, totals, r, s, n_ctas, stream);
}

int act_rows_for(int LF) { return act_rows(LF <= 16 ? 16 : 32); }

}  // namespace romap
