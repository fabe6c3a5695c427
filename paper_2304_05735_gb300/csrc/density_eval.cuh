// The density net of one object evaluated at arbitrary object-frame points in FP32 (FP32 master parameters): the
// hash encoding gathered from the FP32 table, the first layer with ReLU (then the single-network model's further
// 64x64 hidden layers), and output 0 of the output layer, sigma = exp(clamp(o_0, -15, 15)).  Used by the occupancy
// update and the mesh extraction.
#pragma once
#include "device_common.cuh"

namespace romap {

// XL: the single-network model has hidden layers after the first (g.extra > 0)
template <int LFP, bool XL>
struct DensityWeights {
  float w1[kH * LFP];  // first layer [64][LFP], columns past LF zero
  float w2[kH];        // row 0 of the output layer (log-density)
  float wx[XL ? 2 : 1][XL ? kH * kH : 1];  // single-network hidden layers 2 and 3, [out][in]
};

// Whole block: copies the weights of params P into shared memory (the caller synchronises afterwards).
template <int LFP, bool XL>
__device__ __forceinline__ void load_density_weights(DensityWeights<LFP, XL>& s, const GridParams& g, const float* P) {
  for (int i = threadIdx.x; i < kH * LFP; i += blockDim.x) {
    const int j = i / LFP, k = i % LFP;
    s.w1[i] = k < g.LF ? P[g.mlp_off[0] + j * g.LF + k] : 0.f;
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) s.w2[i] = P[g.mlp_off[1] + i];
  if constexpr (XL)
    for (int x = 0; x < g.extra; ++x)
      for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) s.wx[x][i] = P[g.mlp_off[5 + x] + i];
}

template <int LFP, bool XL>
__device__ __forceinline__ float density_at(const DensityWeights<LFP, XL>& s, const GridParams& g, const ObjectDev& ob,
                                            const float x[3]) {
  float e[LFP];
#pragma unroll
  for (int k = 0; k < LFP; ++k) e[k] = 0.f;
  const float2* tab = reinterpret_cast<const float2*>(ob.params);
#pragma unroll
  for (int l = 0; l < LFP / 2; ++l) {
    if (l >= g.L) break;
    Corners c;
    level_corners(g, l, x, ob.half, ob.inv_ext, c);
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 v = tab[g.off[l] + c.idx[k]];
      a0 = fmaf(c.w[k], v.x, a0);
      a1 = fmaf(c.w[k], v.y, a1);
    }
    e[2 * l] = a0;
    e[2 * l + 1] = a1;
  }
  float o0 = 0.f;
  if constexpr (!XL) {
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
      float h = 0.f;
#pragma unroll
      for (int k = 0; k < LFP; ++k) h = fmaf(s.w1[j * LFP + k], e[k], h);
      o0 = fmaf(s.w2[j], fmaxf(h, 0.f), o0);
    }
  } else {
    float h[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      float a = 0.f;
#pragma unroll
      for (int k = 0; k < LFP; ++k) a = fmaf(s.w1[j * LFP + k], e[k], a);
      h[j] = fmaxf(a, 0.f);
    }
    for (int x = 0; x < g.extra; ++x) {
      float hn[kH];
#pragma unroll
      for (int i = 0; i < kH; ++i) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < kH; ++j) a = fmaf(s.wx[x][i * kH + j], h[j], a);
        hn[i] = fmaxf(a, 0.f);
      }
#pragma unroll
      for (int i = 0; i < kH; ++i) h[i] = hn[i];
    }
#pragma unroll
    for (int j = 0; j < kH; ++j) o0 = fmaf(s.w2[j], h[j], o0);
  }
  return expf(fminf(fmaxf(o0, -15.f), 15.f));
}

}  // namespace romap
