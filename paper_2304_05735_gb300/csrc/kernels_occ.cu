// Occupancy update from the learned density (empty-space skipping; the paper samples the whole box): the object's
// density net, evaluated with its FP32 master parameters at the centre of each of the 64^3 cells of its box, feeds a
// per-cell moving maximum d = max(decay d, sigma), and the cells with d > threshold form the new bitgrid that culls
// samples (a culled sample has sigma := 0 and keeps its delta).  One thread per cell; cell index x + 64 y + 4096 z,
// so each warp covers 32 consecutive x and its ballot is one 32-bit half of a bitgrid word.
#include "device_common.cuh"

namespace romap {
namespace {

constexpr int kCells = 64 * 64 * 64;

template <int LFP>
__global__ void __launch_bounds__(256) k_occ_update(GridParams g, const ObjectDev* objs, int slot, float decay,
                                                   float threshold, int reset, float* dens, uint32_t* bits) {
  __shared__ float w1[kH * LFP];  // first layer [64][LF]
  __shared__ float w2[kH];        // row 0 of the second layer (log-density)
  const ObjectDev& ob = objs[slot];
  const float* P = ob.params;
  for (int i = threadIdx.x; i < kH * LFP; i += blockDim.x) {  // columns past LF are zero
    const int j = i / LFP, k = i % LFP;
    w1[i] = k < g.LF ? P[g.mlp_off[0] + j * g.LF + k] : 0.f;
  }
  if (threadIdx.x < kH) w2[threadIdx.x] = P[g.mlp_off[1] + threadIdx.x];
  __syncthreads();
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;  // grid covers exactly kCells
  const int idx[3] = {cell & 63, (cell >> 6) & 63, cell >> 12};
  float x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // cell centre, FP32 in a fixed order: -a + (i + 0.5) ((a - (-a)) / 64)
    const float lo = -ob.half[a];
    const float w = __fdiv_rn(__fsub_rn(ob.half[a], lo), 64.0f);
    x[a] = __fadd_rn(lo, __fmul_rn(__fadd_rn((float)idx[a], 0.5f), w));
  }
  float e[LFP];
#pragma unroll
  for (int k = 0; k < LFP; ++k) e[k] = 0.f;
  const float2* tab = reinterpret_cast<const float2*>(P);
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
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float h = 0.f;
#pragma unroll
    for (int k = 0; k < LFP; ++k) h = fmaf(w1[j * LFP + k], e[k], h);
    o0 = fmaf(w2[j], fmaxf(h, 0.f), o0);
  }
  const float sigma = expf(fminf(fmaxf(o0, -15.f), 15.f));
  const float d = reset ? sigma : fmaxf(decay * dens[cell], sigma);
  dens[cell] = d;
  const unsigned m = __ballot_sync(0xffffffffu, d > threshold);
  if ((threadIdx.x & 31) == 0) bits[cell >> 5] = m;
}

}  // namespace

void launch_occ_update(const GridParams& g, const ObjectDev* objs, int slot, float decay, float threshold, int reset,
                       float* dens, uint64_t* bits, cudaStream_t stream) {
  uint32_t* b32 = reinterpret_cast<uint32_t*>(bits);  // word w = halves 2w (cells 64w..64w+31) and 2w+1
  if (g.LF <= 16) k_occ_update<16><<<kCells / 256, 256, 0, stream>>>(g, objs, slot, decay, threshold, reset, dens, b32);
  else k_occ_update<32><<<kCells / 256, 256, 0, stream>>>(g, objs, slot, decay, threshold, reset, dens, b32);
}

}  // namespace romap
