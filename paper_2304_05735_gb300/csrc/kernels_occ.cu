// Occupancy update from the learned density (empty-space skipping; the paper samples the whole box): the object's
// density net, evaluated with its FP32 master parameters at the centre of each of the 64^3 cells of its box, feeds a
// per-cell moving maximum d = max(decay d, sigma), and the cells with d > threshold form the new bitgrid that culls
// samples (a culled sample has sigma := 0 and keeps its delta).  One thread per cell; cell index x + 64 y + 4096 z,
// so each warp covers 32 consecutive x and its ballot is one 32-bit half of a bitgrid word.
#include "density_eval.cuh"

namespace romap {
namespace {

constexpr int kCells = 64 * 64 * 64;

template <int LFP, bool XL>
__global__ void __launch_bounds__(256) k_occ_update(GridParams g, const ObjectDev* objs, int slot, float decay,
                                                   float threshold, int reset, float* dens, uint32_t* bits) {
  __shared__ DensityWeights<LFP, XL> sw;
  const ObjectDev& ob = objs[slot];
  load_density_weights<LFP, XL>(sw, g, ob.params);
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
  const float sigma = density_at<LFP, XL>(sw, g, ob, x);
  const float d = reset ? sigma : fmaxf(decay * dens[cell], sigma);
  dens[cell] = d;
  const unsigned m = __ballot_sync(0xffffffffu, d > threshold);
  if ((threadIdx.x & 31) == 0) bits[cell >> 5] = m;
}

}  // namespace

void launch_occ_update(const GridParams& g, const ObjectDev* objs, int slot, float decay, float threshold, int reset,
                       float* dens, uint64_t* bits, cudaStream_t stream) {
  uint32_t* b32 = reinterpret_cast<uint32_t*>(bits);  // word w = halves 2w (cells 64w..64w+31) and 2w+1
  auto k = g.LF <= 16 ? (g.extra ? k_occ_update<16, true> : k_occ_update<16, false>)
                      : (g.extra ? k_occ_update<32, true> : k_occ_update<32, false>);
  k<<<kCells / 256, 256, 0, stream>>>(g, objs, slot, decay, threshold, reset, dens, b32);
}

}  // namespace romap
