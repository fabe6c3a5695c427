// Mixed-precision training step, alternative tile shapes of the fused tile kernel of tc_tile_kernel.cuh (BF16 or
// FP16 operands, the two-network model), in a translation unit of their own so that they compile in parallel with
// the lockstep tile-pair instances: one tile per CTA with two CTAs per SM (TPC = 1), and tile pairs whose two
// warpgroups run decoupled (DEC).
#include "tc_tile_kernel.cuh"

namespace romap {

void launch_tile_tc1(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                     int max_tiles, int n_ctas, int interleave, cudaStream_t stream) {
  if (g.f16) {
    if (g.LF <= 16) launch_tc_t<16, false, false, true, 1>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, false, true, 1>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else {
    if (g.LF <= 16) launch_tc_t<16, false, false, false, 1>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, false, false, 1>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  }
}

void launch_tile_tcd(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                     int max_tiles, int n_ctas, int interleave, cudaStream_t stream) {
  if (g.f16) {
    if (g.LF <= 16)
      launch_tc_t<16, false, false, true, 2, true>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, false, true, 2, true>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else {
    if (g.LF <= 16)
      launch_tc_t<16, false, false, false, 2, true>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, false, false, 2, true>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  }
}

}  // namespace romap
