// Mixed-precision training step with one tile per CTA and two CTAs per SM: the instances of the fused tile kernel of
// tc_tile_kernel.cuh with TPC = 1 (BF16 or FP16 operands, the two-network model), in a translation unit of their own
// so that they compile in parallel with the tile-pair instances.
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

}  // namespace romap
