// Mixed-precision training step with FP16 MLP operands (ROMAP_PREC_MIXED_FP16): the instances of the fused tile
// kernel of tc_tile_kernel.cuh with FP16 A/B operands, in a translation unit of their own so that they compile in
// parallel with the BF16 and FP8 instances.
#include "tc_tile_kernel.cuh"

namespace romap {

void launch_tile_tc_f16(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                        int max_tiles, int n_ctas, int interleave, cudaStream_t stream) {
  if (g.single_net) {
    if (g.LF <= 16) launch_tc_t<16, false, true, true, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, true, true, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else {
    if (g.LF <= 16) launch_tc_t<16, false, false, true, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, false, true, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  }
}

}  // namespace romap
