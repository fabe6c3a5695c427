// Mixed-precision training step: the instances of the fused tile kernel with BF16 and FP8 operands (the kernel
// itself is in tc_tile_kernel.cuh), the placement of rays in the tile plan, the FP16 table refresh and the
// failure-detection self-test kernel.
#include "tc_tile_kernel.cuh"

namespace romap {
namespace {
using namespace tc;

// Places every ray of the batch in the tile plan.  A ray with c > 0 live samples has rank j among its entry's rays of
// count c (offset of its ray block for count c + rank within the block, in ray order); the segments of count c
// (in rank order) give its pattern, tile and copy; the ray goes to its position in plan_perm with its first slot in
// plan_rstart, and its slots' {ray, sample index} go to plan_slot.  Rays without live samples add their loss here
// (C_hat = background, D_hat = 0) and write their outputs.
__global__ void __launch_bounds__(256) k_plan_rays(GridParams g, BatchDesc b, RayBuf R, BatchDyn* dyn) {
  __shared__ uint32_t s_wcnt[8][kPlanCounts];  // rays of each count per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bi = b.block_obj[blockIdx.x];
  const int rl = (blockIdx.x - b.block_base[bi]) * 256 + threadIdx.x;
  const int n_obj = b.ray_base[bi + 1] - b.ray_base[bi];
  const bool valid = rl < n_obj;
  const int64_t r = b.ray_base[bi] + rl;
  const int c = valid ? (int)R.count[r] : -1;
  for (int k = threadIdx.x; k < 8 * kPlanCounts; k += blockDim.x) (&s_wcnt[0][0])[k] = 0u;
  __syncthreads();
  const uint32_t same = __match_any_sync(0xffffffffu, c);
  const uint32_t rank = __popc(same & ((1u << lane) - 1u));
  if (c > 0 && rank == 0) s_wcnt[warp][c] = __popc(same);
  __syncthreads();
  if (c > 0) {
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_wcnt[w][c];
    const int j = (int)(b.plan_bcnt[blockIdx.x * kPlanCounts + c] + before + rank);
    const int nseg = b.plan_nseg[(size_t)bi * kPlanCounts + c];
    const int4* sg = b.plan_seg + ((size_t)bi * kPlanCounts + c) * kPlanSegsPerCount * 2;
    int k = 0;
    while (k + 1 < nseg && j >= sg[2 * k].x + sg[2 * k].z * sg[2 * k].w) ++k;
    const int4 s0 = sg[2 * k], s1 = sg[2 * k + 1];
    const int q = j - s0.x, tt = q / s0.z, cp = q - tt * s0.z;
    const int64_t tile = (int64_t)b.plan_ent[bi] + s0.y + tt;
    const int pos = b.ray_base[bi] + s1.w + tt * s1.z + s1.y + cp;
    const int start = s1.x + cp * c;
    if (!ROMAP_IN_BOUNDS(pos >= b.ray_base[bi] && pos < b.ray_base[bi + 1] && start >= 0 && start + c <= kTile &&
                             tile >= 0 && tile < b.plan_cap_tiles,
                         g.status))
      return;
    b.plan_perm[pos] = (int32_t)r;
    b.plan_rstart[pos] = start;
    int2* slot = b.plan_slot + tile * kTile + start;
    for (int i = 0; i < c; ++i) slot[i] = make_int2((int)r, i);
  } else if (c == 0) {
    const float bg0 = R.bg[3 * r], bg1 = R.bg[3 * r + 1], bg2 = R.bg[3 * r + 2];
    float* o = R.out + 6 * r;
    o[0] = bg0; o[1] = bg1; o[2] = bg2; o[3] = 0.f; o[4] = 0.f; o[5] = 0.f;
    const RayLoss q = ray_loss(g, ray_target(R, r), bg0, bg1, bg2, 0.f, 0.f, 1.0f / (float)n_obj);
    add_ray_loss(dyn, bi, q, nullptr);
  }
}

}  // namespace


void launch_tile_tc(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, RayBuf r, int32_t* status,
                    int max_tiles, int n_ctas, int interleave, cudaStream_t stream) {
  if (g.f16) {  // FP16 operands: instances in kernels_tc16.cu (never combined with FP8)
    launch_tile_tc_f16(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else if (g.fp8) {  // (the single-network model is never combined with FP8)
    if (g.LF <= 16) launch_tc_t<16, true, false, false, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, true, false, false, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else if (g.single_net) {
    if (g.LF <= 16) launch_tc_t<16, false, true, false, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, true, false, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  } else {
    if (g.LF <= 16) launch_tc_t<16, false, false, false, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
    else launch_tc_t<32, false, false, false, 2>(g, b, dyn, r, status, max_tiles, n_ctas, interleave, stream);
  }
}

void launch_plan_rays(const GridParams& g, const BatchDesc& b, RayBuf r, BatchDyn* dyn, cudaStream_t stream) {
  if (b.n_blocks <= 0) return;
  k_plan_rays<<<b.n_blocks, 256, 0, stream>>>(g, b, r, dyn);
}

// Failure-detection self-test: a bounded wait on an mbarrier that nothing signals must give up, record the
// time-out in the status word (bit 1), free the tensor memory it holds and return.
__global__ void k_selftest_wait(int32_t* status, int limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tslot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::tc_before();
  __syncthreads();
  tc::tc_after();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit)) atomicOr(status, 2);
  tc::tc_before();
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(32));
}

void launch_selftest_wait(int32_t* status, int limit, cudaStream_t stream) {
  k_selftest_wait<<<1, 64, 0, stream>>>(status, limit);
}

// FP16 copy of the hash table (n_hash is even)
__global__ void k_to_half(const float* __restrict__ src, __half2* __restrict__ dst, int64_t n2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __floats2half2_rn(src[2 * i], src[2 * i + 1]);
}

void launch_to_half(const float* params, uint16_t* table_h, int64_t n_hash, cudaStream_t stream) {
  int64_t n2 = n_hash / 2;
  int blocks = (int)((n2 + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) return;
  k_to_half<<<blocks, 256, 0, stream>>>(params, reinterpret_cast<__half2*>(table_h), n2);
}

}  // namespace romap
