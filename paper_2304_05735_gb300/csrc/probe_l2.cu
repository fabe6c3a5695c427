// Measured roof of the fused training kernel's memory path.
//
// The fused kernel's hash gather (8 corners x L levels of 4-byte FP16 feature pairs per sample) and hash-gradient
// scatter (as many 8-byte FP32 pair reductions) hit tables that stay in the 129 MB L2 while CTAs work on the same
// few objects; DRAM carries a small fraction of those bytes.  What bounds them is the rate at which the SMs can
// issue scattered requests through L1 to L2.  These kernels measure that rate on the running GPU: every lane of every
// warp draws its own pseudo-random address (xorshift), so every lane is a separate request, into buffers small
// enough to stay L2-resident (32 MiB for loads, 64 MiB for reductions, after a warm-up pass).
//   gather: 4-byte loads;  reduce: red.global.add.v2.f32;  mix: one of each per step (the fused kernel's 1:1 mix).
// Each rate is the best of three timed launches (CUDA events on the caller's stream).
#include <cuda_runtime.h>

#include <cstdint>

#include "romap.h"
#include "romap_internal.cuh"

namespace romap {
namespace {

constexpr int kProbeChains = 8;  // independent requests in flight per thread

__device__ __forceinline__ uint32_t xorshift(uint32_t x) {
  x ^= x << 13;
  x ^= x >> 17;
  x ^= x << 5;
  return x;
}

__device__ __forceinline__ void probe_red2(float2* addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// mode 0: loads only, 1: reductions only, 2: one load and one reduction per chain step
template <int MODE>
__global__ void __launch_bounds__(256) k_probe(const uint32_t* __restrict__ lbuf, uint32_t lmask, float2* rbuf,
                                               uint32_t rmask, int iters, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s[k] = (tid * kProbeChains + k) * 2654435761u + 0x9E3779B9u;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) {
      s[k] = xorshift(s[k]);
      if (MODE != 1) acc += lbuf[s[k] & lmask];
      if (MODE != 0) probe_red2(rbuf + ((s[k] >> 3) & rmask), 1e-30f, 1e-30f);
    }
  }
  if (acc == 0x12345678u) sink[0] = acc;  // keeps the loads
}

}  // namespace
}  // namespace romap

using namespace romap;

extern "C" ROMAP_API romap_status romap_measure_request_rates(void* cuda_stream, double* out) {
  if (!out) return ROMAP_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return ROMAP_ERR_CUDA;
  const size_t lwords = (size_t)8 << 20;  // 32 MiB of 4-byte words
  const size_t rpairs = (size_t)8 << 20;  // 64 MiB of float pairs
  uint32_t* lbuf = nullptr;
  float2* rbuf = nullptr;
  uint32_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  romap_status st = ROMAP_OK;
  if (cudaMalloc(&lbuf, lwords * 4) != cudaSuccess || cudaMalloc(&rbuf, rpairs * 8) != cudaSuccess ||
      cudaMalloc(&sink, 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = ROMAP_ERR_OOM;
  }
  if (st == ROMAP_OK && (cudaMemsetAsync(lbuf, 1, lwords * 4, stream) != cudaSuccess ||
                         cudaMemsetAsync(rbuf, 0, rpairs * 8, stream) != cudaSuccess))
    st = ROMAP_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 256;
  const double requests = (double)blocks * threads * iters * kProbeChains;
  for (int mode = 0; mode < 3 && st == ROMAP_OK; ++mode) {
    float best = 0.f;
    for (int rep = 0; rep < 4; ++rep) {  // the first launch warms L2 and is not counted
      cudaEventRecord(e0, stream);
      if (mode == 0)
        k_probe<0><<<blocks, threads, 0, stream>>>(lbuf, (uint32_t)(lwords - 1), rbuf, (uint32_t)(rpairs - 1),
                                                     iters, sink);
      else if (mode == 1)
        k_probe<1><<<blocks, threads, 0, stream>>>(lbuf, (uint32_t)(lwords - 1), rbuf, (uint32_t)(rpairs - 1),
                                                     iters, sink);
      else
        k_probe<2><<<blocks, threads, 0, stream>>>(lbuf, (uint32_t)(lwords - 1), rbuf, (uint32_t)(rpairs - 1),
                                                     iters, sink);
      cudaEventRecord(e1, stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = ROMAP_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    out[mode] = best > 0.f ? requests / (best * 1e-3) : 0.0;  // per second: loads, reductions, load+reduce pairs
  }
  if (st == ROMAP_OK && cudaGetLastError() != cudaSuccess) st = ROMAP_ERR_CUDA;
  cudaStreamSynchronize(stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(lbuf);
  cudaFree(rbuf);
  cudaFree(sink);
  return st;
}
