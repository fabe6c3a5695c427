// Volume rendering (Sec. V-B, Eq. 6), the losses of Eq. 7-11, the
// compositing adjoint, and the fused Adam update.
//
// Compositing: one warp per ray; the samples of a ray are contiguous.  The
// transmittance T_i = exp(-sum_{j<i} sigma_j delta_j) comes from a warp
// shuffle prefix scan of sigma*delta carried across 32-sample chunks; the
// occupancy o_i = 1 - exp(-sigma_i delta_i) is formed with expm1f to avoid
// cancellation.  The adjoint walks the chunks backwards with a suffix scan:
//   dC/dsigma_i = delta_i [T_{i+1} c_i - sum_{j>i} w_j c_j - T_{N+1} bg]
//   dD/dsigma_i = delta_i [T_{i+1} t_i - sum_{j>i} w_j t_j]
//   dA/dsigma_i = delta_i T_{N+1},  dC/dc_i = w_i.
// Every ray composites over its own background colour (zero density then
// renders that colour, which is what the random-colour loss of Eq. 9 asks
// background rays to learn).
#include <cuda_fp16.h>

#include "device_common.cuh"
#include "romap_internal.cuh"

namespace romap {

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_incl_prefix(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}
__device__ inline float warp_incl_suffix(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float n = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += n;
  }
  return v;
}

// MODE 0: render outputs only.  1: training loss (Eq. 7-11) + adjoint.
// 2: adjoint of an upstream gradient of the per-ray outputs.
template <int MODE>
__global__ void __launch_bounds__(256) k_composite(GridParams g, BatchDesc b, RayBuf R, SampleBuf S, BatchDyn* dyn,
                                                   int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= b.n_rays) return;
  const uint32_t cnt = R.count[r], off = R.off[r];
  const float bg0 = R.bg[3 * r], bg1 = R.bg[3 * r + 1], bg2 = R.bg[3 * r + 2];

  // ---- forward: Eq. 6 -----------------------------------------------------
  float carry = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Dh = 0.f, ssum = 0.f;
  if (g.accuracy) {  // the log-sum of transmittance, the weights and their sums in FP64
    double carry_d = 0.0, C0d = 0.0, C1d = 0.0, C2d = 0.0, Dhd = 0.0;
    for (uint32_t base = 0; base < cnt; base += 32) {
      const uint32_t j = base + lane;
      const bool in = j < cnt;
      const float sg = in ? S.sigma[off + j] : 0.f;
      const double sd = (double)sg * (double)(in ? S.dt[off + j] : 0.f);
      double incl = sd;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
      }
      double excl = __shfl_up_sync(0xffffffffu, incl, 1);
      if (lane == 0) excl = 0.0;
      const double P = carry_d + excl;
      const double w = exp(-P) * (-expm1(-sd));
      if (in) {
        C0d += w * (double)S.rgb[3 * (off + j)];
        C1d += w * (double)S.rgb[3 * (off + j) + 1];
        C2d += w * (double)S.rgb[3 * (off + j) + 2];
        Dhd += w * (double)S.t[off + j];
        ssum += sg;
        if (MODE != 0) S.dsigma[off + j] = (float)P;
      }
      carry_d += __shfl_sync(0xffffffffu, incl, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      C0d += __shfl_xor_sync(0xffffffffu, C0d, o);
      C1d += __shfl_xor_sync(0xffffffffu, C1d, o);
      C2d += __shfl_xor_sync(0xffffffffu, C2d, o);
      Dhd += __shfl_xor_sync(0xffffffffu, Dhd, o);
    }
    ssum = warp_sum(ssum);
    const double Tend_d = exp(-carry_d);
    carry = (float)carry_d;
    const float Ch0 = (float)(Tend_d * bg0 + C0d), Ch1 = (float)(Tend_d * bg1 + C1d);
    const float Ch2 = (float)(Tend_d * bg2 + C2d);
    C0 = Ch0; C1 = Ch1; C2 = Ch2; Dh = (float)Dhd;
    if (lane == 0) {
      float* o = R.out + 6 * r;
      o[0] = Ch0; o[1] = Ch1; o[2] = Ch2; o[3] = Dh; o[4] = (float)(-expm1(-carry_d)); o[5] = ssum;
    }
  }
  for (uint32_t base = 0; base < cnt && !g.accuracy; base += 32) {
    const uint32_t j = base + lane;
    const bool in = j < cnt;
    const float sg = in ? S.sigma[off + j] : 0.f;
    const float dt = in ? S.dt[off + j] : 0.f;
    const float tt = in ? S.t[off + j] : 0.f;
    const float sd = sg * dt;
    const float incl = warp_incl_prefix(sd, lane);
    float excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.f;
    const float P = carry + excl;
    const float w = expf(-P) * (-expm1f(-sd));
    if (in) {
      C0 = fmaf(w, S.rgb[3 * (off + j)], C0);
      C1 = fmaf(w, S.rgb[3 * (off + j) + 1], C1);
      C2 = fmaf(w, S.rgb[3 * (off + j) + 2], C2);
      Dh = fmaf(w, tt, Dh);
      ssum += sg;
      if (MODE != 0) S.dsigma[off + j] = P;  // exclusive prefix, consumed by the adjoint below
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  const float Tend = expf(-carry);
  float Ch0, Ch1, Ch2;
  if (g.accuracy) {  // rendered above
    Ch0 = C0; Ch1 = C1; Ch2 = C2;
  } else {
    C0 = warp_sum(C0); C1 = warp_sum(C1); C2 = warp_sum(C2); Dh = warp_sum(Dh); ssum = warp_sum(ssum);
    const float A = -expm1f(-carry);
    Ch0 = fmaf(Tend, bg0, C0); Ch1 = fmaf(Tend, bg1, C1); Ch2 = fmaf(Tend, bg2, C2);
    if (lane == 0) {
      float* o = R.out + 6 * r;
      o[0] = Ch0; o[1] = Ch1; o[2] = Ch2; o[3] = Dh; o[4] = A; o[5] = ssum;
    }
  }
  if (MODE == 0) return;

  // ---- loss (Eq. 7-11) or upstream gradient --------------------------------
  float gC0, gC1, gC2, gD, gA = 0.f, gdir = 0.f;
  if (MODE == 1) {
    const int bi = R.obj[r];
    const float invB = 1.0f / (float)(b.ray_base[bi + 1] - b.ray_base[bi]);
    const int cls = R.cls[r];
    float loss = 0.f, l_rgb = 0.f, l_rr = 0.f, l_dep = 0.f, l_den = 0.f;
    gC0 = gC1 = gC2 = gD = 0.f;
    if (cls != kClsOccluder) {
      const float t0 = cls == kClsObject ? R.rgb[3 * r] : bg0;
      const float t1 = cls == kClsObject ? R.rgb[3 * r + 1] : bg1;
      const float t2 = cls == kClsObject ? R.rgb[3 * r + 2] : bg2;
      const float e0 = Ch0 - t0, e1 = Ch1 - t1, e2 = Ch2 - t2;
      const float sq = e0 * e0 + e1 * e1 + e2 * e2;
      loss += sq;
      if (cls == kClsObject) l_rgb = sq; else l_rr = sq;
      gC0 = 2.f * e0 * invB; gC1 = 2.f * e1 * invB; gC2 = 2.f * e2 * invB;
      const float dep = R.depth[r];
      if (isfinite(dep)) {
        const float e = Dh - dep;
        loss += g.lambda1 * fabsf(e);
        l_dep = fabsf(e);
        gD = g.lambda1 * (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) * invB;
      }
      if (cls == kClsBackground) {
        loss += g.lambda2 * ssum;
        l_den = ssum;
        gdir = g.lambda2 * invB;
      }
    }
    if (lane == 0) {
      if (g.det) {  // fixed-point sums (converted after the backward): the same bits in any order
        unsigned long long* Q = dyn[bi].loss_fix;
        red_add_fix(Q + 0, loss, status, kFixLossBits, kFixLossMaxContribution);
        red_add_fix(Q + 1, l_rgb, status, kFixLossBits, kFixLossMaxContribution);
        red_add_fix(Q + 2, l_rr, status, kFixLossBits, kFixLossMaxContribution);
        red_add_fix(Q + 3, l_dep, status, kFixLossBits, kFixLossMaxContribution);
        red_add_fix(Q + 4, l_den, status, kFixLossBits, kFixLossMaxContribution);
      } else {
        float* L = dyn[bi].loss;
        atomicAdd(L + 0, loss);
        if (l_rgb != 0.f) atomicAdd(L + 1, l_rgb);
        if (l_rr != 0.f) atomicAdd(L + 2, l_rr);
        if (l_dep != 0.f) atomicAdd(L + 3, l_dep);
        if (l_den != 0.f) atomicAdd(L + 4, l_den);
      }
      if (!isfinite(loss) && status) atomicOr(status, 1);
    }
  } else {
    const float* u = R.gout + 6 * r;
    gC0 = u[0]; gC1 = u[1]; gC2 = u[2]; gD = u[3]; gA = u[4]; gdir = u[5];
  }

  // ---- adjoint, chunks in reverse order -----------------------------------
  float SC0 = 0.f, SC1 = 0.f, SC2 = 0.f, SD = 0.f;  // sum_{j > chunk} w_j c_j, w_j t_j
  const float bgterm = Tend * (gC0 * bg0 + gC1 * bg1 + gC2 * bg2);
  if (cnt == 0) return;
  for (int base = (int)((cnt - 1) / 32) * 32; base >= 0; base -= 32) {
    const uint32_t j = (uint32_t)base + lane;
    const bool in = j < cnt;
    const float sg = in ? S.sigma[off + j] : 0.f;
    const float dt = in ? S.dt[off + j] : 0.f;
    const float tt = in ? S.t[off + j] : 0.f;
    const float P = in ? S.dsigma[off + j] : 0.f;
    const float c0 = in ? S.rgb[3 * (off + j)] : 0.f;
    const float c1 = in ? S.rgb[3 * (off + j) + 1] : 0.f;
    const float c2 = in ? S.rgb[3 * (off + j) + 2] : 0.f;
    const float sd = sg * dt;
    const float Ti = expf(-P);
    const float Tn = expf(-(P + sd));
    const float w = in ? Ti * (-expm1f(-sd)) : 0.f;
    const float wc0 = w * c0, wc1 = w * c1, wc2 = w * c2, wt = w * tt;
    float s0 = warp_incl_suffix(wc0, lane), s1 = warp_incl_suffix(wc1, lane);
    float s2 = warp_incl_suffix(wc2, lane), s3 = warp_incl_suffix(wt, lane);
    float e0 = __shfl_down_sync(0xffffffffu, s0, 1), e1 = __shfl_down_sync(0xffffffffu, s1, 1);
    float e2 = __shfl_down_sync(0xffffffffu, s2, 1), e3 = __shfl_down_sync(0xffffffffu, s3, 1);
    if (lane == 31) e0 = e1 = e2 = e3 = 0.f;
    const float suf0 = SC0 + e0, suf1 = SC1 + e1, suf2 = SC2 + e2, sufD = SD + e3;
    float gs = gC0 * (Tn * c0 - suf0) + gC1 * (Tn * c1 - suf1) + gC2 * (Tn * c2 - suf2) - bgterm;
    gs += gD * (Tn * tt - sufD) + gA * Tend;
    gs = dt * gs + gdir;
    if (in) {
      S.dsigma[off + j] = gs;
      S.drgb[3 * (off + j)] = gC0 * w;
      S.drgb[3 * (off + j) + 1] = gC1 * w;
      S.drgb[3 * (off + j) + 2] = gC2 * w;
    }
    SC0 += __shfl_sync(0xffffffffu, s0, 0);
    SC1 += __shfl_sync(0xffffffffu, s1, 0);
    SC2 += __shfl_sync(0xffffffffu, s2, 0);
    SD += __shfl_sync(0xffffffffu, s3, 0);
  }
}

void launch_composite(int mode, const GridParams& g, const BatchDesc& b, RayBuf r, SampleBuf s, BatchDyn* dyn,
                      int32_t* status, cudaStream_t stream) {
  if (b.n_rays <= 0) return;
  unsigned blocks = (unsigned)(((int64_t)b.n_rays * 32 + 255) / 256);
  if (mode == 0) k_composite<0><<<blocks, 256, 0, stream>>>(g, b, r, s, dyn, status);
  else if (mode == 1) k_composite<1><<<blocks, 256, 0, stream>>>(g, b, r, s, dyn, status);
  else k_composite<2><<<blocks, 256, 0, stream>>>(g, b, r, s, dyn, status);
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba) with bias correction over every parameter of every
// batch object; zeroes the gradient; optionally refreshes the FP16 copy of
// the hash table.  float4 streaming, grid (chunks, objects).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void adam4(float4& p, float4& m, float4& v, const float4 gr, float b1, float b2, float ob1,
                                      float ob2, float lr, float eps, float c1, float c2) {
  float* pp = &p.x; float* mm = &m.x; float* vv = &v.x;
  const float* gg = &gr.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    mm[k] = b1 * mm[k] + ob1 * gg[k];
    vv[k] = b2 * vv[k] + ob2 * gg[k] * gg[k];
    pp[k] -= lr * (mm[k] * c1) / (sqrtf(vv[k] * c2) + eps);
  }
}

// Exact skip of never-touched parameters.  Every chunk of kAdamChunk parameters (64 float4 groups, two per lane of one
// warp) has a touched flag, 0 while every gradient the chunk has received was 0.  Such a chunk has m = v = g = 0, for
// which the Adam step is exactly nothing: m' = b1 0 + (1 - b1) 0 = 0, v' = 0, p' = p - lr 0 / (0 + eps) = p, the
// gradient is already 0 and the FP16 copy already equals p.  So the warp reads only the chunk's gradient and moves
// on; the first non-zero (or NaN) gradient flags the chunk, which is updated at every step from then on, as in dense
// Adam.  The results are bit-identical to updating every parameter.
__device__ __forceinline__ bool nonzero4(const float4& a) {
  return a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f;
}

__global__ void __launch_bounds__(256) k_adam(GridParams g, BatchDesc b, int write_half, int prev) {
  const ObjectDev& ob = b.objs[b.slot[blockIdx.y]];
  // bias corrections of this step, set with the step counter; prev: the update of the step before, run after the
  // counter has already advanced (it overlaps the next step's sampling)
  const float c1 = prev ? ob.bc1_prev : ob.bc1, c2 = prev ? ob.bc2_prev : ob.bc2;
  const float b1 = g.beta1, b2 = g.beta2, lr = g.lr, eps = g.eps;
  const float ob1 = 1.0f - b1, ob2 = 1.0f - b2;
  float4* P = reinterpret_cast<float4*>(ob.params);
  float4* G = reinterpret_cast<float4*>(ob.grad);
  float4* M = reinterpret_cast<float4*>(ob.m);
  float4* V = reinterpret_cast<float4*>(ob.v);
  __half2* H = reinterpret_cast<__half2*>(ob.table_h);
  uint8_t* touched = g.adam_dense ? nullptr : ob.touched;
  const bool half = write_half && ob.table_h;
  const int64_t n4 = g.n_params_pad / 4;
  const int64_t nh4 = g.n_hash / 4;  // n_hash is even; the FP16 copy covers whole float4s below n_hash
  constexpr int kChunk4 = kAdamChunk / 4;
  const int64_t n_chunks = (n4 + kChunk4 - 1) / kChunk4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_chunks; c += warps) {
    const int64_t i = c * kChunk4 + lane, j = i + 32;
    const bool vi = i < n4, vj = j < n4;
    float4 g0, g1, m0 = zero, m1 = zero, v0 = zero, v1 = zero, p0 = zero, p1 = zero;
    const bool was = touched == nullptr || touched[c] != 0;  // one byte, the same for the whole warp
    if (was) {  // issue every load of the chunk at once
      g0 = vi ? G[i] : zero; g1 = vj ? G[j] : zero;
      if (vi) { m0 = __ldcs(M + i); v0 = __ldcs(V + i); p0 = P[i]; }
      if (vj) { m1 = __ldcs(M + j); v1 = __ldcs(V + j); p1 = P[j]; }
    } else {
      g0 = vi ? G[i] : zero; g1 = vj ? G[j] : zero;
      if (!__any_sync(0xffffffffu, nonzero4(g0) || nonzero4(g1))) continue;  // m = v = g = 0: nothing changes
      if (lane == 0) touched[c] = 1;
      if (vi) { m0 = __ldcs(M + i); v0 = __ldcs(V + i); p0 = P[i]; }
      if (vj) { m1 = __ldcs(M + j); v1 = __ldcs(V + j); p1 = P[j]; }
    }
    if (vi) {
      adam4(p0, m0, v0, g0, b1, b2, ob1, ob2, lr, eps, c1, c2);
      P[i] = p0;
      __stcs(M + i, m0);
      __stcs(V + i, v0);
      G[i] = zero;
      if (half && i < nh4) { H[2 * i] = __floats2half2_rn(p0.x, p0.y); H[2 * i + 1] = __floats2half2_rn(p0.z, p0.w); }
    }
    if (vj) {
      adam4(p1, m1, v1, g1, b1, b2, ob1, ob2, lr, eps, c1, c2);
      P[j] = p1;
      __stcs(M + j, m1);
      __stcs(V + j, v1);
      G[j] = zero;
      if (half && j < nh4) { H[2 * j] = __floats2half2_rn(p1.x, p1.y); H[2 * j + 1] = __floats2half2_rn(p1.z, p1.w); }
    }
  }
}

// Deterministic mode: fixed-point gradient -> FP32 gradient (added; zero accumulators are skipped) and accumulator
// reset; block (0, entry) also converts the entry's fixed-point loss sums.
__global__ void __launch_bounds__(256) k_fix_finish(GridParams g, BatchDesc b, BatchDyn* dyn) {
  const ObjectDev& ob = b.objs[b.slot[blockIdx.y]];
  if (blockIdx.x == 0 && threadIdx.x < 5) {
    const int k = threadIdx.x;
    dyn[blockIdx.y].loss[k] = (float)ldexp((double)(long long)dyn[blockIdx.y].loss_fix[k], -kFixLossBits);
  }
  longlong2* Q = reinterpret_cast<longlong2*>(ob.gfix);
  float2* G = reinterpret_cast<float2*>(ob.grad);
  if (!Q) return;
  const int64_t n2 = g.n_params_pad / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const longlong2 q = Q[i];
    if (q.x == 0 && q.y == 0) continue;
    float2 gg = G[i];
    gg.x += (float)ldexp((double)q.x, -kFixBits);
    gg.y += (float)ldexp((double)q.y, -kFixBits);
    G[i] = gg;
    Q[i] = make_longlong2(0, 0);
  }
}

void launch_fix_finish(const GridParams& g, const BatchDesc& b, BatchDyn* dyn, cudaStream_t stream) {
  if (b.n <= 0) return;
  int64_t n2 = g.n_params_pad / 2;
  int chunks = (int)((n2 + 255) / 256);
  int max_chunks = 4096 / (b.n < 1 ? 1 : b.n) + 1;
  if (max_chunks < 16) max_chunks = 16;
  if (chunks > max_chunks) chunks = max_chunks;
  k_fix_finish<<<dim3(chunks, b.n), 256, 0, stream>>>(g, b, dyn);
}

__global__ void k_touched_from_moments(int64_t n4, const float4* __restrict__ M, const float4* __restrict__ V,
                                       uint8_t* __restrict__ touched) {
  constexpr int kChunk4 = kAdamChunk / 4;
  const int64_t n_chunks = (n4 + kChunk4 - 1) / kChunk4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_chunks; c += warps) {
    bool nz = false;
    for (int64_t i = c * kChunk4 + lane; i < (c + 1) * kChunk4 && i < n4; i += 32)
      nz = nz || nonzero4(M[i]) || nonzero4(V[i]);
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) touched[c] = nz ? 1 : 0;
  }
}

void launch_touched_from_moments(const GridParams& g, const float* m, const float* v, uint8_t* touched,
                                 cudaStream_t stream) {
  const int64_t n4 = g.n_params_pad / 4;
  const int64_t n_chunks = (n4 + kAdamChunk / 4 - 1) / (kAdamChunk / 4);
  int blocks = (int)((n_chunks + 7) / 8);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_touched_from_moments<<<blocks, 256, 0, stream>>>(n4, reinterpret_cast<const float4*>(m),
                                                     reinterpret_cast<const float4*>(v), touched);
}

__global__ void k_advance_step(GridParams g, BatchDesc b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < b.n) {
    ObjectDev& ob = b.objs[b.slot[i]];
    set_object_step(ob, ob.step + 1u, g.beta1, g.beta2);
  }
}

// Per-object loss of the batch's last step, L = (loss sum) / B with the same FP32 operations as the host read, into a
// device array: the source of an asynchronous loss copy.
__global__ void k_final_losses(const BatchDyn* __restrict__ dyn, const int32_t* __restrict__ ray_base, int n,
                               float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float B = (float)(ray_base[i + 1] - ray_base[i]);
  const float inv = B > 0.f ? 1.0f / B : 0.0f;
  out[i] = dyn[i].loss[0] * inv;
}

void launch_final_losses(const BatchDyn* dyn, const BatchDesc& b, float* out, cudaStream_t stream) {
  if (b.n <= 0) return;
  k_final_losses<<<(b.n + 127) / 128, 128, 0, stream>>>(dyn, b.ray_base, b.n, out);
}

void launch_adam_update(const GridParams& g, const BatchDesc& b, int write_half, int prev, cudaStream_t stream) {
  if (b.n <= 0) return;
  int64_t n4 = g.n_params_pad / 4;
  int chunks = (int)((n4 + 511) / 512);  // blocks of 8 warps, one 64-float4 chunk per warp and round
  int max_chunks = 4096 / (b.n < 1 ? 1 : b.n) + 1;  // about 4k blocks of 256 threads, two float4 groups per lane
  if (max_chunks < 16) max_chunks = 16;
  if (chunks > max_chunks) chunks = max_chunks;
  k_adam<<<dim3(chunks, b.n), 256, 0, stream>>>(g, b, write_half, prev);
}

void launch_advance_step(const GridParams& g, const BatchDesc& b, cudaStream_t stream) {
  if (b.n <= 0) return;
  k_advance_step<<<(b.n + 127) / 128, 128, 0, stream>>>(g, b);
}

void launch_adam(const GridParams& g, const BatchDesc& b, int write_half, cudaStream_t stream) {
  launch_adam_update(g, b, write_half, 0, stream);
  launch_advance_step(g, b, stream);
}

__global__ void k_split_outputs(const float* __restrict__ ray_out, int64_t n, float* rgb, float* depth,
                                float* opacity) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float* o = ray_out + 6 * r;
  rgb[3 * r] = o[0]; rgb[3 * r + 1] = o[1]; rgb[3 * r + 2] = o[2];
  depth[r] = o[3];
  opacity[r] = o[4];
}

void launch_split_outputs(const float* ray_out, int64_t n, float* rgb, float* depth, float* opacity,
                          cudaStream_t stream) {
  if (n <= 0) return;
  k_split_outputs<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(ray_out, n, rgb, depth, opacity);
}

}  // namespace romap
