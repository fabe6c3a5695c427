// Mesh extraction by marching cubes (Table 3: 64^3 per object): 64^3 cubes over the object box, the density net at
// the 65^3 lattice vertices x_a = -a + i ((a - (-a)) / 64) (FP32, FP32 master parameters), one shared vertex per
// lattice edge whose ends lie on opposite sides of the iso-level (linear interpolation), and per cube the
// triangles of its inside/outside pattern from the constructed case table, as indices into the vertex buffer.
// Vertices are numbered in the order (lattice vertex, axis) by an exclusive prefix sum; triangles in cube order.
#include <cstdint>

#include "density_eval.cuh"

namespace romap {
namespace {

constexpr int kLat = 65;
constexpr int kLatN = kLat * kLat * kLat;
constexpr int kCubes = 64 * 64 * 64;
constexpr int kRow = 3 * kMcMaxTri + 1;

__constant__ int8_t c_mc_tri[256 * kRow];
__constant__ uint8_t c_mc_cnt[256];

template <int LFP, bool XL>
__global__ void __launch_bounds__(256) k_lattice_density(GridParams g, const ObjectDev* objs, int slot, float* dens) {
  __shared__ DensityWeights<LFP, XL> sw;
  const ObjectDev& ob = objs[slot];
  load_density_weights<LFP, XL>(sw, g, ob.params);
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= kLatN) return;
  const int idx[3] = {v % kLat, (v / kLat) % kLat, v / (kLat * kLat)};
  float x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = -ob.half[a];
    const float w = __fdiv_rn(__fsub_rn(ob.half[a], lo), 64.0f);
    x[a] = __fadd_rn(lo, __fmul_rn((float)idx[a], w));
  }
  dens[v] = density_at<LFP, XL>(sw, g, ob, x);
}

// bit d set: the lattice edge from v along axis d crosses the iso-level
__device__ __forceinline__ uint32_t crossing_bits(const float* dens, float iso, int v) {
  const int i = v % kLat, j = (v / kLat) % kLat, k = v / (kLat * kLat);
  const bool in = dens[v] > iso;
  uint32_t b = 0;
  if (i < 64 && (dens[v + 1] > iso) != in) b |= 1u;
  if (j < 64 && (dens[v + kLat] > iso) != in) b |= 2u;
  if (k < 64 && (dens[v + kLat * kLat] > iso) != in) b |= 4u;
  return b;
}

__global__ void k_mc_edge_count(const float* dens, float iso, uint32_t* cnt) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < kLatN) cnt[v] = __popc(crossing_bits(dens, iso, v));
}

__global__ void k_mc_vertices(const float* dens, float iso, const uint32_t* off, const ObjectDev* objs, int slot,
                              int64_t cap, float* verts, int32_t* evid) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= kLatN) return;
  const float* half = objs[slot].half;
  const uint32_t b = crossing_bits(dens, iso, v);
  const int idx[3] = {v % kLat, (v / kLat) % kLat, v / (kLat * kLat)};
  const int step[3] = {1, kLat, kLat * kLat};
  uint32_t id = off[v];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!((b >> d) & 1u)) {
      evid[3 * v + d] = -1;
      continue;
    }
    evid[3 * v + d] = (int32_t)id;
    if ((int64_t)id < cap) {
      const float s0 = dens[v], s1 = dens[v + step[d]];
      const float t = (iso - s0) / (s1 - s0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float lo = -half[a];
        const float w = __fdiv_rn(__fsub_rn(half[a], lo), 64.0f);
        const float p0 = __fadd_rn(lo, __fmul_rn((float)idx[a], w));
        const float p1 = __fadd_rn(lo, __fmul_rn((float)(idx[a] + (a == d ? 1 : 0)), w));
        verts[3 * (int64_t)id + a] = p0 + t * (p1 - p0);
      }
    }
    ++id;
  }
}

__device__ __forceinline__ int cube_case(const float* dens, float iso, int c, int* v0) {
  const int i = c & 63, j = (c >> 6) & 63, k = c >> 12;
  *v0 = i + kLat * j + kLat * kLat * k;
  int cs = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int v = *v0 + (q & 1) + kLat * ((q >> 1) & 1) + kLat * kLat * ((q >> 2) & 1);
    cs |= (dens[v] > iso ? 1 : 0) << q;
  }
  return cs;
}

__global__ void k_mc_tri_count(const float* dens, float iso, uint32_t* cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kCubes) return;
  int v0;
  cnt[c] = c_mc_cnt[cube_case(dens, iso, c, &v0)];
}

__global__ void k_mc_triangles(const float* dens, float iso, const uint32_t* off, const int32_t* evid, int64_t cap,
                               int32_t* tris) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kCubes) return;
  int v0;
  const int cs = cube_case(dens, iso, c, &v0);
  const int n = c_mc_cnt[cs];
  for (int t = 0; t < n; ++t) {
    const int64_t tid = (int64_t)off[c] + t;
    if (tid >= cap) return;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int e = c_mc_tri[cs * kRow + 3 * t + r];
      // edge e = 4 d + q along axis d; q holds the other two axes' corner bits, lower axis first
      const int d = e >> 2, q = e & 3;
      const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
      const int lo = o1 < o2 ? o1 : o2, hi = o1 < o2 ? o2 : o1;
      const int corner = ((q & 1) << lo) | (((q >> 1) & 1) << hi);
      const int v = v0 + (corner & 1) + kLat * ((corner >> 1) & 1) + kLat * kLat * ((corner >> 2) & 1);
      tris[3 * tid + r] = evid[3 * v + d];
    }
  }
}

// Exclusive prefix sum of n <= 1024 * 1024 values: per 1024-element block, then the block sums, then the adds.
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t* in, uint32_t* out, int n, uint32_t* bsum) {
  __shared__ uint32_t ws[32];
  const int i = blockIdx.x * 1024 + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t v = i < n ? in[i] : 0u;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = w > 0 ? ws[w - 1] : 0u;
  if (i < n) out[i] = before + x - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = before + x;
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t* bsum, int nb, uint32_t* total) {
  __shared__ uint32_t ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t v = threadIdx.x < (unsigned)nb ? bsum[threadIdx.x] : 0u;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const uint32_t before = w > 0 ? ws[w - 1] : 0u;
  if (threadIdx.x < (unsigned)nb) bsum[threadIdx.x] = before + x - v;
  if (threadIdx.x == 1023) *total = before + x;
}

__global__ void k_scan_add(uint32_t* out, int n, const uint32_t* bsum) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n && blockIdx.x > 0) out[i] += bsum[blockIdx.x];
}

void scan_u32(const uint32_t* in, uint32_t* out, int n, uint32_t* bsum, uint32_t* total, cudaStream_t stream) {
  const int nb = (n + 1023) / 1024;  // <= 1024
  k_scan_block<<<nb, 1024, 0, stream>>>(in, out, n, bsum);
  k_scan_sums<<<1, 1024, 0, stream>>>(bsum, nb, total);
  k_scan_add<<<nb, 1024, 0, stream>>>(out, n, bsum);
}

}  // namespace

size_t mc_workspace_bytes() {
  return sizeof(float) * kLatN + 2 * sizeof(uint32_t) * kLatN + 3 * sizeof(int32_t) * kLatN +
         2 * sizeof(uint32_t) * kCubes + 2 * 1024 * sizeof(uint32_t) + 4 * sizeof(uint32_t) + 8 * 256;
}

int mc_lattice_points() { return kLatN; }

void launch_lattice_density(const GridParams& g, const ObjectDev* objs, int slot, float* dens, cudaStream_t stream) {
  const int blocks = (kLatN + 255) / 256;
  auto k = g.LF <= 16 ? (g.extra ? k_lattice_density<16, true> : k_lattice_density<16, false>)
                      : (g.extra ? k_lattice_density<32, true> : k_lattice_density<32, false>);
  k<<<blocks, 256, 0, stream>>>(g, objs, slot, dens);
}

// Counting pass (emit = 0): uploads the case table, evaluates the lattice densities into ws (laid out below) and
// writes the vertex and triangle totals to totals_out[0..1].  Emission pass (emit = 1, after a counting pass on the
// same ws): vertices and triangles, each up to its capacity.  Returns the kernels launched.
int launch_mc(const GridParams& g, const ObjectDev* objs, int slot, float iso, char* ws,
              int emit, int64_t cap_v, float* verts, int64_t cap_t, int32_t* tris, uint32_t* totals_out,
              const int8_t* table, const uint8_t* counts, cudaStream_t stream) {
  char* p = ws;
  float* dens = reinterpret_cast<float*>(p); p += sizeof(float) * kLatN;
  uint32_t* ecnt = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * kLatN;
  uint32_t* eoff = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * kLatN;
  int32_t* evid = reinterpret_cast<int32_t*>(p); p += 3 * sizeof(int32_t) * kLatN;
  uint32_t* tcnt = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * kCubes;
  uint32_t* toff = reinterpret_cast<uint32_t*>(p); p += sizeof(uint32_t) * kCubes;
  uint32_t* bsum = reinterpret_cast<uint32_t*>(p); p += 2 * 1024 * sizeof(uint32_t);
  (void)p;
  int launches = 0;
  if (!emit) {
    cudaMemcpyToSymbolAsync(c_mc_tri, table, 256 * kRow, 0, cudaMemcpyHostToDevice, stream);
    cudaMemcpyToSymbolAsync(c_mc_cnt, counts, 256, 0, cudaMemcpyHostToDevice, stream);
    launch_lattice_density(g, objs, slot, dens, stream);
    k_mc_edge_count<<<(kLatN + 255) / 256, 256, 0, stream>>>(dens, iso, ecnt);
    scan_u32(ecnt, eoff, kLatN, bsum, totals_out, stream);
    k_mc_tri_count<<<kCubes / 256, 256, 0, stream>>>(dens, iso, tcnt);
    scan_u32(tcnt, toff, kCubes, bsum + 1024, totals_out + 1, stream);
    launches = 9;
  } else {
    k_mc_vertices<<<(kLatN + 255) / 256, 256, 0, stream>>>(dens, iso, eoff, objs, slot, cap_v, verts, evid);
    k_mc_triangles<<<kCubes / 256, 256, 0, stream>>>(dens, iso, toff, evid, cap_t, tris);
    launches = 2;
  }
  return launches;
}

}  // namespace romap
