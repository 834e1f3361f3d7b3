// World radius of every point for stochastic point discarding (Sec. 3.1,
// "Stochastic Point Discarding": r_world = distance to the k-th nearest
// point, k = 4 in the paper), exact, on a hashed uniform grid.
//
//   1. bounding box (float min/max as ordered integers, atomics)
//   2. cell size h: the median k-NN distance of 256 sampled points, each found
//      by one block scanning the whole cloud (the only host synchronisation)
//   3. counting sort of the points by the hash of their cell
//   4. per point: visit cells in shells of growing Chebyshev radius r around
//      its own, keep the k smallest squared distances, and stop once the k-th
//      is <= (r h)^2 (no point outside the visited cube can be closer); the
//      work per point is bounded (see k_query).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "launch.h"

namespace adop {
namespace knn {
namespace {

constexpr int kMaxK = 16;
constexpr int kSamples = 256;

__device__ __forceinline__ uint32_t ordered(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__global__ void k_bbox(const float* __restrict__ xyz, int64_t n, uint32_t* box) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const uint32_t o = ordered(__ldg(xyz + 3 * i + d));
      lo[d] = min(lo[d], o);
      hi[d] = max(hi[d], o);
    }
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], s));
      hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], s));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(box + d, lo[d]);
      atomicMax(box + 3 + d, hi[d]);
    }
  }
}

// keep the k smallest values of a sorted ascending list
__device__ __forceinline__ void insert_k(float* best, int k, int& m, float d2) {
  if (m == k && d2 >= best[k - 1]) return;
  int q = m < k ? m++ : k - 1;
  while (q > 0 && best[q - 1] > d2) {
    best[q] = best[q - 1];
    --q;
  }
  best[q] = d2;
}

// One block per sampled point: the k smallest squared distances over the cloud.
__global__ void __launch_bounds__(256) k_sample_knn(const float* __restrict__ xyz, int64_t n, int k, float* out) {
  __shared__ float s_best[256 * kMaxK];
  const int64_t si = (int64_t)blockIdx.x * n / kSamples;
  const float px = __ldg(xyz + 3 * si), py = __ldg(xyz + 3 * si + 1), pz = __ldg(xyz + 3 * si + 2);
  float best[kMaxK];
  int m = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    if (j == si) continue;
    const float dx = __ldg(xyz + 3 * j) - px, dy = __ldg(xyz + 3 * j + 1) - py, dz = __ldg(xyz + 3 * j + 2) - pz;
    insert_k(best, k, m, dx * dx + dy * dy + dz * dz);
  }
  for (int q = 0; q < k; ++q) s_best[threadIdx.x * kMaxK + q] = q < m ? best[q] : INFINITY;
  __syncthreads();
  if (threadIdx.x == 0) {
    float all[kMaxK];
    int mm = 0;
    for (int t = 0; t < (int)blockDim.x; ++t)
      for (int q = 0; q < k; ++q) {
        const float v = s_best[t * kMaxK + q];
        if (v == INFINITY) break;
        insert_k(all, k, mm, v);
      }
    out[blockIdx.x] = mm < k ? INFINITY : sqrtf(all[k - 1]);
  }
}

struct Grid {
  float ox, oy, oz, inv_h, h;
  uint32_t mask;  // buckets - 1
};

__device__ __forceinline__ void cell_of(const Grid& g, float x, float y, float z, int& cx, int& cy, int& cz) {
  cx = (int)floorf((x - g.ox) * g.inv_h);
  cy = (int)floorf((y - g.oy) * g.inv_h);
  cz = (int)floorf((z - g.oz) * g.inv_h);
}

__device__ __forceinline__ uint32_t bucket(const Grid& g, int cx, int cy, int cz) {
  return (((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u)) & g.mask;
}

__global__ void k_count(const float* __restrict__ xyz, int64_t n, Grid g, uint32_t* __restrict__ bkt,
                        uint32_t* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_of(g, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2), cx, cy, cz);
    const uint32_t b = bucket(g, cx, cy, cz);
    bkt[i] = b;
    atomicAdd(count + b, 1u);
  }
}

// Exclusive scan of `count` (length m) into `start` (length m + 1), three
// phases over tiles of 4096 entries.
constexpr int kScanTile = 4096;

__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* __restrict__ count, int64_t m,
                                                     uint32_t* __restrict__ tile_sum) {
  __shared__ uint32_t warp_sum[32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 4;
  uint32_t s = 0;
  for (int q = 0; q < 4; ++q)
    if (t0 + q < m) s += count[t0 + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = warp_sum[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t* __restrict__ tile_sum, int64_t tiles) {
  // single block: exclusive scan of the tile sums, serial chunks per thread
  __shared__ uint32_t warp_sum[32];
  const int64_t per = (tiles + 1023) / 1024;
  const int64_t a = threadIdx.x * per, b = min(tiles, a + per);
  uint32_t local = 0;
  for (int64_t t = a; t < b; ++t) local += tile_sum[t];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w;
  }
  __syncthreads();
  uint32_t run = incl - local + (warp > 0 ? warp_sum[warp - 1] : 0u);
  for (int64_t t = a; t < b; ++t) {
    const uint32_t v = tile_sum[t];
    tile_sum[t] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t* __restrict__ count, int64_t m,
                                                     const uint32_t* __restrict__ tile_off, uint32_t* __restrict__ start,
                                                     uint32_t* __restrict__ cursor, uint32_t total) {
  __shared__ uint32_t warp_sum[32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 4;
  uint32_t v[4], s = 0;
  for (int q = 0; q < 4; ++q) {
    v[q] = t0 + q < m ? count[t0 + q] : 0u;
    s += v[q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w;
  }
  __syncthreads();
  uint32_t run = tile_off[blockIdx.x] + incl - s + (warp > 0 ? warp_sum[warp - 1] : 0u);
  for (int q = 0; q < 4; ++q)
    if (t0 + q < m) {
      start[t0 + q] = run;
      cursor[t0 + q] = run;
      run += v[q];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) start[m] = total;
}

__global__ void k_scatter(const float* __restrict__ xyz, int64_t n, const uint32_t* __restrict__ bkt,
                          uint32_t* __restrict__ cursor, float4* __restrict__ sorted) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t pos = atomicAdd(cursor + bkt[i], 1u);
    sorted[pos] = make_float4(__ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2),
                              __int_as_float((int)i));
  }
}

// Work per point is bounded: at most kMaxRing shells and kMaxScan candidate
// points.  Within those limits the result is exact; past them the point gets
// the k-th smallest distance found so far (an upper bound, and the true value
// is then at least kMaxRing cells away), or +inf if fewer than k were found.
constexpr int kMaxRing = 8;
constexpr int kMaxScan = 1 << 16;

__global__ void __launch_bounds__(256) k_query(const float* __restrict__ xyz, int64_t n, int k, Grid g,
                                               const uint32_t* __restrict__ start, const float4* __restrict__ sorted,
                                               int max_ring, float* __restrict__ radius) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float px = __ldg(xyz + 3 * i), py = __ldg(xyz + 3 * i + 1), pz = __ldg(xyz + 3 * i + 2);
    int cx, cy, cz;
    cell_of(g, px, py, pz, cx, cy, cz);
    float best[kMaxK];
    int m = 0, scanned = 0;
    bool done = false;
    const int rings = min(max_ring, kMaxRing);
    for (int r = 0; r <= rings && !done; ++r) {
      for (int dz = -r; dz <= r && !done; ++dz)
        for (int dy = -r; dy <= r && !done; ++dy)
          for (int dx = -r; dx <= r && !done; ++dx) {
            if (max(abs(dx), max(abs(dy), abs(dz))) != r) continue;  // this shell only
            const int qx = cx + dx, qy = cy + dy, qz = cz + dz;
            const uint32_t b = bucket(g, qx, qy, qz);
            const uint32_t e = __ldg(start + b + 1);
            for (uint32_t s = __ldg(start + b); s < e; ++s) {
              if (++scanned > kMaxScan) {
                done = true;
                break;
              }
              const float4 q = __ldg(sorted + s);
              if (__float_as_int(q.w) == (int)i) continue;
              int ox, oy, oz;
              cell_of(g, q.x, q.y, q.z, ox, oy, oz);
              if (ox != qx || oy != qy || oz != qz) continue;  // another cell in the same bucket
              const float ddx = q.x - px, ddy = q.y - py, ddz = q.z - pz;
              insert_k(best, k, m, ddx * ddx + ddy * ddy + ddz * ddz);
            }
            if (m == k && best[k - 1] == 0.0f) done = true;  // k duplicates: nothing is closer
          }
      // every point outside the visited cube is at least r h away (minus rounding)
      const float reach = (float)r * g.h * (1.0f - 1e-5f);
      done = done || ((m == k) && best[k - 1] <= reach * reach);
    }
    radius[i] = m < k ? INFINITY : sqrtf(best[k - 1]);
  }
}

struct Layout {
  size_t box, samples, bkt, count, start, cursor, tiles, sorted, total;
  int64_t m;
};

size_t up(size_t v) { return (v + 255) / 256 * 256; }

Layout layout(int64_t n) {
  Layout L{};
  int64_t m = 1;
  while (m < n) m <<= 1;
  L.m = m;
  size_t o = 0;
  L.box = o;       o = up(o + 6 * 4);
  L.samples = o;   o = up(o + kSamples * 4);
  L.bkt = o;       o = up(o + (size_t)n * 4);
  L.count = o;     o = up(o + (size_t)m * 4);
  L.start = o;     o = up(o + ((size_t)m + 1) * 4);
  L.cursor = o;    o = up(o + (size_t)m * 4);
  L.tiles = o;     o = up(o + (size_t)((m + kScanTile - 1) / kScanTile) * 4);
  L.sorted = o;    o = up(o + (size_t)n * 16);
  L.total = o;
  return L;
}

}  // namespace
}  // namespace knn
}  // namespace adop

using namespace adop::knn;

extern "C" {

size_t adop_point_radius_workspace_bytes(int64_t n) {
  if (n < 0 || n >= ((int64_t)1 << 31)) return 0;
  return layout(n < 1 ? 1 : n).total;
}

adop_status adop_point_radius(const float* xyz, int64_t n, int32_t k, float* radius, void* workspace,
                              size_t workspace_bytes, adop_stream stream) {
  auto fail = [](adop_status st, const char* msg) {
    adop::set_last_error(msg);
    return st;
  };
  if (n < 0 || n >= ((int64_t)1 << 31)) return fail(ADOP_ERR_INVALID_ARG, "point count outside [0, 2^31)");
  if (k < 1 || k > kMaxK) return fail(ADOP_ERR_INVALID_ARG, "k outside [1, 16]");
  if (n == 0) return ADOP_OK;
  if (!xyz || !radius) return fail(ADOP_ERR_INVALID_ARG, "xyz and radius must not be NULL");
  const Layout L = layout(n);
  if (workspace_bytes < L.total) return fail(ADOP_ERR_OUT_OF_MEMORY, "workspace too small for adop_point_radius");
  if (!workspace || ((uintptr_t)workspace & 255) != 0)
    return fail(ADOP_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  uint32_t* box = reinterpret_cast<uint32_t*>(ws + L.box);
  float* samples = reinterpret_cast<float*>(ws + L.samples);
  uint32_t* bkt = reinterpret_cast<uint32_t*>(ws + L.bkt);
  uint32_t* count = reinterpret_cast<uint32_t*>(ws + L.count);
  uint32_t* start = reinterpret_cast<uint32_t*>(ws + L.start);
  uint32_t* cursor = reinterpret_cast<uint32_t*>(ws + L.cursor);
  uint32_t* tiles = reinterpret_cast<uint32_t*>(ws + L.tiles);
  float4* sorted = reinterpret_cast<float4*>(ws + L.sorted);
  const int blocks = adop::num_sms() * 8;
  cudaError_t e;
  const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
  if ((e = cudaMemcpyAsync(box, init, sizeof(init), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
  k_bbox<<<blocks, 256, 0, s>>>(xyz, n, box);
  k_sample_knn<<<kSamples, 256, 0, s>>>(xyz, n, k, samples);
  uint32_t hbox[6];
  float hs[kSamples];
  if ((e = cudaMemcpyAsync(hbox, box, sizeof(hbox), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(hs, samples, sizeof(hs), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
  auto unord = [](uint32_t o) {
    uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
    memcpy(&f, &b, 4);
    return f;
  };
  float lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = unord(hbox[d]);
    hi[d] = unord(hbox[3 + d]);
  }
  const float extent = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 0.0f});
  if (!std::isfinite(extent)) return fail(ADOP_ERR_INVALID_ARG, "non-finite point positions");
  std::vector<float> v;
  for (float x : hs)
    if (std::isfinite(x)) v.push_back(x);
  float h = 0.0f;
  if (!v.empty()) {
    std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
    h = 1.5f * v[v.size() / 2];
  }
  // at least extent / 2^20 (bounded cell coordinates) and a tiny absolute floor
  h = std::max({h, extent / 1048576.0f, 1e-20f});
  if (v.empty()) h = std::max(extent, 1e-20f);  // fewer than k + 1 points
  const int max_ring = (int)std::ceil(extent / h) + 2;
  Grid g{lo[0], lo[1], lo[2], 1.0f / h, h, (uint32_t)(L.m - 1)};
  if ((e = cudaMemsetAsync(count, 0, (size_t)L.m * 4, s)) != cudaSuccess) return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
  k_count<<<blocks, 256, 0, s>>>(xyz, n, g, bkt, count);
  const int64_t nt = (L.m + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)nt, 1024, 0, s>>>(count, L.m, tiles);
  k_scan_sums<<<1, 1024, 0, s>>>(tiles, nt);
  k_scan_apply<<<(unsigned)nt, 1024, 0, s>>>(count, L.m, tiles, start, cursor, (uint32_t)n);
  k_scatter<<<blocks, 256, 0, s>>>(xyz, n, bkt, cursor, sorted);
  k_query<<<blocks, 256, 0, s>>>(xyz, n, k, g, start, sorted, max_ring, radius);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
  return ADOP_OK;
}

}  // extern "C"
