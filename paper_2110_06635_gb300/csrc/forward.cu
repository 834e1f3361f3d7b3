// Forward pass of the one-pixel point rasterizer (Sec. 3.1): a depth-only
// pass, an accumulate pass for the points that pass the fuzzy depth test and
// a per-pixel normalise pass (the three-pass structure of the paper's
// implementation details), preceded by a clear of the per-pixel state.
//
// Work decomposition: blockIdx.y selects the camera; blocks stride over
// points (or pixels) with a grid of whole waves of the kernel's resident
// blocks over the GPU's SMs (stride_grid).
#include <cuda_runtime.h>

#include "launch.h"

namespace adop {

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  return sms;
}

int point_blocks(int64_t n, int ncam) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  const int64_t cap = ((int64_t)num_sms() * 8 + ncam - 1) / ncam;
  int64_t b = want < cap ? want : cap;
  return (int)(b < 1 ? 1 : b);
}

namespace {
// Resident blocks per SM of kernel k (occupancy calculator), cached per
// calling thread: a launch asks the runtime once per kernel and thread.
int resident_blocks(const void* k, size_t smem) {
  struct Entry {
    const void* k;
    size_t smem;
    int n;
  };
  constexpr int kEntries = 256;
  static thread_local Entry cache[kEntries];
  static thread_local int used = 0;
  for (int i = 0; i < used; ++i)
    if (cache[i].k == k && cache[i].smem == smem) return cache[i].n;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kThreads, smem) != cudaSuccess || n < 1) n = 1;
  if (used < kEntries) cache[used++] = Entry{k, smem, n};
  return n;
}
}  // namespace

dim3 stride_grid(const void* k, int64_t work, int ncam, int waves, size_t smem) {
  const int64_t want = (work + kThreads - 1) / kThreads;
  const int64_t cap = ((int64_t)num_sms() * resident_blocks(k, smem) * waves + ncam - 1) / ncam;
  const int64_t b = want < cap ? want : cap;
  return dim3((unsigned)(b < 1 ? 1 : b), (unsigned)ncam);
}

// ---------------------------------------------------------------------------
// clear: key = UINT64_MAX (empty), count = 0, acc = 0 for every pixel
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(kThreads) k_clear(const __grid_constant__ LaunchCams cams,
                                                    const __grid_constant__ PointArgs a) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const int64_t total = cam.off[a.levels];
  // a pixel's sums as 256-bit stores (one full sector each) where C % 8 == 0
  // and acc is 32-byte aligned -- the workspace's always is, a caller's frame
  // need only be 16-byte aligned (23.1 -> 22.2 us on the 1080p step)
  const bool v8 = (C % 8 == 0) && (((uintptr_t)cam.acc & 31u) == 0u);
  int lc = 0;  // the layer of g: g only grows, so its layer only advances
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    while (lc + 1 < a.levels && g >= cam.off[lc + 1]) ++lc;
    const int l = lc;
    const int64_t p = g - cam.off[l];
    cam.key[l][p] = ~0ull;
    cam.cnt[l][p] = 0u;
    float* acc = cam.acc + g * C;
    if (v8) {
      const float z[C] = {};
      store_row<C>(acc, z);
    } else if constexpr (C % 4 == 0) {
#pragma unroll
      for (int v = 0; v < C / 4; ++v) reinterpret_cast<float4*>(acc)[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
      for (int k = 0; k < C; ++k) acc[k] = 0.0f;
    }
  }
}

// ---------------------------------------------------------------------------
// K1 depth pass: key[l][p] = min over points of (bits(z) << 32 | i)
// One thread per point; the keys are read first and the 64-bit atomicMin is
// issued only where the point can still win (most points are occluded).
// Every layer's key is read before any atomic, so that the kL reads are in
// flight together rather than one round trip per layer (65.5 -> 60.2 us on
// the 1080p step).  (Measured on GB300: grouping lanes that share a pixel
// with __match_any_sync was 4x slower -- the per-group warp intrinsics
// serialise -- and interleaving two points per thread 25% slower.)
// The pass also records, per point, the layers where it may still pass the
// fuzzy test (cam.early, one byte): it cannot where its depth already exceeds
// f32(z_cur (1 + alpha)) for the key z_cur it read, since keys only decrease
// (z_cur >= the final z_min, and f32(. * (1 + alpha)) is monotone), so the
// accumulate pass's test would reject it there as well.  The accumulate
// pass skips those layers' key reads, and skips outright the points outside
// the view or behind at every layer (on the 120M-point frame, 70% of the
// points are outside the view: accumulate 770 -> 581 us, and 528 us once the
// position is read only for points with a layer left).
// ---------------------------------------------------------------------------
template <int kL>
__global__ void __launch_bounds__(kThreads) k_depth(const __grid_constant__ LaunchCams cams,
                                                    const __grid_constant__ PointArgs a) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const float* __restrict__ xyz = cam.xyz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cam.n; i += (int64_t)gridDim.x * blockDim.x) {
    float X0, X1, X2, u0, v0, zd;
    uint32_t em = 0;  // layers where the point may still pass the fuzzy test
    transform(cam, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2), X0, X1, X2);
    if (camera(cam, X0, X1, X2, u0, v0, zd) && (zd > a.znear) && in_pyramid(u0, v0, cam.w, cam.h, a.levels) &&
        !(cam.normals && !normal_keep(cam, cam.normals, i, X0, X1, X2))) {
      const unsigned long long key = depth_key(zd, i);
      const float rw = a.radius ? __ldg(a.radius + i) : 0.0f, bt = a.radius ? __ldg(a.beta + i) : 0.0f;
      int32_t pix[kL];  // pixel within layer l (< 2^28), -1: none
#pragma unroll
      for (int l = 0; l < kL; ++l) {
        int32_t pu, pv;
        const bool keep = l < a.levels && (!a.radius || discard_keep(cam, zd, rw, bt, a.g2, l));
        pix[l] = (keep && pixel_in(u0, v0, l, cam.w, cam.h, pu, pv)) ? pv * (cam.w >> l) + pu : -1;
      }
      // (an L1-cached read may be stale, but keys only decrease: a stale value
      // can cost an atomic that loses, never skip one that wins, and it can
      // only keep a layer in the mask that a fresh value would have dropped)
      unsigned long long cur[kL];
#pragma unroll
      for (int l = 0; l < kL; ++l) cur[l] = pix[l] >= 0 ? __ldca(cam.key[l] + pix[l]) : 0ull;
#pragma unroll
      for (int l = 0; l < kL; ++l) {
        if (pix[l] < 0) continue;
        if (key < cur[l]) {
          atomicMin(cam.key[l] + pix[l], key);
          em |= 1u << l;
        } else if (!(zd > __fmul_rn(__uint_as_float((uint32_t)(cur[l] >> 32)), a.a1))) {
          em |= 1u << l;  // behind the current nearest point, but within the fuzzy threshold
        }
      }
    }
    if (cam.early) __stcs(cam.early + i, (uint8_t)em);
  }
}

// ---------------------------------------------------------------------------
// K2 accumulate: points with z <= f32(z_min * (1 + alpha)) add their
// descriptor to the pixel's FP32 sum (float4 vector atomics) and increment
// |Lambda|; each point's layer mask of passed tests is written for the
// backward pass, with the point's layer-0 screen tile in bits 8..31.  As in
// K1, every layer's key is read before the tests.
// ---------------------------------------------------------------------------
// 6 resident blocks per SM (at most 40 registers) where that costs no spills:
// 5 -> 6 blocks took the 1080p accumulate pass from 95 to 91 us.
template <int C, int kL>
constexpr int accum_min_blocks() {
  return (C <= 8 && kL <= 4) ? 6 : 1;
}

template <int C, typename TF, int kL>
__global__ void __launch_bounds__(kThreads, accum_min_blocks<C, kL>())
    k_accum(const __grid_constant__ LaunchCams cams, const __grid_constant__ PointArgs a) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const TF* feat = reinterpret_cast<const TF*>(cam.feat);
  const float* __restrict__ xyz = cam.xyz;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t em_next = (cam.early && i0 < cam.n) ? (uint32_t)__ldcs(cam.early + i0) : 0xFFu;
  for (int64_t i = i0; i < cam.n; i += S) {
    uint32_t mask = 0;  // bit l: the point is in Lambda of its layer-l pixel
    // the depth pass's mask first: a point that can pass at no layer costs
    // one byte read and its mask write, not its position (on the 120M-point
    // frame, where 70% of the points are outside the view, the pass went from
    // 583 to 528 us; in the 5M-point view the occluded points lie among the
    // visible ones, whose loads wait for the added round trip: 91.5 -> 92.8 us)
    const uint32_t em = em_next;
    // the next point's byte, one grid-stride step ahead: a point then waits
    // for one round trip (its position) instead of two (120M-point frame:
    // accumulate 512 -> 466 us; 16-camera training step 4.18 -> 3.83 ms of
    // accumulate passes)
    em_next = (cam.early && i + S < cam.n) ? (uint32_t)__ldcs(cam.early + i + S) : 0xFFu;
    if (em == 0u) {
      if (cam.vis) cam.vis[i] = 0u;
      continue;
    }
    // the forward's last reads of the position and descriptors are streamed
    // (evict-first), so that the pixel state keeps its place in L2 for the
    // key reads and atomics (1080p step -1 us, 120M-point frame -6 us)
    const float x0 = __ldcs(xyz + 3 * i), x1 = __ldcs(xyz + 3 * i + 1), x2 = __ldcs(xyz + 3 * i + 2);
    float X0, X1, X2, u0 = 0.0f, v0 = 0.0f, zd;
    transform(cam, x0, x1, x2, X0, X1, X2);
    if (camera(cam, X0, X1, X2, u0, v0, zd) && (zd > a.znear) && in_pyramid(u0, v0, cam.w, cam.h, a.levels) &&
        !(cam.normals && !normal_keep(cam, cam.normals, i, X0, X1, X2))) {
      const float rw = a.radius ? __ldg(a.radius + i) : 0.0f, bt = a.radius ? __ldg(a.beta + i) : 0.0f;
      int32_t pix[kL];  // pixel within layer l (< 2^28), -1: none
      uint32_t zb[kL];
#pragma unroll
      for (int l = 0; l < kL; ++l) {
        int32_t pu, pv;
        const bool keep = ((em >> l) & 1u) && l < a.levels && (!a.radius || discard_keep(cam, zd, rw, bt, a.g2, l));
        pix[l] = (keep && pixel_in(u0, v0, l, cam.w, cam.h, pu, pv)) ? pv * (cam.w >> l) + pu : -1;
      }
#pragma unroll
      for (int l = 0; l < kL; ++l)
        zb[l] = pix[l] >= 0 ? (uint32_t)(__ldg(cam.key[l] + pix[l]) >> 32) : 0u;
      float f[C];
      bool loaded = false;
#pragma unroll
      for (int l = 0; l < kL; ++l) {
        if (pix[l] < 0 || !(zd <= __fmul_rn(__uint_as_float(zb[l]), a.a1))) continue;
        if (!loaded) {
          load_feat_last<C, TF>(feat, i, f);
          if (a.log_desc) {
#pragma unroll
            for (int k = 0; k < C; ++k) f[k] = expf(f[k]);
          }
          loaded = true;
        }
        atomic_add_vec<C>(cam.acc + (cam.off[l] + pix[l]) * C, f);
        atomicAdd(cam.cnt[l] + pix[l], 1u);
        mask |= 1u << l;
      }
    }
    if (cam.vis) {
      uint32_t tile = 0;
      if (mask) {  // layer-0 screen tile of the point (position clamped to the image)
        const int32_t tu = min(max(__float2int_rn(u0), 0), cam.w - 1) >> kTileShift;
        const int32_t tv = min(max(__float2int_rn(v0), 0), cam.h - 1) >> kTileShift;
        tile = (uint32_t)(tv * cam.tiles_x + tu);
      }
      cam.vis[i] = (tile << 8) | mask;
    }
  }
}

// ---------------------------------------------------------------------------
// K3 normalise: I = sum / |Lambda| (Eq. blend), background where empty (k_env_fill
// writes the environment map's pixels),
// photometric epilogue on layer 0, cast to the output type, planar layout
// ---------------------------------------------------------------------------
template <int C, typename TO>
__global__ void __launch_bounds__(kThreads) k_normalize(const __grid_constant__ LaunchCams cams,
                                                        const __grid_constant__ PointArgs a) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const int64_t total = cam.off[a.levels];
  int lc = 0;  // the layer of g: g only grows, so its layer only advances
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    while (lc + 1 < a.levels && g >= cam.off[lc + 1]) ++lc;
    const int l = lc;
    TO* img = reinterpret_cast<TO*>(cam.image[l]);
    if (img == nullptr) continue;
    const int64_t p = g - cam.off[l];
    const int64_t np = cam.off[l + 1] - cam.off[l];
    // the count and the sums are loaded together: one round trip per pixel
    const uint32_t n = cam.cnt[l][p];
    float v[C];
    load_vec<C>(cam.acc + g * C, v);
    if (n == 0) {
      if (a.env) continue;  // the environment map's pixels: k_env_fill
#pragma unroll
      for (int k = 0; k < C; ++k) v[k] = a.background ? __ldg(a.background + k) : 0.0f;
    } else {  // one reciprocal per pixel (within 2 ulp of the quotient)
      const float rn = __frcp_rn((float)n);
#pragma unroll
      for (int k = 0; k < C; ++k) v[k] *= rn;
    }
    if (l == 0 && cam.epi) {
      const int32_t pu = (int32_t)(p % cam.w), pv = (int32_t)(p / cam.w);
#pragma unroll
      for (int k = 0; k < (C < 3 ? C : 3); ++k) v[k] = epilogue(cam, k, pu, pv, v[k], nullptr);
    }
#pragma unroll
    for (int k = 0; k < C; ++k) img[k * np + p] = from_f32<TO>(v[k]);
  }
}

int64_t most_pixels(const LaunchCams& cams, const PointArgs& a) {
  int64_t most = 0;
  for (int k = 0; k < a.ncam; ++k) most = cams.c[k].off[a.levels] > most ? cams.c[k].off[a.levels] : most;
  return most;
}

cudaError_t launch_clear(const LaunchCams& cams, const PointArgs& a, int c, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int64_t px = most_pixels(cams, a);
  ADOP_DISPATCH_C(c, e = launch_strided(k_clear<kC>, px, a.ncam, kPixelWaves, 0, s, cams, a));
  return e;
}

int64_t most_points(const LaunchCams& cams, const PointArgs& a) {
  int64_t most = 0;
  for (int k = 0; k < a.ncam; ++k) most = cams.c[k].n > most ? cams.c[k].n : most;
  return most;
}

cudaError_t launch_depth(const LaunchCams& cams, const PointArgs& a, cudaStream_t s) {
  const int64_t n = most_points(cams, a);
  if (n == 0) return cudaSuccess;
  if (a.levels <= 4) return launch_strided(k_depth<4>, n, a.ncam, kPointWaves, 0, s, cams, a);
  return launch_strided(k_depth<ADOP_MAX_LEVELS>, n, a.ncam, kPointWaves, 0, s, cams, a);
}

cudaError_t launch_accum(const LaunchCams& cams, const PointArgs& a, int c, adop_dtype fd, cudaStream_t s) {
  const int64_t n = most_points(cams, a);
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (a.levels <= 4) {
    ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(fd, TF, e = launch_strided(k_accum<kC, TF, 4>, n, a.ncam, kPointWaves, 0,
                                                                  s, cams, a)));
  } else {
    ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(fd, TF, e = launch_strided(k_accum<kC, TF, ADOP_MAX_LEVELS>, n, a.ncam,
                                                                  kPointWaves, 0, s, cams, a)));
  }
  return e;
}

cudaError_t launch_normalize(const LaunchCams& cams, const PointArgs& a, int c, adop_dtype od, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int64_t px = most_pixels(cams, a);
  ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(od, TO, e = launch_strided(k_normalize<kC, TO>, px, a.ncam, kPixelWaves, 0, s,
                                                                cams, a)));
  return e;
}

}  // namespace adop
