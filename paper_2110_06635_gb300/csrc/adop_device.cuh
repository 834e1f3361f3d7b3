// Device-side building blocks of the rasterizer: per-launch camera constants,
// the FP32 projection (Sec. 3.1, P_l = 2^-l C(Rx + t)), rounding to pixels
// (Eq. round, Eq. boundscheck), descriptor loads and vector atomics.
//
// The projection is written with explicit round-to-nearest intrinsics
// (__fmul_rn / __fadd_rn / __fdiv_rn) so that no multiply-add is contracted:
// every pixel and depth is the result of one fixed sequence of IEEE binary32
// operations, which keeps depth/index buffers reproducible bit for bit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/adop.h"

namespace adop {

constexpr int kMaxCamsPerLaunch = 16;
constexpr int kThreads = 256;
constexpr int kTileShift = 5;  // 32 x 32 pixel screen tiles for binning the backward's points

__host__ __device__ constexpr int32_t tiles_along(int32_t n) { return (n + (1 << kTileShift) - 1) >> kTileShift; }

// Everything a kernel needs to know about one camera, passed by value in the
// kernel's parameter space (uniform per block: blockIdx.y selects the camera).
struct DevCam {
  // the cloud this camera renders in the forward point passes (a launch of
  // the render entry points gives every camera the same cloud; a server
  // batch may mix its resident clouds)
  const float* xyz;
  const void* feat;
  const float* normals;  // non-NULL only when normal culling is on
  int64_t n;
  float R[9];
  float t[3];
  float fx, fy, cx, cy, k1, k2, k3, p1, p2;
  float ifx, ify;  // f32(1 / fx), f32(1 / fy) (the inverse camera)
  int32_t w, h;
  int32_t model;  // 0 pinhole + Brown-Conrady, 1 fisheye (stereographic)
  int64_t off[ADOP_MAX_LEVELS + 1];  // first pixel of each layer in the concatenated pyramid
  unsigned long long* key[ADOP_MAX_LEVELS];
  uint32_t* cnt[ADOP_MAX_LEVELS];
  void* image[ADOP_MAX_LEVELS];
  const float* grad[ADOP_MAX_LEVELS];
  float* acc;    // pixel-major FP32 sums, c floats per pixel
  float* info;   // backward: per pixel {z_min, 1/(1+|Lambda|) (1: empty), <G, I>, 1/|Lambda|}
  float* gpm;    // backward: upstream gradient, pixel-major, g_stride(c) floats per pixel
  uint32_t* vis;  // per point: layer mask (bits 0-7) | layer-0 screen tile << 8 (or NULL)
  uint8_t* early;  // per point: the layers where it may still pass the fuzzy test, written by the depth
                   // pass for the accumulate pass (NULL: not kept)
  // screen-tile binning of the visible points for the backward pass
  int32_t tiles_x, tiles;    // kTileShift-pixel tiles per row, total
  int32_t* bin_count;        // per tile: visible points (the scatter cursor of the path without a table)
  int32_t* bin_off;          // tiles + 1 exclusive offsets
  int32_t* bin_list;         // visible point indices, tile by tile (NULL: no binning)
  int32_t* bin_table;        // [block][tile]: a binning block's first slot within the tile's range
  int32_t bin_rows;          // binning blocks the table has rows for
  // photometric epilogue (Sec. 3.3); ev_scale = 2^-EV, computed on the host
  int32_t epi;
  int32_t leaky;  // training response curve (Eq. resonseleak) instead of clamping
  int32_t crf_n;
  float ev_scale;
  float wb[3];
  float vig_c[2];
  float vig_a[3];
  const float* crf;
  // environment map gradient: acc holds each empty pixel's sampled value
  // (the caller passed the forward's kept state)
  int32_t env_in_acc;
};

struct LaunchCams {
  DevCam c[kMaxCamsPerLaunch];
};

// Floats per pixel of the pixel-major upstream gradient: c, padded to a
// multiple of 4 from c = 3 on so that every pixel starts on 16 bytes.
__host__ __device__ constexpr int g_stride(int c) { return c <= 2 ? c : (c + 3) / 4 * 4; }

// L2 cache policies (createpolicy, sm_80+): data that other threads will read
// again soon (per-pixel records) is kept with evict_last; streamed per-point
// data uses evict_first so that it does not push the records out.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ float4 ld_keep(const float4* ptr, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(ptr), "l"(pol));
  return v;
}

// Load n floats (n a multiple of 4, 2, or 1) from a suitably aligned address.
template <int N>
__device__ __forceinline__ void load_vec(const float* __restrict__ src, float* dst) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int v = 0; v < N / 4; ++v) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(src) + v);
      dst[4 * v] = q.x; dst[4 * v + 1] = q.y; dst[4 * v + 2] = q.z; dst[4 * v + 3] = q.w;
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int v = 0; v < N / 2; ++v) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(src) + v);
      dst[2 * v] = q.x; dst[2 * v + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) dst[k] = __ldg(src + k);
  }
}

// Store n floats to a suitably aligned address with the widest vector stores.
template <int N>
__device__ __forceinline__ void store_vec(float* dst, const float* src) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int v = 0; v < N / 4; ++v)
      reinterpret_cast<float4*>(dst)[v] = make_float4(src[4 * v], src[4 * v + 1], src[4 * v + 2], src[4 * v + 3]);
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int v = 0; v < N / 2; ++v) reinterpret_cast<float2*>(dst)[v] = make_float2(src[2 * v], src[2 * v + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) dst[k] = src[k];
  }
}

// Store n floats to a 32-byte-aligned row: 256-bit stores when n is a
// multiple of 8 (sm_100+), else as store_vec.
template <int N>
__device__ __forceinline__ void store_row(float* dst, const float* src) {
  if constexpr (N % 8 == 0) {
#pragma unroll
    for (int v = 0; v < N / 8; ++v) {
      const float* q = src + 8 * v;
      asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                   :: "l"(dst + 8 * v), "f"(q[0]), "f"(q[1]), "f"(q[2]), "f"(q[3]), "f"(q[4]), "f"(q[5]), "f"(q[6]),
                      "f"(q[7]) : "memory");
    }
  } else {
    store_vec<N>(dst, src);
  }
}

// load_vec with the L2 policy on every 16-byte piece (scalar pieces: plain loads).
template <int N>
__device__ __forceinline__ void load_keep(const float* __restrict__ src, float* dst, uint64_t pol) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int v = 0; v < N / 4; ++v) {
      const float4 q = ld_keep(reinterpret_cast<const float4*>(src) + v, pol);
      dst[4 * v] = q.x; dst[4 * v + 1] = q.y; dst[4 * v + 2] = q.z; dst[4 * v + 3] = q.w;
    }
  } else {
    load_vec<N>(src, dst);
  }
}

// load_keep for rows whose start is 32-byte aligned: 256-bit loads (sm_100+)
// when N is a multiple of 8, so that a pixel's C = 8 gradient is one load.
template <int N>
__device__ __forceinline__ void load_keep_row(const float* __restrict__ src, float* dst, uint64_t pol) {
  if constexpr (N % 8 == 0) {
#pragma unroll
    for (int v = 0; v < N / 8; ++v) {
      float* d = dst + 8 * v;
      asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
          : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]), "=f"(d[6]), "=f"(d[7])
          : "l"(src + 8 * v), "l"(pol));
    }
  } else {
    load_keep<N>(src, dst, pol);
  }
}

// ---------------------------------------------------------------------------
// FP32 projection contract
// ---------------------------------------------------------------------------

__device__ __forceinline__ void transform(const DevCam& cam, float x0, float x1, float x2,
                                          float& X0, float& X1, float& X2) {
  X0 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(cam.R[0], x0), __fmul_rn(cam.R[1], x1)),
                           __fmul_rn(cam.R[2], x2)), cam.t[0]);
  X1 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(cam.R[3], x0), __fmul_rn(cam.R[4], x1)),
                           __fmul_rn(cam.R[5], x2)), cam.t[1]);
  X2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(cam.R[6], x0), __fmul_rn(cam.R[7], x1)),
                           __fmul_rn(cam.R[8], x2)), cam.t[2]);
}

// Camera model C: layer-0 pixel coordinates (u0, v0) of a camera-space point
// and its depth for the depth test -- z for the pinhole, the distance |X|
// for the fisheye (the paper's rule for a model without a z).  Returns false
// where the model is undefined (fisheye: the negative optical axis).
__device__ __forceinline__ bool camera(const DevCam& cam, float X0, float X1, float X2, float& u0, float& v0,
                                       float& depth) {
  if (cam.model == 1) {
    // stereographic: normalised radius 2 tan(theta/2) = 2 rho / (|X| + Z)
    const float d = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(X0, X0), __fmul_rn(X1, X1)), __fmul_rn(X2, X2)));
    const float s = __fadd_rn(d, X2);
    depth = d;
    if (!(s > 0.0f)) return false;
    const float a = __fdiv_rn(2.0f, s);
    const float xn = __fmul_rn(a, X0), yn = __fmul_rn(a, X1);
    const float r2 = __fadd_rn(__fmul_rn(xn, xn), __fmul_rn(yn, yn));
    const float dd = __fadd_rn(
        1.0f, __fmul_rn(r2, __fadd_rn(cam.k1, __fmul_rn(r2, __fadd_rn(cam.k2, __fmul_rn(r2, cam.k3))))));
    u0 = __fadd_rn(__fmul_rn(cam.fx, __fmul_rn(xn, dd)), cam.cx);
    v0 = __fadd_rn(__fmul_rn(cam.fy, __fmul_rn(yn, dd)), cam.cy);
    return true;
  }
  depth = X2;
  const float xn = __fdiv_rn(X0, X2);
  const float yn = __fdiv_rn(X1, X2);
  const float r2 = __fadd_rn(__fmul_rn(xn, xn), __fmul_rn(yn, yn));
  const float d = __fadd_rn(
      1.0f, __fmul_rn(r2, __fadd_rn(cam.k1, __fmul_rn(r2, __fadd_rn(cam.k2, __fmul_rn(r2, cam.k3))))));
  if (cam.p1 == 0.0f && cam.p2 == 0.0f) {
    // no tangential terms: they are exact zeros for finite inputs, and a
    // non-finite xn or yn fails the bounds test either way
    u0 = __fadd_rn(__fmul_rn(cam.fx, __fmul_rn(xn, d)), cam.cx);
    v0 = __fadd_rn(__fmul_rn(cam.fy, __fmul_rn(yn, d)), cam.cy);
    return true;
  }
  const float a = __fmul_rn(xn, yn);
  const float tx = __fadd_rn(__fmul_rn(__fmul_rn(2.0f, cam.p1), a),
                             __fmul_rn(cam.p2, __fadd_rn(r2, __fmul_rn(2.0f, __fmul_rn(xn, xn)))));
  const float ty = __fadd_rn(__fmul_rn(cam.p1, __fadd_rn(r2, __fmul_rn(2.0f, __fmul_rn(yn, yn)))),
                             __fmul_rn(__fmul_rn(2.0f, cam.p2), a));
  const float xd = __fadd_rn(__fmul_rn(xn, d), tx);
  const float yd = __fadd_rn(__fmul_rn(yn, d), ty);
  u0 = __fadd_rn(__fmul_rn(cam.fx, xd), cam.cx);
  v0 = __fadd_rn(__fmul_rn(cam.fy, yd), cam.cy);
  return true;
}

// Eq. normalculling as printed: keep iff (R n)^T (R x + t) > 0.
__device__ __forceinline__ bool normal_keep(const DevCam& cam, const float* nrm, int64_t i, float X0,
                                            float X1, float X2) {
  const float n0 = nrm[3 * i], n1 = nrm[3 * i + 1], n2 = nrm[3 * i + 2];
  const float r0 = __fadd_rn(__fadd_rn(__fmul_rn(cam.R[0], n0), __fmul_rn(cam.R[1], n1)), __fmul_rn(cam.R[2], n2));
  const float r1 = __fadd_rn(__fadd_rn(__fmul_rn(cam.R[3], n0), __fmul_rn(cam.R[4], n1)), __fmul_rn(cam.R[5], n2));
  const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(cam.R[6], n0), __fmul_rn(cam.R[7], n1)), __fmul_rn(cam.R[8], n2));
  const float dot = __fadd_rn(__fadd_rn(__fmul_rn(r0, X0), __fmul_rn(r1, X1)), __fmul_rn(r2, X2));
  return dot > 0.0f;
}

// Exact 2^-l.
__device__ __forceinline__ float layer_scale(int l) { return __int_as_float((127 - l) << 23); }

// Eq. round (nearest, ties to even) + Eq. boundscheck at layer l.  Coordinates
// outside ]-1, w_l + 1[ (and NaN) are rejected before the integer conversion.
__device__ __forceinline__ bool pixel_at(float u0, float v0, int l, int32_t w, int32_t h, int32_t& pu,
                                         int32_t& pv) {
  const int32_t wl = w >> l, hl = h >> l;
  const float s = layer_scale(l);
  const float ul = __fmul_rn(u0, s), vl = __fmul_rn(v0, s);
  if (!(ul > -1.0f && ul < __fadd_rn((float)wl, 1.0f))) return false;
  if (!(vl > -1.0f && vl < __fadd_rn((float)hl, 1.0f))) return false;
  pu = __float2int_rn(ul);
  pv = __float2int_rn(vl);
  return pu >= 0 && pu < wl && pv >= 0 && pv < hl;
}

// pixel_at for a position that passed in_pyramid: there |u0 2^-l| and
// |v0 2^-l| stay below 2^15, so the conversion cannot overflow, and a
// coordinate outside ]-1, w_l + 1[ rounds to a pixel outside [0, w_l): the
// integer test alone gives pixel_at's result.
__device__ __forceinline__ bool pixel_in(float u0, float v0, int l, int32_t w, int32_t h, int32_t& pu,
                                         int32_t& pv) {
  const float s = layer_scale(l);
  pu = __float2int_rn(__fmul_rn(u0, s));
  pv = __float2int_rn(__fmul_rn(v0, s));
  return (uint32_t)pu < (uint32_t)(w >> l) && (uint32_t)pv < (uint32_t)(h >> l);
}

// One test for all layers: false when (u0, v0) is out of bounds at every
// layer l < levels (u0 <= -2^(levels-1) or u0 >= w + 2^(levels-1) puts
// u0 2^-l outside ]-1, w_l + 1[ for each such l; likewise v), so pixel_at
// need not run four times for the many points outside the view.  Exact:
// it never rejects a point that some layer keeps.
__device__ __forceinline__ bool in_pyramid(float u0, float v0, int32_t w, int32_t h, int levels) {
  const float m = (float)(1 << (levels - 1));
  return u0 > -m && u0 < (float)w + m && v0 > -m && v0 < (float)h + m;
}

// Eq. discard (stochastic point discarding): keep the point at layer l iff
// (t * t) * g2 > 1 - beta, t = (f32(fx 2^-l) * r_world) / z, g2 = f32(gamma^2):
// the paper's r_screen / sqrt(1 - beta) > 1 / gamma without the square root,
// with r_screen = fx r_world / (z 2^l).  Fixed FP32 order, no contraction.
__device__ __forceinline__ bool discard_keep(const DevCam& cam, float z, float r, float beta, float g2, int l) {
  const float t = __fdiv_rn(__fmul_rn(__fmul_rn(cam.fx, layer_scale(l)), r), z);
  return __fmul_rn(__fmul_rn(t, t), g2) > __fsub_rn(1.0f, beta);
}

__device__ __forceinline__ unsigned long long depth_key(float z, int64_t i) {
  return ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)(uint32_t)i;
}

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Load the C descriptors of point i (row-major n x C) as FP32, with the widest
// aligned vector loads the row size allows (rows start 16-byte aligned when
// C * sizeof(T) is a multiple of 16).
template <int C, typename T>
__device__ __forceinline__ void load_feat(const T* __restrict__ feat, int64_t i, float (&f)[C]) {
  constexpr int kBytes = C * (int)sizeof(T);
  const T* row = feat + i * C;
  if constexpr (kBytes % 16 == 0) {
    constexpr int kVec = kBytes / 16;
    constexpr int kPer = 16 / (int)sizeof(T);
#pragma unroll
    for (int v = 0; v < kVec; ++v) {
      uint4 raw = __ldg(reinterpret_cast<const uint4*>(row) + v);
      const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
      for (int k = 0; k < kPer; ++k) f[v * kPer + k] = to_f32<T>(e[k]);
    }
  } else if constexpr (kBytes % 8 == 0) {
    constexpr int kVec = kBytes / 8;
    constexpr int kPer = 8 / (int)sizeof(T);
#pragma unroll
    for (int v = 0; v < kVec; ++v) {
      uint2 raw = __ldg(reinterpret_cast<const uint2*>(row) + v);
      const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
      for (int k = 0; k < kPer; ++k) f[v * kPer + k] = to_f32<T>(e[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < C; ++k) f[k] = to_f32<T>(row[k]);
  }
}

// load_feat with streaming loads (evict-first), for a last read.
template <int C, typename T>
__device__ __forceinline__ void load_feat_last(const T* __restrict__ feat, int64_t i, float (&f)[C]) {
  constexpr int kBytes = C * (int)sizeof(T);
  const T* row = feat + i * C;
  if constexpr (kBytes % 16 == 0) {
    constexpr int kVec = kBytes / 16;
    constexpr int kPer = 16 / (int)sizeof(T);
#pragma unroll
    for (int v = 0; v < kVec; ++v) {
      uint4 raw = __ldcs(reinterpret_cast<const uint4*>(row) + v);
      const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
      for (int k = 0; k < kPer; ++k) f[v * kPer + k] = to_f32<T>(e[k]);
    }
  } else {
    load_feat<C, T>(feat, i, f);
  }
}

// The descriptors of point i as linear FP32 values: stored values, or exp of
// them for logarithmic descriptors (converted during rasterization, Sec. 3.2).
template <int C, typename T>
__device__ __forceinline__ void load_desc(const T* __restrict__ feat, int64_t i, bool log_desc, float (&f)[C]) {
  load_feat<C, T>(feat, i, f);
  if (log_desc) {
#pragma unroll
    for (int k = 0; k < C; ++k) f[k] = expf(f[k]);
  }
}

// acc[0..C) += f (FP32), as few global atomics as the alignment allows
// (sm_90+ has float2/float4 vector atomics on global memory).
template <int C>
__device__ __forceinline__ void atomic_add_vec(float* a, const float (&f)[C]) {
  if constexpr (C % 4 == 0) {
#pragma unroll
    for (int v = 0; v < C / 4; ++v)
      atomicAdd(reinterpret_cast<float4*>(a) + v, make_float4(f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]));
  } else if constexpr (C % 2 == 0) {
#pragma unroll
    for (int v = 0; v < C / 2; ++v) atomicAdd(reinterpret_cast<float2*>(a) + v, make_float2(f[2 * v], f[2 * v + 1]));
  } else {
#pragma unroll
    for (int k = 0; k < C; ++k) atomicAdd(a + k, f[k]);
  }
}

// Programmatic dependent launch (sm_90+).  Every kernel that the library
// launches with launch_pdl() calls this before its first memory access.  The
// wait returns once the grids before it in the stream have completed and
// their writes are visible, so the body runs exactly in stream order; the
// trigger after it lets the next grid's blocks be placed on SMs as this grid's
// last blocks retire (they wait in the same call), which hides the launch
// latency between the kernels of a step.  Without a programmatic predecessor
// both instructions do nothing.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Layer of a pixel index g in [0, off[levels]).
__device__ __forceinline__ int layer_of(const DevCam& cam, int levels, int64_t g) {
  int l = 0;
#pragma unroll
  for (int k = 1; k < ADOP_MAX_LEVELS; ++k)
    if (k < levels && g >= cam.off[k]) l = k;
  return l;
}

// Response curve of channel ch at x (Sec. 3.3): the LUT of crf_n samples on
// [0,1] with linear interpolation, the input clamped to [0,1] -- or, in
// training (cam.leaky), leaking outside it as in Eq. resonseleak with
// alpha = 0.01 -- and the identity without a LUT.  *slope = dR/dx; *seg and
// *frac: the LUT segment and the weight of its upper sample (seg = -1: no LUT
// sample is used).
__device__ __forceinline__ float response(const DevCam& cam, int ch, float x, float* slope, int* seg, float* frac) {
  *seg = -1;
  *frac = 0.0f;
  if (cam.crf == nullptr || cam.crf_n < 2) {
    *slope = 1.0f;
    return x;
  }
  constexpr float kLeak = 0.01f;
  if (cam.leaky && x < 0.0f) {
    *slope = kLeak;
    return kLeak * x;
  }
  if (cam.leaky && x > 1.0f) {
    const float rs = rsqrtf(x);
    *slope = 0.5f * kLeak * rs / x;
    return -kLeak * rs + kLeak + 1.0f;
  }
  const int n = cam.crf_n;
  const float xc = fminf(fmaxf(x, 0.0f), 1.0f);
  const float pos = xc * (float)(n - 1);
  const int i0 = min((int)floorf(pos), n - 2);
  const float fr = pos - (float)i0;
  const float* lut = cam.crf + ch * n;
  const float lo = __ldg(lut + i0), hi = __ldg(lut + i0 + 1);
  *seg = i0;
  *frac = fr;
  *slope = (x < 0.0f || x > 1.0f) ? 0.0f : (hi - lo) * (float)(n - 1);
  return lo * (1.0f - fr) + hi * fr;
}

// Photometric model of Sec. 3.3 on one value of channel ch at layer-0 pixel
// (u, v): exposure 2^-EV, white balance, vignette 1 + a2 r^2 + a4 r^4 + a6 r^6
// with r = |(u/w, v/h) - c_v|, then the response curve.  If dydx is given it
// receives d out / d in.
__device__ __forceinline__ float epilogue(const DevCam& cam, int ch, int32_t u, int32_t v, float x,
                                          float* dydx) {
  const float ru = __fdiv_rn((float)u, (float)cam.w) - cam.vig_c[0];
  const float rv = __fdiv_rn((float)v, (float)cam.h) - cam.vig_c[1];
  const float r2 = ru * ru + rv * rv;
  const float vig = 1.0f + r2 * (cam.vig_a[0] + r2 * (cam.vig_a[1] + r2 * cam.vig_a[2]));
  const float scale = cam.ev_scale * cam.wb[ch] * vig;
  float slope, frac;
  int seg;
  const float y = response(cam, ch, x * scale, &slope, &seg, &frac);
  if (dydx) *dydx = slope * scale;
  return y;
}

// ---------------------------------------------------------------------------
// environment map (Sec. 3.1): the value of a pixel where no point lands
// ---------------------------------------------------------------------------

constexpr int kInvertSteps = 20;  // fixed-point / Newton steps of the inverse camera

// Newton steps on r radial(r^2) = r_d, radial(s) = 1 + s (k1 + s (k2 + s k3)):
// the undistorted normalised radius of a distorted one (both camera models
// share the radial polynomial).  Converges in a few steps for the moderate
// distortion of calibrated lenses; stops when a step is below 1e-7 r.
__device__ __forceinline__ float undistort_radius(const DevCam& cam, float rd) {
  float r = rd;
  for (int it = 0; it < kInvertSteps; ++it) {
    const float r2 = r * r;
    const float f = r * (1.0f + r2 * (cam.k1 + r2 * (cam.k2 + r2 * cam.k3))) - rd;
    const float fp = 1.0f + r2 * (3.0f * cam.k1 + r2 * (5.0f * cam.k2 + r2 * 7.0f * cam.k3));
    const float step = __fdividef(f, fp);
    r -= step;
    if (!(fabsf(step) > 1e-7f * r)) break;
  }
  return r;
}

// Inverse camera model C^-1: the unit camera-space direction of the ray
// through layer-0 pixel coordinates (u0, v0).  Radial distortion only (the
// fisheye, and the pinhole with p1 = p2 = 0): Newton on the radius; with
// tangential terms, fixed-point steps (xn, yn) <- ((xd, yd) -
// tangential(xn, yn)) / radial(xn, yn), which contract for the moderate
// distortion of calibrated lenses.  The fisheye then inverts the
// stereographic map, (xn, yn) -> (4 xn, 4 yn, 4 - r^2) / (4 + r^2).  FP32.
__device__ __forceinline__ void camera_inverse(const DevCam& cam, float u0, float v0, float (&d)[3]) {
  const float xd = (u0 - cam.cx) * cam.ifx, yd = (v0 - cam.cy) * cam.ify;
  float xn = xd, yn = yd;
  if (cam.model == 1 || (cam.p1 == 0.0f && cam.p2 == 0.0f)) {
    const float rd = sqrtf(xd * xd + yd * yd);
    const float s = rd > 0.0f ? __fdividef(undistort_radius(cam, rd), rd) : 1.0f;
    xn = xd * s;
    yn = yd * s;
  } else {
    for (int it = 0; it < kInvertSteps; ++it) {
      const float r2 = xn * xn + yn * yn;
      const float rad = 1.0f + r2 * (cam.k1 + r2 * (cam.k2 + r2 * cam.k3));
      const float tx = 2.0f * cam.p1 * xn * yn + cam.p2 * (r2 + 2.0f * xn * xn);
      const float ty = cam.p1 * (r2 + 2.0f * yn * yn) + 2.0f * cam.p2 * xn * yn;
      const float inv = __fdividef(1.0f, rad);
      const float nx = (xd - tx) * inv, ny = (yd - ty) * inv;
      const bool still = fabsf(nx - xn) + fabsf(ny - yn) > 1e-7f * (fabsf(nx) + fabsf(ny) + 1e-3f);
      xn = nx;
      yn = ny;
      if (!still) break;
    }
  }
  if (cam.model == 1) {
    const float r2 = xn * xn + yn * yn;
    const float inv = __fdividef(1.0f, 4.0f + r2);
    d[0] = 4.0f * xn * inv;
    d[1] = 4.0f * yn * inv;
    d[2] = (4.0f - r2) * inv;
    return;
  }
  const float inv = rsqrtf(xn * xn + yn * yn + 1.0f);
  d[0] = xn * inv;
  d[1] = yn * inv;
  d[2] = inv;
}

// The four texels (indices into one env_h x env_w plane) and bilinear
// weights that layer-l pixel (pu, pv) samples: world direction
// R^T C^-1(pu 2^l, pv 2^l), longitude atan2(d_x, d_z) and colatitude
// acos(d_y) mapped to texel coordinates with centres at integers; longitude
// wraps, colatitude clamps.  Every index is in range whatever the inputs.
struct EnvTaps {
  int32_t t[4];
  float w[4];
};

__device__ __forceinline__ EnvTaps env_taps(const DevCam& cam, int32_t ew, int32_t eh, int l, int32_t pu,
                                            int32_t pv) {
  constexpr float kPi = 3.14159265358979323846f;
  float dc[3];
  camera_inverse(cam, (float)(pu << l), (float)(pv << l), dc);
  const float dx = cam.R[0] * dc[0] + cam.R[3] * dc[1] + cam.R[6] * dc[2];
  const float dy = cam.R[1] * dc[0] + cam.R[4] * dc[1] + cam.R[7] * dc[2];
  const float dz = cam.R[2] * dc[0] + cam.R[5] * dc[1] + cam.R[8] * dc[2];
  const float phi = atan2f(dx, dz);
  const float theta = acosf(fminf(fmaxf(dy, -1.0f), 1.0f));
  const float ue = (phi + kPi) * ((float)ew * (0.5f / kPi)) - 0.5f;
  const float ve = theta * ((float)eh / kPi) - 0.5f;
  const float fu0 = floorf(ue), fv0 = floorf(ve);
  const float fu = ue - fu0, fv = ve - fv0;
  const int32_t iu0 = (int32_t)fu0, iv0 = (int32_t)fv0;
  // longitude lies in [-pi, pi], so iu0 is in [-1, ew - 1] up to rounding;
  // the clamp keeps a NaN direction in range too
  int32_t ua = iu0 < 0 ? iu0 + ew : iu0;
  ua = ua >= ew ? ua - ew : ua;
  ua = min(max(ua, 0), ew - 1);
  const int32_t ub = ua + 1 == ew ? 0 : ua + 1;
  const int32_t va = min(max(iv0, 0), eh - 1), vb = min(max(iv0 + 1, 0), eh - 1);
  EnvTaps e;
  e.t[0] = va * ew + ua;
  e.t[1] = va * ew + ub;
  e.t[2] = vb * ew + ua;
  e.t[3] = vb * ew + ub;
  e.w[0] = (1.0f - fu) * (1.0f - fv);
  e.w[1] = fu * (1.0f - fv);
  e.w[2] = (1.0f - fu) * fv;
  e.w[3] = fu * fv;
  return e;
}

// Bilinear sample of the C channels of a texel-major map (texel t's C
// floats at env + t C) at the taps.
template <int C>
__device__ __forceinline__ void env_sample(const float* __restrict__ env, const EnvTaps& e, float (&v)[C]) {
#pragma unroll
  for (int k = 0; k < C; ++k) v[k] = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float tx[C];
    load_vec<C>(env + (int64_t)e.t[j] * C, tx);
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = fmaf(e.w[j], tx[k], v[k]);
  }
}

}  // namespace adop
