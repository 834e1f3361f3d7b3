// Backward pass of the one-pixel point rasterizer (Sec. 3.1, "Backward
// Pass"): feature gradients, the approximate one-pixel spatial gradient
// (Eqs. induce, gradp, spatialderiv) and the chain rule to positions, the
// SE(3) tangent of the pose (Eq. tangent) and the intrinsics (Eq. partial).
//
//   k_bwd_prepass  one thread per pixel: packs what a point needs to know
//                  about a pixel -- min depth, |Lambda|, <G, I> in one 16-byte
//                  record, and the (epilogue-chained) upstream gradient G
//                  pixel-major -- so that the pixels a point visits cost one
//                  16-byte read each, plus one contiguous G read only where
//                  the induced change is non-zero.
//   k_bwd_points   one thread per point and camera: visits, in every layer
//                  where the accumulate pass recorded the point in Lambda, its
//                  pixel and the 4 neighbours; writes its own dL/dtau and
//                  dL/dx (owner computes: no atomics for one camera), and
//                  reduces pose/intrinsic terms warp -> block into per-block
//                  partial sums.
//   k_bwd_items    the same when the forward recorded each point's layer
//                  mask: warps compact their (point, layer) pairs in shared
//                  memory and process them densely; with binning, the
//                  visible points are visited 32x32-pixel screen tile by
//                  tile, so the pixel records a warp reads stay in cache,
//                  and (gradients assigned) the points in no Lambda get
//                  their zero gradients after the pairs.
//   k_bin_*        count the visible points per screen tile, scan, scatter
//                  their indices tile by tile.
//   k_bwd_reduce   sums the block partials in a fixed order (no float atomics
//                  across blocks; the partials themselves follow the order in
//                  which the binning lists the points).
#include <cuda_runtime.h>

#include "launch.h"

namespace adop {

template <int C, typename TG>
__global__ void __launch_bounds__(kThreads) k_bwd_prepass(const __grid_constant__ LaunchCams cams,
                                                          const __grid_constant__ PointArgs a) {
  pdl_entry();
  constexpr int GS = g_stride(C);
  const DevCam& cam = cams.c[blockIdx.y];
  const int64_t total = cam.off[a.levels];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int l = layer_of(cam, a.levels, g);
    const int64_t p = g - cam.off[l];
    const int64_t np = cam.off[l + 1] - cam.off[l];
    // every load up front, independent of the count: one round trip per pixel
    const uint32_t n = cam.cnt[l][p];
    const unsigned long long key = cam.key[l][p];
    float I[C], G[GS];
    load_vec<C>(cam.acc + g * C, I);
    const TG* gl = reinterpret_cast<const TG*>(cam.grad[l]);  // stored as TG, widened to FP32
#pragma unroll
    for (int k = 0; k < C; ++k) G[k] = gl ? to_f32<TG>(gl[k * np + p]) : 0.0f;
    if (n == 0 && !a.env) {
#pragma unroll
      for (int k = 0; k < C; ++k) I[k] = a.background ? __ldg(a.background + k) : 0.0f;
    }
    // one reciprocal per pixel (within 2 ulp of the quotient); 0 for an empty pixel
    const float rn = n != 0 ? __frcp_rn((float)n) : 0.0f;
    if (n != 0) {  // (an empty pixel's acc holds the environment map's value, kept by k_env_fill)
#pragma unroll
      for (int k = 0; k < C; ++k) I[k] *= rn;
    }
#pragma unroll
    for (int k = C; k < GS; ++k) G[k] = 0.0f;
    if (l == 0 && cam.epi) {
      const int32_t pu = (int32_t)(p % cam.w), pv = (int32_t)(p / cam.w);
#pragma unroll
      for (int k = 0; k < (C < 3 ? C : 3); ++k) {
        float d;
        epilogue(cam, k, pu, pv, I[k], &d);
        G[k] *= d;
      }
    }
    float gi = 0.0f;
#pragma unroll
    for (int k = 0; k < C; ++k) gi = fmaf(G[k], I[k], gi);
    // the reciprocals that the point pass needs, computed once here: 1/(1+|Lambda|)
    // for a neighbour's joins-the-blend case (exactly 1 for an empty pixel, at
    // most 1/2 otherwise) and 1/|Lambda| for the feature gradient
    reinterpret_cast<float4*>(cam.info)[g] =
        make_float4(__uint_as_float((uint32_t)(key >> 32)), __frcp_rn(1.0f + (float)n), gi, rn);
    store_row<GS>(cam.gpm + g * GS, G);  // (rows of GS floats in a 256-byte-aligned workspace block)
  }
}

// Chain rule from the layer-0 pixel gradient (du0, dv0) to the camera-space
// point, the pose tangent (left increment exp(xi)(R,t): dX/dnu = I,
// dX/domega = -[X]x), the intrinsics (fx, fy, cx, cy, k1, k2) and the world
// position (dL/dx = R^T dL/dX).  FP32.
__device__ __forceinline__ void chain_rule(const DevCam& cam, float X0, float X1, float X2, float du0, float dv0,
                                           float (&red)[12], float (&gx)[3]) {
  if (cam.model == 1) {
    // fisheye (stereographic): a = 2 / (|X| + Z), (xn, yn) = a (X, Y)
    const float d = sqrtf(X0 * X0 + X1 * X1 + X2 * X2);
    const float s = d + X2;
    const float a = 2.0f / s;
    const float xn = a * X0, yn = a * X1;
    const float r2 = xn * xn + yn * yn;
    const float dd = 1.0f + r2 * (cam.k1 + r2 * (cam.k2 + r2 * cam.k3));
    const float ddr = cam.k1 + r2 * (2.0f * cam.k2 + 3.0f * cam.k3 * r2);
    const float gxd = cam.fx * du0, gyd = cam.fy * dv0;
    // through (xd, yd) = (xn, yn) dd(r2)
    const float gxn = gxd * (dd + 2.0f * xn * xn * ddr) + gyd * (2.0f * xn * yn * ddr);
    const float gyn = gxd * (2.0f * xn * yn * ddr) + gyd * (dd + 2.0f * yn * yn * ddr);
    // (xn, yn) = a (X0, X1), da/dX = -2/s^2 (X/d + e_z)
    const float c = -2.0f / (s * s) * (gxn * X0 + gyn * X1);
    const float dX0 = gxn * a + c * X0 / d, dX1 = gyn * a + c * X1 / d, dX2 = c * (X2 / d + 1.0f);
    red[0] += dX0;
    red[1] += dX1;
    red[2] += dX2;
    red[3] += X1 * dX2 - X2 * dX1;
    red[4] += X2 * dX0 - X0 * dX2;
    red[5] += X0 * dX1 - X1 * dX0;
    red[6] += du0 * xn * dd;
    red[7] += dv0 * yn * dd;
    red[8] += du0;
    red[9] += dv0;
    red[10] += (gxd * xn + gyd * yn) * r2;
    red[11] += (gxd * xn + gyd * yn) * r2 * r2;
    gx[0] = cam.R[0] * dX0 + cam.R[3] * dX1 + cam.R[6] * dX2;
    gx[1] = cam.R[1] * dX0 + cam.R[4] * dX1 + cam.R[7] * dX2;
    gx[2] = cam.R[2] * dX0 + cam.R[5] * dX1 + cam.R[8] * dX2;
    return;
  }
  const float iz = 1.0f / X2;
  const float xn = X0 * iz, yn = X1 * iz;
  const float r2 = xn * xn + yn * yn;
  const float d = 1.0f + r2 * (cam.k1 + r2 * (cam.k2 + r2 * cam.k3));
  const float dd = cam.k1 + r2 * (2.0f * cam.k2 + 3.0f * cam.k3 * r2);
  const float xd = xn * d + 2.0f * cam.p1 * xn * yn + cam.p2 * (r2 + 2.0f * xn * xn);
  const float yd = yn * d + cam.p1 * (r2 + 2.0f * yn * yn) + 2.0f * cam.p2 * xn * yn;
  const float cross = 2.0f * xn * yn * dd + 2.0f * cam.p1 * xn + 2.0f * cam.p2 * yn;
  const float dxd_dxn = d + 2.0f * xn * xn * dd + 2.0f * cam.p1 * yn + 6.0f * cam.p2 * xn;
  const float dyd_dyn = d + 2.0f * yn * yn * dd + 6.0f * cam.p1 * yn + 2.0f * cam.p2 * xn;
  const float gxd = cam.fx * du0, gyd = cam.fy * dv0;
  const float gxn = gxd * dxd_dxn + gyd * cross;
  const float gyn = gxd * cross + gyd * dyd_dyn;
  const float dX0 = gxn * iz, dX1 = gyn * iz, dX2 = -(gxn * xn + gyn * yn) * iz;
  red[0] += dX0;
  red[1] += dX1;
  red[2] += dX2;
  red[3] += X1 * dX2 - X2 * dX1;
  red[4] += X2 * dX0 - X0 * dX2;
  red[5] += X0 * dX1 - X1 * dX0;
  red[6] += du0 * xd;
  red[7] += dv0 * yd;
  red[8] += du0;
  red[9] += dv0;
  red[10] += (gxd * xn + gyd * yn) * r2;
  red[11] += (gxd * xn + gyd * yn) * r2 * r2;
  gx[0] = cam.R[0] * dX0 + cam.R[3] * dX1 + cam.R[6] * dX2;
  gx[1] = cam.R[1] * dX0 + cam.R[4] * dX1 + cam.R[7] * dX2;
  gx[2] = cam.R[2] * dX0 + cam.R[5] * dX1 + cam.R[8] * dX2;
}

// One dL/dtau row of C values rounded once to the 16-bit type T, with the
// widest stores the row allows (16-byte aligned rows).
template <int C, typename T>
__device__ __forceinline__ void store_row16(float* grad_feat, int64_t i, const float (&gf)[C]) {
  T* dst = reinterpret_cast<T*>(grad_feat) + i * C;
  if constexpr (C % 8 == 0) {
#pragma unroll
    for (int v = 0; v < C / 8; ++v) {
      uint4 w;
      T* e = reinterpret_cast<T*>(&w);
#pragma unroll
      for (int k = 0; k < 8; ++k) e[k] = from_f32<T>(gf[8 * v + k]);
      __stcs(reinterpret_cast<uint4*>(dst) + v, w);
    }
  } else if constexpr (C % 4 == 0) {
    uint2 w;
    T* e = reinterpret_cast<T*>(&w);
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = from_f32<T>(gf[k]);
    __stcs(reinterpret_cast<uint2*>(dst), w);
  } else {
#pragma unroll
    for (int k = 0; k < C; ++k) dst[k] = from_f32<T>(gf[k]);
  }
}

// Write one point's dL/dtau and dL/dx: overwrite (streaming stores, dL/dtau
// in FP32 or rounded to b.feat_out), accumulate (owner computes) or add
// atomically (several cameras).
template <int C>
__device__ __forceinline__ void write_point_grads(const BwdArgs& b, int64_t i, const float (&gf)[C],
                                                  const float (&gx)[3], bool touched) {
  if (b.mode == kGradAssign) {
    if (b.grad_feat && b.feat_out == ADOP_BF16) {
      store_row16<C, __nv_bfloat16>(b.grad_feat, i, gf);
    } else if (b.grad_feat && b.feat_out == ADOP_F16) {
      store_row16<C, __half>(b.grad_feat, i, gf);
    } else if (b.grad_feat) {
      float* dst = b.grad_feat + i * C;
      if constexpr (C % 4 == 0) {
#pragma unroll
        for (int v = 0; v < C / 4; ++v)
          __stcs(reinterpret_cast<float4*>(dst) + v, make_float4(gf[4 * v], gf[4 * v + 1], gf[4 * v + 2], gf[4 * v + 3]));
      } else {
#pragma unroll
        for (int k = 0; k < C; ++k) __stcs(dst + k, gf[k]);
      }
    }
    if (b.grad_xyz) {
      __stcs(b.grad_xyz + 3 * i, gx[0]);
      __stcs(b.grad_xyz + 3 * i + 1, gx[1]);
      __stcs(b.grad_xyz + 3 * i + 2, gx[2]);
    }
  } else if (touched) {
    if (b.mode == kGradAccumulate) {
      if (b.grad_feat) {
        float* dst = b.grad_feat + i * C;
#pragma unroll
        for (int k = 0; k < C; ++k) dst[k] += gf[k];
      }
      if (b.grad_xyz) {
        b.grad_xyz[3 * i] += gx[0];
        b.grad_xyz[3 * i + 1] += gx[1];
        b.grad_xyz[3 * i + 2] += gx[2];
      }
    } else {
      if (b.grad_feat) atomic_add_vec<C>(b.grad_feat + i * C, gf);
      if (b.grad_xyz) {
        atomicAdd(b.grad_xyz + 3 * i, gx[0]);
        atomicAdd(b.grad_xyz + 3 * i + 1, gx[1]);
        atomicAdd(b.grad_xyz + 3 * i + 2, gx[2]);
      }
    }
  }
}

// Pose / intrinsics terms: warp shuffle -> shared memory -> one partial per block.
__device__ __forceinline__ void block_partials(const BwdArgs& b, float (&red)[12]) {
  __shared__ float sm[kThreads / 32][12];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    float v = red[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    float v = 0.0f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) v += sm[w][threadIdx.x];
    b.partials[((int64_t)blockIdx.y * 12 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
}

// Eq. spatialderiv at the 4 neighbours (+u, -u, +v, -v) of pixel (pu, pv) of a
// layer whose records start at `base`, contracted with the upstream gradient
// there; returns the layer-pixel gradients g_u, g_v of Eq. gradp.
template <int C>
__device__ __forceinline__ void spatial_grad(const DevCam& cam, const float4* __restrict__ info, int64_t base,
                                             int32_t pu, int32_t pv, int32_t wl, int32_t hl, float z, float a1,
                                             const float* tau, float& g_u, float& g_v, uint64_t pol) {
  constexpr int GS = g_stride(C);
  float cq[4];
  float4 iq[4];
  int64_t gq[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {  // issue the 4 record loads together
    const int32_t qu = pu + (s == 0 ? 1 : (s == 1 ? -1 : 0));
    const int32_t qv = pv + (s == 2 ? 1 : (s == 3 ? -1 : 0));
    gq[s] = (qu < 0 || qu >= wl || qv < 0 || qv >= hl) ? -1 : base + (int64_t)qv * wl + qu;
    iq[s] = gq[s] >= 0 ? ld_keep(info + gq[s], pol) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    cq[s] = 0.0f;
    if (gq[s] < 0) continue;
    float wgt;
    if (iq[s].y == 1.0f) wgt = 1.0f;                            // empty: 1/(1+0) = 1, overwrite
    else if (z > __fmul_rn(iq[s].x, a1)) wgt = 0.0f;            // behind the target surface
    else if (__fmul_rn(z, a1) < iq[s].x) wgt = 1.0f;            // in front: replaces the mean
    else wgt = iq[s].y;                                          // joins the fuzzy blend: 1/(1+|Lambda|)
    if (wgt == 0.0f) continue;
    float G[GS];
    load_keep_row<GS>(cam.gpm + gq[s] * GS, G, pol);
    float dot = 0.0f;
#pragma unroll
    for (int k = 0; k < C; ++k) dot = fmaf(G[k], tau[k], dot);
    cq[s] = wgt * (dot - iq[s].z);
  }
  g_u = 0.5f * (cq[0] - cq[1]);
  g_v = 0.5f * (cq[2] - cq[3]);
}

template <int C, typename TF>
__global__ void __launch_bounds__(kThreads, 4) k_bwd_points(const __grid_constant__ LaunchCams cams,
                                                            const __grid_constant__ PointArgs a,
                                                            const __grid_constant__ BwdArgs b) {
  pdl_entry();
  constexpr int GS = g_stride(C);
  const DevCam& cam = cams.c[blockIdx.y];
  const TF* feat = reinterpret_cast<const TF*>(a.feat);
  const float4* info = reinterpret_cast<const float4*>(cam.info);
  const bool spatial_out = b.grad_xyz != nullptr || b.partials != nullptr;
  const uint64_t pol = policy_evict_last();
  float red[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) red[k] = 0.0f;

  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    float gf[C];
#pragma unroll
    for (int k = 0; k < C; ++k) gf[k] = 0.0f;
    float gx[3] = {0.0f, 0.0f, 0.0f};
    bool touched = false;
    // layers in which the point is in Lambda of its pixel, as recorded by the
    // accumulate pass; without the record every in-bounds layer is examined
    const uint32_t vmask = cam.vis ? (cam.vis[i] & 0xFFu) : 0xFFu;
    if (vmask != 0u || b.all_projected) {
      float X0, X1, X2, u0 = 0.0f, v0 = 0.0f, zd;
      transform(cam, __ldg(a.xyz + 3 * i), __ldg(a.xyz + 3 * i + 1), __ldg(a.xyz + 3 * i + 2), X0, X1, X2);
      const bool valid = camera(cam, X0, X1, X2, u0, v0, zd) && (zd > a.znear) &&
                         !(a.normals && !normal_keep(cam, a.normals, i, X0, X1, X2));
      if (valid) {
        float tau[C];
        bool loaded = false;
        float du0 = 0.0f, dv0 = 0.0f;
        bool spatial = false;
        const float rw = a.radius ? __ldg(a.radius + i) : 0.0f, bt = a.radius ? __ldg(a.beta + i) : 0.0f;
        for (int l = 0; l < a.levels; ++l) {
          if (!((vmask >> l) & 1u) && !b.all_projected) continue;
          if (a.radius && !discard_keep(cam, zd, rw, bt, a.g2, l)) continue;
          int32_t pu, pv;
          if (!pixel_at(u0, v0, l, cam.w, cam.h, pu, pv)) continue;
          const int32_t wl = cam.w >> l, hl = cam.h >> l;
          const int64_t base = cam.off[l];
          const int64_t gp = base + (int64_t)pv * wl + pu;
          const float4 ip = __ldg(info + gp);
          const bool vis = cam.vis ? (((vmask >> l) & 1u) != 0u) : (zd <= __fmul_rn(ip.x, a.a1));
          if (vis) {
            // dI(p)/dtau_i = 1/|Lambda(p)| for every member of Lambda(p)
            float G[GS];
            load_vec<GS>(cam.gpm + gp * GS, G);
#pragma unroll
            for (int k = 0; k < C; ++k) gf[k] += G[k] * ip.w;  // ip.w = f32(1/|Lambda|)
            touched = true;
          }
          if (!(vis || b.all_projected) || !spatial_out) continue;
          if (!loaded) {
            load_desc<C, TF>(feat, i, a.log_desc, tau);
            loaded = true;
          }
          float g_u, g_v;
          spatial_grad<C>(cam, info, base, pu, pv, wl, hl, zd, a.a1, tau, g_u, g_v, pol);
          const float sc = layer_scale(l);
          du0 = fmaf(g_u, sc, du0);
          dv0 = fmaf(g_v, sc, dv0);
          spatial = true;
        }
        if (spatial && (du0 != 0.0f || dv0 != 0.0f)) {
          chain_rule(cam, X0, X1, X2, du0, dv0, red, gx);
          touched = true;
        }
        if (a.log_desc && touched) {  // d exp(tau) / d tau = exp(tau)
          if (!loaded) load_desc<C, TF>(feat, i, true, tau);
#pragma unroll
          for (int k = 0; k < C; ++k) gf[k] *= tau[k];
        }
      }
    }

    write_point_grads<C>(b, i, gf, gx, touched);
  }
  if (b.partials != nullptr) block_partials(b, red);
}

// Eq. spatialderiv for records already loaded (iq[s], -1 in gq[s]: no
// neighbour).  The rows of the neighbours with a non-zero weight are read
// 16 bytes at a time for all four together, so that their misses overlap
// (the second half of a row then hits L1); each dot product keeps the order
// k = 0 .. C-1.
template <int C>
__device__ __forceinline__ void spatial_grad_loaded(const DevCam& cam, const float4 (&iq)[4], const int32_t (&gq)[4],
                                                    float z, float a1, const float* tau, float& g_u, float& g_v,
                                                    uint64_t pol) {
  constexpr int GS = g_stride(C);
  static_assert(GS % 4 == 0, "rows of whole float4s");
  float wgt[4], dot[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    float w = 0.0f;
    if (gq[s] >= 0) {
      if (iq[s].y == 1.0f) w = 1.0f;                         // empty: 1/(1+0) = 1, overwrite
      else if (z > __fmul_rn(iq[s].x, a1)) w = 0.0f;         // behind the target surface
      else if (__fmul_rn(z, a1) < iq[s].x) w = 1.0f;         // in front: replaces the mean
      else w = iq[s].y;                                       // joins the fuzzy blend: 1/(1+|Lambda|)
    }
    wgt[s] = w;
    dot[s] = 0.0f;
  }
  const float4* rows = reinterpret_cast<const float4*>(cam.gpm);
#pragma unroll
  for (int h = 0; h < GS / 4; ++h) {
    float4 g4[4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
      g4[s] = wgt[s] != 0.0f ? ld_keep(rows + (int64_t)gq[s] * (GS / 4) + h, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float gv[4] = {g4[s].x, g4[s].y, g4[s].z, g4[s].w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * h + j < C) dot[s] = fmaf(gv[j], tau[4 * h + j], dot[s]);
    }
  }
  float cq[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) cq[s] = wgt[s] != 0.0f ? wgt[s] * (dot[s] - iq[s].z) : 0.0f;
  g_u = 0.5f * (cq[0] - cq[1]);
  g_v = 0.5f * (cq[2] - cq[3]);
}

// One (point, layer) pair in Lambda: v[0..C) = G(p)/|Lambda(p)| (dI/dtau
// contracted with the upstream gradient) and v[C], v[C+1] = the layer-0
// pixel gradient (du0, dv0) of Eq. gradp at this layer.  sp: the point's
// record (z, u0, v0, X, tau).
template <int C>
__device__ __forceinline__ void pair_contrib(const DevCam& cam, const PointArgs& a, const float4* __restrict__ info,
                                             const float* sp, int l, bool spatial_out, uint64_t pol,
                                             float (&v)[C + 2]) {
  constexpr int GS = g_stride(C);
  int32_t pu, pv;
  // a listed pair's point passed a fuzzy test, so in_pyramid held for the same (u0, v0)
  if (!pixel_in(sp[1], sp[2], l, cam.w, cam.h, pu, pv)) return;  // always in bounds for a listed pair
  const int32_t wl = cam.w >> l, hl = cam.h >> l;
  const int64_t lb = cam.off[l];
  const int64_t gp = lb + (int64_t)pv * wl + pu;
  const float4 ip = ld_keep(info + gp, pol);
  float G[GS];
  load_keep_row<GS>(cam.gpm + gp * GS, G, pol);
  if constexpr (GS % 4 == 0) {
    // the 4 neighbour records are issued with the pixel's own record and row,
    // so that a pair waits for one wave of misses before its case tests
    // (with the rows of spatial_grad_loaded: step 0.4243 -> 0.4213 ms;
    // issuing only the rows together: no change)
    int32_t gq[4];
    float4 iq[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int32_t qu = pu + (s == 0 ? 1 : (s == 1 ? -1 : 0));
      const int32_t qv = pv + (s == 2 ? 1 : (s == 3 ? -1 : 0));
      gq[s] = (!spatial_out || qu < 0 || qu >= wl || qv < 0 || qv >= hl) ? -1 : (int32_t)(lb + (int64_t)qv * wl + qu);
      iq[s] = gq[s] >= 0 ? ld_keep(info + gq[s], pol) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = G[c] * ip.w;  // ip.w = f32(1/|Lambda|)
    if (spatial_out) {
      float g_u, g_v;
      spatial_grad_loaded<C>(cam, iq, gq, sp[0], a.a1, sp + 6, g_u, g_v, pol);  // tau read from shared memory
      const float sc = layer_scale(l);
      v[C] = g_u * sc;
      v[C + 1] = g_v * sc;
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = G[c] * ip.w;  // ip.w = f32(1/|Lambda|)
    if (spatial_out) {
      float g_u, g_v;
      spatial_grad<C>(cam, info, lb, pu, pv, wl, hl, sp[0], a.a1, sp + 6, g_u, g_v, pol);  // tau read from shared memory
      const float sc = layer_scale(l);
      v[C] = g_u * sc;
      v[C + 1] = g_v * sc;
    }
  }
}

// The same backward when the accumulate pass recorded each point's layer mask
// (and only points in Lambda get spatial gradients).  Each warp takes 32
// consecutive points.  Nearly every one of them is in Lambda at layer 0, so a
// first round gives every lane its own point's layer-0 pair, summed straight
// into that point's sums.  The pairs of the coarser layers are then listed in
// shared memory and processed densely, one pair per lane, so that lanes are
// not idle on the (majority of) occluded pairs; a point's sums over those
// layers are segmented warp reductions (its pairs are consecutive in the
// list).  (Layer 0 first, without the list and its reduction: 178.5 -> 173.7
// us on the 1080p step.)  The owning lane then applies the chain rule and
// writes its point's gradients.
template <int C, typename TF, bool BINNED>
__global__ void __launch_bounds__(kThreads, 4) k_bwd_items(const __grid_constant__ LaunchCams cams,
                                                           const __grid_constant__ PointArgs a,
                                                           const __grid_constant__ BwdArgs b) {
  pdl_entry();
  constexpr int GS = g_stride(C);
  constexpr int PS = (6 + C) | 1;  // per point: z, u0, v0, X (camera space), tau (odd stride: no bank conflicts)
  constexpr int AS = (C + 2) | 1;  // per point: sum of G/|Lambda|, du0, dv0
  constexpr int kWarps = kThreads / 32;
  __shared__ float s_pt[kWarps][32 * PS];
  __shared__ float s_acc[kWarps][32 * AS];
  __shared__ uint8_t s_item[kWarps][32 * ADOP_MAX_LEVELS];
  __shared__ float s_red[12][kThreads];  // per thread: its points' pose / intrinsics terms
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DevCam& cam = cams.c[blockIdx.y];
  const TF* feat = reinterpret_cast<const TF*>(a.feat);
  const float4* info = reinterpret_cast<const float4*>(cam.info);
  const bool spatial_out = b.grad_xyz != nullptr || b.partials != nullptr;
  float* pt = s_pt[warp];
  float* acc = s_acc[warp];
  uint8_t* item = s_item[warp];
  const uint64_t pol = policy_evict_last();
#pragma unroll
  for (int k = 0; k < 12; ++k) s_red[k][threadIdx.x] = 0.0f;

  // the points to visit: all, in index order, or the visible ones tile by tile
  const int64_t count = BINNED ? (int64_t)cam.bin_off[cam.tiles] : a.n;
  const int64_t stride = (int64_t)gridDim.x * kWarps * 32;
  for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32; base < count; base += stride) {
    const int64_t j = base + lane;
    const int64_t i = j < count ? (BINNED ? (int64_t)__ldcs(cam.bin_list + j) : j) : a.n;
    const uint32_t mask = i < a.n ? (__ldcs(cam.vis + i) & 0xFFu) : 0u;
    if (mask) {
      float X0, X1, X2, u0 = 0.0f, v0 = 0.0f, zd = 0.0f;
      transform(cam, __ldcs(a.xyz + 3 * i), __ldcs(a.xyz + 3 * i + 1), __ldcs(a.xyz + 3 * i + 2), X0, X1, X2);
      camera(cam, X0, X1, X2, u0, v0, zd);  // defined: the point passed a fuzzy test
      float tau[C];
      load_desc<C, TF>(feat, i, a.log_desc, tau);
      float* sp = pt + lane * PS;
      sp[0] = zd;
      sp[1] = u0;
      sp[2] = v0;
      sp[3] = X0;
      sp[4] = X1;
      sp[5] = X2;
#pragma unroll
      for (int k = 0; k < C; ++k) sp[6 + k] = tau[k];
    }
    // round 0: every lane's own layer-0 pair (nearly every point in Lambda has
    // one), straight into its point's sums -- no list, no reduction
    {
      float v[C + 2];
#pragma unroll
      for (int c = 0; c < C + 2; ++c) v[c] = 0.0f;
      if (mask & 1u) pair_contrib<C>(cam, a, info, pt + lane * PS, 0, spatial_out, pol, v);
#pragma unroll
      for (int c = 0; c < C + 2; ++c) acc[lane * AS + c] = v[c];
    }
    // the coarser layers' pairs: listed densely (exclusive scan of the
    // per-lane counts), one pair per lane
    const uint32_t rest = mask & ~1u;
    const int cnt = __popc(rest);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int slot = incl - cnt;
    for (uint32_t m = rest; m; m &= m - 1) item[slot++] = (uint8_t)((lane << 3) | (__ffs(m) - 1));
    __syncwarp();
    for (int r = 0; r < total; r += 32) {  // warp-uniform: every lane takes part in the shuffles
      const int k = r + lane;
      float v[C + 2];
#pragma unroll
      for (int c = 0; c < C + 2; ++c) v[c] = 0.0f;
      int src = -1 - lane;  // lanes without a pair form runs of their own
      if (k < total) {
        const int it = item[k];
        src = it >> 3;
        pair_contrib<C>(cam, a, info, pt + src * PS, it & 7, spatial_out, pol, v);
      }
      // A point's pairs are consecutive in the list: sum each run of equal
      // src over the lanes (segmented reduction, run ends from a ballot), and
      // let the run's first lane add it to the point's sums.  Runs are
      // disjoint within a round and rounds follow each other, so plain adds
      // suffice.
      const int next = __shfl_down_sync(0xffffffffu, src, 1);
      const int prev = __shfl_up_sync(0xffffffffu, src, 1);
      const uint32_t tails = __ballot_sync(0xffffffffu, lane == 31 || next != src);
      const int end = __ffs(tails & (0xffffffffu << lane)) - 1;
      // a run is at most levels - 1 long (one pair per coarse layer); stop at
      // the first step that no run needs
      for (int o = 1; o < a.levels - 1 && __any_sync(0xffffffffu, lane + o <= end); o <<= 1) {
#pragma unroll
        for (int c = 0; c < C + 2; ++c) {
          const float t = __shfl_down_sync(0xffffffffu, v[c], o);
          if (lane + o <= end) v[c] += t;
        }
      }
      if (src >= 0 && (lane == 0 || prev != src)) {
        float* ap = acc + src * AS;
#pragma unroll
        for (int c = 0; c < C + 2; ++c) ap[c] += v[c];
      }
    }
    __syncwarp();
    if (i < a.n) {
      const float* sp = pt + lane * PS;
      float gf[C];
#pragma unroll
      for (int k = 0; k < C; ++k) gf[k] = acc[lane * AS + k] * (a.log_desc && mask ? sp[6 + k] : 1.0f);
      // (binned: the points in no Lambda get zero gradients after the loop)
      float gx[3] = {0.0f, 0.0f, 0.0f};
      const float du0 = acc[lane * AS + C], dv0 = acc[lane * AS + C + 1];
      if (mask && (du0 != 0.0f || dv0 != 0.0f)) {
        float red[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) red[k] = s_red[k][threadIdx.x];
        chain_rule(cam, sp[3], sp[4], sp[5], du0, dv0, red, gx);
#pragma unroll
        for (int k = 0; k < 12; ++k) s_red[k][threadIdx.x] = red[k];
      }
      write_point_grads<C>(b, i, gf, gx, mask != 0u);
    }
    __syncwarp();
  }
  if (BINNED && b.mode == kGradAssign) {
    // the points in no Lambda get zero gradients here: streaming stores that
    // overlap the blocks still busy with latency-bound pairs (in the binning
    // kernel they cost 34 us, here 24).  Four grid-stride steps at a time, so
    // that their mask loads are in flight together while each store still
    // covers consecutive points across the warp (point pass 170 -> 166 us on
    // the 5M-point view, 959 -> 890 us on the 120M-point frame; two at a time
    // 167 / 870 us)
    const float zf[C] = {};
    const float zx[3] = {0.0f, 0.0f, 0.0f};
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < a.n; i0 += 4 * S) {
      uint32_t m[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) m[u] = i0 + u * S < a.n ? (__ldcs(cam.vis + i0 + u * S) & 0xFFu) : 1u;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (m[u] == 0u) write_point_grads<C>(b, i0 + u * S, zf, zx, false);
    }
  }
  if (b.partials != nullptr) {  // block sum of the pose / intrinsics terms: warp w takes terms w, w + 8
    __syncthreads();
    for (int k = warp; k < 12; k += kWarps) {
      float t = 0.0f;
      for (int j = lane; j < kThreads; j += 32) t += s_red[k][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) b.partials[((int64_t)blockIdx.y * 12 + k) * gridDim.x + blockIdx.x] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// screen-tile binning of the visible points: count, exclusive scan, scatter
// ---------------------------------------------------------------------------

// Runs of equal keys among consecutive lanes (inactive lanes are runs of
// their own): the lane's run head, the run length and the lane's rank in it.
__device__ __forceinline__ void lane_run(uint32_t key, bool active, int lane, int& head, int& len, int& rank) {
  const uint32_t k = active ? key : (0xFF000000u | (uint32_t)lane);  // tiles < 2^24: never equal to a sentinel
  const uint32_t prev = __shfl_up_sync(0xffffffffu, k, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || k != prev);
  head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  const unsigned above = lane == 31 ? 0u : (heads & (0xffffffffu << (lane + 1)));
  const int end = above ? __ffs(above) - 1 : 32;
  len = end - head;
  rank = lane - head;
}

__global__ void __launch_bounds__(kThreads) k_bin_count(const __grid_constant__ LaunchCams cams,
                                                        const __grid_constant__ PointArgs a) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
    const int64_t i = base + lane;
    const uint32_t v = i < a.n ? __ldg(cam.vis + i) : 0u;
    const bool active = (v & 0xFFu) != 0u;
    const uint32_t tile = min(v >> 8, (uint32_t)cam.tiles - 1u);
    int head, len, rank;
    lane_run(tile, active, lane, head, len, rank);
    if (active && rank == 0) atomicAdd(cam.bin_count + tile, len);
  }
}

// One block per camera: exclusive scan of the tile counts; the counts become
// the scatter cursors (= the offsets).
__global__ void __launch_bounds__(1024) k_bin_scan(const __grid_constant__ LaunchCams cams) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.x];
  __shared__ int32_t warp_sum[32];
  const int T = cam.tiles;
  const int per = (T + 1023) / 1024;
  const int t0 = threadIdx.x * per;
  int32_t local = 0;
  for (int t = t0; t < min(t0 + per, T); ++t) local += cam.bin_count[t];
  // block-wide exclusive scan of the per-thread sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w;
  }
  __syncthreads();
  int32_t run = incl - local + (warp > 0 ? warp_sum[warp - 1] : 0);
  for (int t = t0; t < min(t0 + per, T); ++t) {
    const int32_t c = cam.bin_count[t];
    cam.bin_off[t] = run;
    cam.bin_count[t] = run;
    run += c;
  }
  if (threadIdx.x == 1023) cam.bin_off[T] = warp_sum[31];
}

template <int C>
__global__ void __launch_bounds__(kThreads) k_bin_scatter(const __grid_constant__ LaunchCams cams,
                                                          const __grid_constant__ PointArgs a,
                                                          const __grid_constant__ BwdArgs b) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
    const int64_t i = base + lane;
    const uint32_t v = i < a.n ? __ldg(cam.vis + i) : 0u;
    const bool active = (v & 0xFFu) != 0u;
    const uint32_t tile = min(v >> 8, (uint32_t)cam.tiles - 1u);
    int head, len, rank;
    lane_run(tile, active, lane, head, len, rank);
    int32_t slot = 0;
    if (active && rank == 0) slot = atomicAdd(cam.bin_count + tile, len);
    slot = __shfl_sync(0xffffffffu, slot, head) + rank;
    if (active) cam.bin_list[slot] = (int32_t)i;
  }
}

// Block-local binning (tiles <= kBinSmemTiles): every block takes one
// contiguous chunk of points, so it touches few tiles; it counts them in
// shared memory and issues one global atomic per touched tile, instead of
// one per run of lanes (which serialises on the few tiles that a surface
// being streamed covers).  The value each of those atomics returns is the
// block's first slot within the tile's range; the count kernel keeps it in
// the block's row of cam.bin_table, and the scatter (same grid, same
// chunks) adds the tile's offset and places its points without counting
// them again: one read of the masks instead of two (binning on the
// 120M-point frame 267 -> 194 us; unchanged on the 5M-point view).
constexpr int kBinBlocksPerSm = 8;

__device__ __forceinline__ void chunk_of(int64_t n, int64_t& c0, int64_t& c1) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  c0 = (int64_t)blockIdx.x * per;
  c1 = min(n, c0 + per);
}

__global__ void __launch_bounds__(kThreads) k_bin_count_blk(const __grid_constant__ LaunchCams cams,
                                                            const __grid_constant__ PointArgs a) {
  pdl_entry();
  extern __shared__ int32_t bins[];
  const DevCam& cam = cams.c[blockIdx.y];
  const int T = cam.tiles;
  for (int t = threadIdx.x; t < T; t += blockDim.x) bins[t] = 0;
  __syncthreads();
  int64_t c0, c1;
  chunk_of(a.n, c0, c1);
#pragma unroll 4
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    const uint32_t v = __ldg(cam.vis + i);
    if (v & 0xFFu) atomicAdd(bins + min(v >> 8, (uint32_t)T - 1u), 1);
  }
  __syncthreads();
  int32_t* row = cam.bin_table + (int64_t)blockIdx.x * T;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const int32_t c = bins[t];
    row[t] = c ? atomicAdd(cam.bin_count + t, c) : 0;
  }
}

template <int C>
__global__ void __launch_bounds__(kThreads) k_bin_scatter_blk(const __grid_constant__ LaunchCams cams,
                                                              const __grid_constant__ PointArgs a,
                                                              const __grid_constant__ BwdArgs b) {
  pdl_entry();
  extern __shared__ int32_t bins[];  // this block's next slot per tile
  const DevCam& cam = cams.c[blockIdx.y];
  const int T = cam.tiles;
  const int32_t* row = cam.bin_table + (int64_t)blockIdx.x * T;
  for (int t = threadIdx.x; t < T; t += blockDim.x) bins[t] = cam.bin_off[t] + row[t];
  __syncthreads();
  int64_t c0, c1;
  chunk_of(a.n, c0, c1);
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    const uint32_t v = __ldg(cam.vis + i);
    if (v & 0xFFu) cam.bin_list[atomicAdd(bins + min(v >> 8, (uint32_t)T - 1u), 1)] = (int32_t)i;
  }
}

// Block (k, camera) sums element k of the pose / intrinsics terms over all
// block partials (laid out element-major, [camera][12][block], so that the
// loads coalesce): each thread a strided share, then the warps, then the
// warp sums in order: a fixed order for given partials.
constexpr int kReduceThreads = 256;

__global__ void __launch_bounds__(kReduceThreads) k_bwd_reduce(const float* __restrict__ partials, int blocks_x,
                                                               float* grad_pose, float* grad_intr) {
  pdl_entry();
  __shared__ float sm[kReduceThreads / 32];
  const int k = blockIdx.x, cam = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* pk = partials + ((int64_t)cam * 12 + k) * blocks_x;
  float v = 0.0f;
  for (int bi = threadIdx.x; bi < blocks_x; bi += kReduceThreads) v += pk[bi];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < kReduceThreads / 32; ++w) t += sm[w];
    if (k < 6) {
      if (grad_pose) grad_pose[cam * 6 + k] += t;
    } else if (grad_intr) {
      grad_intr[cam * 6 + k - 6] += t;
    }
  }
}

cudaError_t launch_bwd_prepass(const LaunchCams& cams, const PointArgs& a, int c, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int64_t px = most_pixels(cams, a);
  ADOP_DISPATCH_C(c, ADOP_DISPATCH_T((adop_dtype)a.grad_dtype, TG,
                                     e = launch_strided(k_bwd_prepass<kC, TG>, px, a.ncam, kPixelWaves, 0, s, cams,
                                                        a)));
  return e;
}

cudaError_t launch_bwd_points(const LaunchCams& cams, const PointArgs& a, const BwdArgs& b, int c,
                              adop_dtype fd, int blocks_x, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const dim3 grid(blocks_x, a.ncam);
  bool dense = !b.all_projected, binned = true;
  for (int k = 0; k < a.ncam; ++k) {
    dense = dense && cams.c[k].vis != nullptr;
    binned = binned && cams.c[k].bin_list != nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (dense && binned) {
    ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(fd, TF, e = launch_pdl(k_bwd_items<kC, TF, true>, grid, kThreads, 0, s, cams, a,
                                                              b)));
  } else if (dense) {
    ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(fd, TF, e = launch_pdl(k_bwd_items<kC, TF, false>, grid, kThreads, 0, s, cams, a,
                                                              b)));
  } else {
    ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(fd, TF, e = launch_pdl(k_bwd_points<kC, TF>, grid, kThreads, 0, s, cams, a,
                                                              b)));
  }
  return e;
}

cudaError_t launch_bin(const LaunchCams& cams, const PointArgs& a, const BwdArgs& b, int c, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  for (int k = 0; k < a.ncam; ++k) {
    cudaError_t e = cudaMemsetAsync(cams.c[k].bin_count, 0, sizeof(int32_t) * (size_t)cams.c[k].tiles, s);
    if (e != cudaSuccess) return e;
  }
  int most = 0;
  for (int k = 0; k < a.ncam; ++k) most = cams.c[k].tiles > most ? cams.c[k].tiles : most;
  if (most <= kBinSmemTiles) {
    const size_t smem = sizeof(int32_t) * (size_t)most;
    int64_t want = (int64_t)num_sms() * kBinBlocksPerSm;
    want = (want + a.ncam - 1) / a.ncam;
    for (int k = 0; k < a.ncam; ++k) want = want < cams.c[k].bin_rows ? want : cams.c[k].bin_rows;
    const dim3 grid((unsigned)(want < 1 ? 1 : want), a.ncam);
    cudaError_t e = launch_pdl(k_bin_count_blk, grid, kThreads, smem, s, cams, a);
    if (e == cudaSuccess) e = launch_pdl(k_bin_scan, dim3(a.ncam), dim3(1024), 0, s, cams);
    if (e == cudaSuccess) ADOP_DISPATCH_C(c, e = launch_pdl(k_bin_scatter_blk<kC>, grid, kThreads, smem, s, cams, a, b));
    return e;
  }
  const dim3 grid(point_blocks(a.n, a.ncam), a.ncam);
  cudaError_t e = launch_pdl(k_bin_count, grid, kThreads, 0, s, cams, a);
  if (e == cudaSuccess) e = launch_pdl(k_bin_scan, dim3(a.ncam), dim3(1024), 0, s, cams);
  if (e == cudaSuccess) ADOP_DISPATCH_C(c, e = launch_pdl(k_bin_scatter<kC>, grid, kThreads, 0, s, cams, a, b));
  return e;
}

cudaError_t launch_bwd_reduce(const float* partials, int ncam, int blocks_x, float* grad_pose,
                              float* grad_intr, cudaStream_t s) {
  return launch_pdl(k_bwd_reduce, dim3(12, ncam), dim3(kReduceThreads), 0, s, partials, blocks_x, grad_pose,
                    grad_intr);
}

}  // namespace adop
