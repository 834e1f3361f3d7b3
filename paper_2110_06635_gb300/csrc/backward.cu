// Backward pass of the one-pixel point rasterizer (Sec. 3.1, "Backward
// Pass"): feature gradients, the approximate one-pixel spatial gradient
// (Eqs. induce, gradp, spatialderiv) and the chain rule to positions, the
// SE(3) tangent of the pose (Eq. tangent) and the intrinsics (Eq. partial).
//
//   k_bwd_prepass  one thread per pixel: packs what a point needs to know
//                  about a pixel into one record -- min depth, |Lambda|,
//                  <G, I> and the (epilogue-chained) upstream gradient G --
//                  so that the 5 pixels a point visits per layer cost 5
//                  contiguous record reads instead of 2c strided gathers.
//   k_bwd_points   one thread per point and camera: visits its pixel and the
//                  4 neighbours in every layer, writes its own dL/dtau and
//                  dL/dx (owner computes: no atomics for one camera), and
//                  reduces pose/intrinsic terms warp -> block into per-block
//                  partial sums.
//   k_bwd_reduce   sums the block partials in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "launch.h"

namespace adop {

template <int C>
__global__ void __launch_bounds__(kThreads) k_bwd_prepass(const __grid_constant__ LaunchCams cams,
                                                          const __grid_constant__ PointArgs a) {
  constexpr int RS = rec_stride(C);
  const DevCam& cam = cams.c[blockIdx.y];
  const int64_t total = cam.off[a.levels];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int l = layer_of(cam, a.levels, g);
    const int64_t p = g - cam.off[l];
    const int64_t np = cam.off[l + 1] - cam.off[l];
    const uint32_t n = cam.cnt[l][p];
    const unsigned long long key = cam.key[l][p];
    float I[C], G[C];
    if (n == 0) {
#pragma unroll
      for (int k = 0; k < C; ++k) I[k] = a.background ? __ldg(a.background + k) : 0.0f;
    } else {
      const float fn = (float)n;
#pragma unroll
      for (int k = 0; k < C; ++k) I[k] = __fdiv_rn(cam.acc[g * C + k], fn);
    }
    const float* gl = cam.grad[l];
#pragma unroll
    for (int k = 0; k < C; ++k) G[k] = gl ? __ldg(gl + k * np + p) : 0.0f;
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
    float r[RS];
    r[0] = __uint_as_float((uint32_t)(key >> 32));
    r[1] = (float)n;
    r[2] = gi;
#pragma unroll
    for (int k = 0; k < C; ++k) r[3 + k] = G[k];
#pragma unroll
    for (int k = 3 + C; k < RS; ++k) r[k] = 0.0f;
    float4* dst = reinterpret_cast<float4*>(cam.rec + g * RS);
#pragma unroll
    for (int v = 0; v < RS / 4; ++v) dst[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
  }
}

template <int RS>
__device__ __forceinline__ void load_rec(const float* rp, float (&r)[RS]) {
#pragma unroll
  for (int v = 0; v < RS / 4; ++v) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(rp) + v);
    r[4 * v] = q.x;
    r[4 * v + 1] = q.y;
    r[4 * v + 2] = q.z;
    r[4 * v + 3] = q.w;
  }
}

template <int C, typename TF>
__global__ void __launch_bounds__(kThreads) k_bwd_points(const __grid_constant__ LaunchCams cams,
                                                         const __grid_constant__ PointArgs a,
                                                         const __grid_constant__ BwdArgs b) {
  constexpr int RS = rec_stride(C);
  const DevCam& cam = cams.c[blockIdx.y];
  const TF* feat = reinterpret_cast<const TF*>(a.feat);
  float red[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) red[k] = 0.0f;

  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    float gf[C];
#pragma unroll
    for (int k = 0; k < C; ++k) gf[k] = 0.0f;
    float gx[3] = {0.0f, 0.0f, 0.0f};
    bool touched = false;

    float X0, X1, X2, u0, v0;
    transform(cam, __ldg(a.xyz + 3 * i), __ldg(a.xyz + 3 * i + 1), __ldg(a.xyz + 3 * i + 2), X0, X1, X2);
    const bool valid = (X2 > a.znear) && !(a.normals && !normal_keep(cam, a.normals, i, X0, X1, X2));
    if (valid) {
      camera(cam, X0, X1, X2, u0, v0);
      float tau[C];
      bool loaded = false;
      float du0 = 0.0f, dv0 = 0.0f;
      bool spatial = false;
      for (int l = 0; l < a.levels; ++l) {
        int32_t pu, pv;
        if (!pixel_at(u0, v0, l, cam.w, cam.h, pu, pv)) continue;
        const int32_t wl = cam.w >> l, hl = cam.h >> l;
        const float* base = cam.rec + cam.off[l] * RS;
        float rp[RS];
        load_rec<RS>(base + ((int64_t)pv * wl + pu) * RS, rp);
        const bool vis = X2 <= __fmul_rn(rp[0], a.a1);
        if (vis) {
          // dI(p)/dtau_i = 1/|Lambda(p)| for every member of Lambda(p)
#pragma unroll
          for (int k = 0; k < C; ++k) gf[k] += __fdiv_rn(rp[3 + k], rp[1]);
          touched = true;
        }
        if (!(vis || b.all_projected) || (b.grad_xyz == nullptr && b.partials == nullptr)) continue;
        if (!loaded) {
          load_feat<C, TF>(feat, i, tau);
          loaded = true;
        }
        // induced change at the 4 neighbours (+u, -u, +v, -v), contracted with G there
        float cq[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int32_t qu = pu + (s == 0 ? 1 : (s == 1 ? -1 : 0));
          const int32_t qv = pv + (s == 2 ? 1 : (s == 3 ? -1 : 0));
          cq[s] = 0.0f;
          if (qu < 0 || qu >= wl || qv < 0 || qv >= hl) continue;
          float rq[RS];
          load_rec<RS>(base + ((int64_t)qv * wl + qu) * RS, rq);
          float wgt;
          if (rq[1] == 0.0f) wgt = 1.0f;                              // empty: overwrite background
          else if (X2 > __fmul_rn(rq[0], a.a1)) wgt = 0.0f;          // behind the target surface
          else if (__fmul_rn(X2, a.a1) < rq[0]) wgt = 1.0f;          // in front: replaces the mean
          else wgt = __frcp_rn(1.0f + rq[1]);                         // joins the fuzzy blend
          if (wgt == 0.0f) continue;
          float dot = 0.0f;
#pragma unroll
          for (int k = 0; k < C; ++k) dot = fmaf(rq[3 + k], tau[k], dot);
          cq[s] = wgt * (dot - rq[2]);
        }
        const float s = layer_scale(l);
        du0 = fmaf(0.5f * (cq[0] - cq[1]), s, du0);
        dv0 = fmaf(0.5f * (cq[2] - cq[3]), s, dv0);
        spatial = true;
      }
      if (spatial && (du0 != 0.0f || dv0 != 0.0f)) {
        // chain rule through the camera model (FP32)
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
        // left increment exp(xi) (R, t): dX/dnu = I, dX/domega = -[X]x
        red[0] += dX0;
        red[1] += dX1;
        red[2] += dX2;
        red[3] += X1 * dX2 - X2 * dX1;
        red[4] += X2 * dX0 - X0 * dX2;
        red[5] += X0 * dX1 - X1 * dX0;
        // intrinsics fx, fy, cx, cy, k1, k2
        red[6] += du0 * xd;
        red[7] += dv0 * yd;
        red[8] += du0;
        red[9] += dv0;
        red[10] += (gxd * xn + gyd * yn) * r2;
        red[11] += (gxd * xn + gyd * yn) * r2 * r2;
        // dL/dx = R^T dL/dX
        gx[0] = cam.R[0] * dX0 + cam.R[3] * dX1 + cam.R[6] * dX2;
        gx[1] = cam.R[1] * dX0 + cam.R[4] * dX1 + cam.R[7] * dX2;
        gx[2] = cam.R[2] * dX0 + cam.R[5] * dX1 + cam.R[8] * dX2;
        touched = true;
      }
    }

    // write this point's gradients
    if (b.mode == kGradAssign) {
      if (b.grad_feat) {
        float* dst = b.grad_feat + i * C;
#pragma unroll
        for (int k = 0; k < C; ++k) dst[k] = gf[k];
      }
      if (b.grad_xyz) {
        b.grad_xyz[3 * i] = gx[0];
        b.grad_xyz[3 * i + 1] = gx[1];
        b.grad_xyz[3 * i + 2] = gx[2];
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

  // pose / intrinsics: warp shuffle -> shared memory -> one partial per block
  if (b.partials == nullptr) return;
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
    b.partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 12 + threadIdx.x] = v;
  }
}

// One block per camera, warp k sums element k over all block partials.
__global__ void __launch_bounds__(384) k_bwd_reduce(const float* __restrict__ partials, int blocks_x,
                                                    float* grad_pose, float* grad_intr) {
  const int cam = blockIdx.x;
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  float v = 0.0f;
  for (int bi = lane; bi < blocks_x; bi += 32) v += partials[((int64_t)cam * blocks_x + bi) * 12 + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    if (k < 6) {
      if (grad_pose) grad_pose[cam * 6 + k] += v;
    } else if (grad_intr) {
      grad_intr[cam * 6 + k - 6] += v;
    }
  }
}

cudaError_t launch_bwd_prepass(const LaunchCams& cams, const PointArgs& a, int c, cudaStream_t s) {
  ADOP_DISPATCH_C(c, k_bwd_prepass<kC><<<pixel_grid(cams, a), kThreads, 0, s>>>(cams, a));
  return cudaGetLastError();
}

cudaError_t launch_bwd_points(const LaunchCams& cams, const PointArgs& a, const BwdArgs& b, int c,
                              adop_dtype fd, int blocks_x, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const dim3 grid(blocks_x, a.ncam);
  ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(fd, TF, k_bwd_points<kC, TF><<<grid, kThreads, 0, s>>>(cams, a, b)));
  return cudaGetLastError();
}

cudaError_t launch_bwd_reduce(const float* partials, int ncam, int blocks_x, float* grad_pose,
                              float* grad_intr, cudaStream_t s) {
  k_bwd_reduce<<<ncam, 384, 0, s>>>(partials, blocks_x, grad_pose, grad_intr);
  return cudaGetLastError();
}

}  // namespace adop
