// Environment map (Sec. 3.1).  An empty pixel shows the bilinear sample
// sum_j w_j E[t_j] along its ray (env_taps: inverse camera, R^T, the
// equirectangular lookup), so dL/dE[t_j] gains w_j G for every channel.
//   k_env_fill  one thread per pyramid pixel: samples the map where no point
//               landed, keeps the value in acc, writes the image pixel.
//   k_env_grad  one thread per pyramid pixel: recomputes the taps, chains
//               layer 0 through the photometric epilogue and adds w_j G with
//               FP32 vector atomics (the map is texel-major: a texel's C
//               floats are contiguous).
#include <cuda_runtime.h>

#include "launch.h"

namespace adop {
namespace {

// Sample the map for every empty pixel: the value goes to acc (the pixel
// state the backward pass reads) and, where the layer's image is written, to
// the image (through the photometric epilogue at layer 0).
template <int C, typename TO>
__global__ void __launch_bounds__(kThreads) k_env_fill(const __grid_constant__ LaunchCams cams,
                                                       const __grid_constant__ PointArgs a) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const int64_t total = cam.off[a.levels];
  int lc = 0;  // the layer of g: g only grows, so its layer only advances
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    while (lc + 1 < a.levels && g >= cam.off[lc + 1]) ++lc;
    const int l = lc;
    const int64_t p = g - cam.off[l];
    if (cam.cnt[l][p] != 0) continue;
    const int32_t wl = cam.w >> l, pi = (int32_t)p;  // a pyramid has fewer than 2^31 pixels
    const int32_t pu = pi % wl, pv = pi / wl;
    float v[C];
    env_sample<C>(a.env, env_taps(cam, a.env_w, a.env_h, l, pu, pv), v);
    store_vec<C>(cam.acc + g * C, v);
    TO* img = reinterpret_cast<TO*>(cam.image[l]);
    if (img == nullptr) continue;
    if (l == 0 && cam.epi) {
#pragma unroll
      for (int k = 0; k < (C < 3 ? C : 3); ++k) v[k] = epilogue(cam, k, pu, pv, v[k], nullptr);
    }
    const int64_t np = cam.off[l + 1] - cam.off[l];
#pragma unroll
    for (int k = 0; k < C; ++k) img[k * np + p] = from_f32<TO>(v[k]);
  }
}

// dL/dE: each empty pixel adds w_j G to its four texels with FP32 vector
// atomics.  (Summing runs of equal taps across the warp first was measured
// slower: the shuffles cost more instructions and registers than the
// atomics they saved.)
template <int C>
__global__ void __launch_bounds__(kThreads) k_env_grad(const __grid_constant__ LaunchCams cams,
                                                       const __grid_constant__ PointArgs a, float* grad_env) {
  pdl_entry();
  const DevCam& cam = cams.c[blockIdx.y];
  const int64_t total = cam.off[a.levels];
  int lc = 0;  // the layer of g: g only grows, so its layer only advances
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    while (lc + 1 < a.levels && g >= cam.off[lc + 1]) ++lc;
    const int l = lc;
    const float* gl = cam.grad[l];
    const int64_t p = g - cam.off[l];
    if (gl == nullptr || cam.cnt[l][p] != 0) continue;
    const int64_t np = cam.off[l + 1] - cam.off[l];
    const int32_t wl = cam.w >> l, pi = (int32_t)p;
    const int32_t pu = pi % wl, pv = pi / wl;
    const EnvTaps e = env_taps(cam, a.env_w, a.env_h, l, pu, pv);
    float G[C];
#pragma unroll
    for (int k = 0; k < C; ++k) G[k] = __ldg(gl + k * np + p);
    if (l == 0 && cam.epi) {
      float I[C];
      if (cam.env_in_acc) {
        load_vec<C>(cam.acc + g * C, I);
      } else {
        env_sample<C>(a.env, e, I);
      }
#pragma unroll
      for (int k = 0; k < (C < 3 ? C : 3); ++k) {
        float d;
        epilogue(cam, k, pu, pv, I[k], &d);
        G[k] *= d;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (e.w[j] == 0.0f) continue;
      float wg[C];
#pragma unroll
      for (int k = 0; k < C; ++k) wg[k] = e.w[j] * G[k];
      atomic_add_vec<C>(grad_env + (int64_t)e.t[j] * C, wg);
    }
  }
}

adop_status fail(adop_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace

cudaError_t launch_env_fill(const LaunchCams& cams, const PointArgs& a, int c, adop_dtype od, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int64_t px = most_pixels(cams, a);
  ADOP_DISPATCH_C(c, ADOP_DISPATCH_T(od, TO, e = launch_strided(k_env_fill<kC, TO>, px, a.ncam, kPixelWaves, 0, s,
                                                                cams, a)));
  return e;
}

cudaError_t launch_env_grad(const LaunchCams& cams, const PointArgs& a, int c, float* grad_env, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int64_t px = most_pixels(cams, a);
  ADOP_DISPATCH_C(c, e = launch_strided(k_env_grad<kC>, px, a.ncam, kPixelWaves, 0, s, cams, a, grad_env));
  return e;
}

}  // namespace adop

using namespace adop;

extern "C" adop_status adop_env_backward(const adop_camera* cams, int32_t n_cam, const adop_params* params,
                                         int32_t c, const adop_frame* frames, const float* const* grad_image,
                                         float* grad_env, adop_stream stream) {
  if (!cams || !params || !frames || !grad_env) return fail(ADOP_ERR_INVALID_ARG, "NULL argument");
  if (!params->env) return fail(ADOP_ERR_INVALID_ARG, "params->env is NULL: no environment map to differentiate");
  if (!env_size_ok(params->env_w, params->env_h))
    return fail(ADOP_ERR_INVALID_ARG, "env_w / env_h outside [1, 16384]");
  if (((uintptr_t)params->env & 15) != 0 || ((uintptr_t)grad_env & 15) != 0)
    return fail(ADOP_ERR_INVALID_ARG, "env / grad_env must be 16-byte aligned");
  if (n_cam < 1 || n_cam > ADOP_MAX_CAMERAS) return fail(ADOP_ERR_INVALID_ARG, "n_cam outside [1, 64]");
  if (!channels_supported(c)) return fail(ADOP_ERR_UNSUPPORTED, "channel count has no kernels");
  if (params->levels < 1 || params->levels > ADOP_MAX_LEVELS) return fail(ADOP_ERR_INVALID_ARG, "levels outside [1, 8]");
  if (params->grad_dtype != ADOP_F32)
    return fail(ADOP_ERR_UNSUPPORTED, "this call reads FP32 upstream gradients only (params->grad_dtype = ADOP_F32)");
  for (int k = 0; k < n_cam; ++k) {
    const adop_intrinsics& K = cams[k].K;
    if (K.w < 1 || K.h < 1 || K.w > 16384 || K.h > 16384)
      return fail(ADOP_ERR_INVALID_ARG, "image size outside [1, 16384]");
    if ((K.w >> (params->levels - 1)) < 1 || (K.h >> (params->levels - 1)) < 1)
      return fail(ADOP_ERR_INVALID_ARG, "image too small for the pyramid");
    if (K.model != 0 && K.model != 1) return fail(ADOP_ERR_INVALID_ARG, "unknown camera model");
    for (int l = 0; l < params->levels; ++l)
      if (!frames[k].count[l] || ((uintptr_t)frames[k].count[l] & 3) != 0)
        return fail(ADOP_ERR_INVALID_ARG, "the environment map gradient needs the forward's count of every layer");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int k0 = 0; k0 < n_cam; k0 += kMaxCamsPerLaunch) {
    const int nc = (n_cam - k0) < kMaxCamsPerLaunch ? (n_cam - k0) : kMaxCamsPerLaunch;
    LaunchCams lc;
    for (int j = 0; j < nc; ++j) {
      const int k = k0 + j;
      set_camera_constants(lc.c[j], cams[k], params->levels, params->flags);
      lc.c[j].acc = frames[k].acc;
      lc.c[j].env_in_acc = frames[k].acc != nullptr ? 1 : 0;
      for (int l = 0; l < params->levels; ++l) {
        lc.c[j].cnt[l] = frames[k].count[l];
        lc.c[j].grad[l] = grad_image ? grad_image[(size_t)k * params->levels + l] : nullptr;
      }
    }
    PointArgs a{};
    a.env = params->env;
    a.env_w = params->env_w;
    a.env_h = params->env_h;
    a.levels = params->levels;
    a.ncam = nc;
    const cudaError_t e = timed("env_grad", s, [&] { return launch_env_grad(lc, a, c, grad_env, s); });
    if (e != cudaSuccess) return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
  }
  return ADOP_OK;
}
