// Gradients of the photometric camera model (Sec. 3.3) with respect to its
// per-image parameters: exposure EV, white balance, vignette centre and
// coefficients, and the response-curve LUT.
//
// One pass over the layer-0 pixels of every camera: each thread recomputes
// the pre-epilogue value I = sum / |Lambda| (or the environment map's or the
// background's value where no point landed), the
// epilogue's input x = I 2^-EV wb V(r) and the response's slope, and adds
//   dL/dEV  += g R'(x) x (-ln 2)          dL/dwb_ch += g R'(x) I 2^-EV V
//   dL/dc_v += g R'(x) I 2^-EV wb V'(r2) (-2 (p - c_v))
//   dL/da_k += g R'(x) I 2^-EV wb r2^k    dL/dlut[j], dL/dlut[j+1] += g (1-f), g f
// The nine sums go warp -> block -> fixed-order grid reduction; the LUT
// gradient is gathered per block in shared memory, then added globally.
#include <cuda_runtime.h>

#include "launch.h"

namespace adop {
namespace {

constexpr int kPhotoParams = 9;
constexpr int kPhotoBlocks = 256;  // blocks per camera
constexpr int kMaxLut = 4000;  // 3 x 4000 floats of shared memory fit the default 48 KB

struct PhotoArgs {
  float* gcrf[kMaxCamsPerLaunch];  // per camera: 3 x crf_n LUT gradient or NULL
  float* partials;                 // [ncam][kPhotoBlocks][9]
};

template <int C>
__global__ void __launch_bounds__(kThreads) k_photo_grad(const __grid_constant__ LaunchCams cams,
                                                         const __grid_constant__ PointArgs a,
                                                         const __grid_constant__ PhotoArgs pa) {
  pdl_entry();
  extern __shared__ float hist[];  // 3 x crf_n
  __shared__ float sm[kThreads / 32][kPhotoParams];
  const DevCam& cam = cams.c[blockIdx.y];
  float* gcrf = pa.gcrf[blockIdx.y];
  const bool lut = cam.crf != nullptr && cam.crf_n >= 2 && gcrf != nullptr;
  if (lut)
    for (int t = threadIdx.x; t < 3 * cam.crf_n; t += blockDim.x) hist[t] = 0.0f;
  __syncthreads();
  float acc[kPhotoParams];
#pragma unroll
  for (int k = 0; k < kPhotoParams; ++k) acc[k] = 0.0f;
  const int64_t np = (int64_t)cam.w * cam.h;
  const float* G = cam.grad[0];
  if (cam.epi && G) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
      const uint32_t n = cam.cnt[0][p];
      const int32_t u = (int32_t)(p % cam.w), v = (int32_t)(p / cam.w);
      const float ru = __fdiv_rn((float)u, (float)cam.w) - cam.vig_c[0];
      const float rv = __fdiv_rn((float)v, (float)cam.h) - cam.vig_c[1];
      const float r2 = ru * ru + rv * rv;
      const float vig = 1.0f + r2 * (cam.vig_a[0] + r2 * (cam.vig_a[1] + r2 * cam.vig_a[2]));
      const float dvig = cam.vig_a[0] + r2 * (2.0f * cam.vig_a[1] + 3.0f * r2 * cam.vig_a[2]);
      float empty[C];
      if (n == 0 && a.env) {  // the environment map's value, kept in acc by the forward
#pragma unroll
        for (int k = 0; k < C; ++k) empty[k] = cam.acc[p * C + k];
      } else if (n == 0) {
#pragma unroll
        for (int k = 0; k < C; ++k) empty[k] = a.background ? __ldg(a.background + k) : 0.0f;
      }
#pragma unroll
      for (int ch = 0; ch < (C < 3 ? C : 3); ++ch) {
        const float I = n ? __fdiv_rn(cam.acc[p * C + ch], (float)n) : empty[ch];
        const float g = __ldg(G + ch * np + p);
        int seg;
        float frac, slope;
        const float x = I * cam.ev_scale * cam.wb[ch] * vig;
        response(cam, ch, x, &slope, &seg, &frac);
        const float gx = g * slope;
        const float base = gx * I * cam.ev_scale;
        acc[0] += gx * x * -0.6931471805599453f;  // d 2^-EV / dEV = -ln 2 * 2^-EV
        acc[1 + ch] += base * vig;
        acc[4] += base * cam.wb[ch] * dvig * (-2.0f * ru);
        acc[5] += base * cam.wb[ch] * dvig * (-2.0f * rv);
        acc[6] += base * cam.wb[ch] * r2;
        acc[7] += base * cam.wb[ch] * r2 * r2;
        acc[8] += base * cam.wb[ch] * r2 * r2 * r2;
        if (lut && seg >= 0) {
          atomicAdd(hist + ch * cam.crf_n + seg, g * (1.0f - frac));
          atomicAdd(hist + ch * cam.crf_n + seg + 1, g * frac);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kPhotoParams; ++k) {
    float s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sm[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < kPhotoParams) {
    float s = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) s += sm[w][threadIdx.x];
    pa.partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kPhotoParams + threadIdx.x] = s;
  }
  if (lut)
    for (int t = threadIdx.x; t < 3 * cam.crf_n; t += blockDim.x)
      if (hist[t] != 0.0f) atomicAdd(gcrf + t, hist[t]);
}

// One block per camera; warp k sums parameter k over the block partials.
__global__ void k_photo_reduce(const float* __restrict__ partials, int blocks, float* grad_photo) {
  pdl_entry();
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  float s = 0.0f;
  for (int b = lane; b < blocks; b += 32) s += partials[((int64_t)blockIdx.x * blocks + b) * kPhotoParams + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) grad_photo[blockIdx.x * kPhotoParams + k] += s;
}

adop_status fail(adop_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

cudaError_t launch_photo(const LaunchCams& lc, const PointArgs& a, const PhotoArgs& pa, int c, size_t smem,
                         cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  ADOP_DISPATCH_C(c, e = launch_pdl(k_photo_grad<kC>, dim3(kPhotoBlocks, a.ncam), kThreads, smem, s, lc, a, pa));
  return e;
}

}  // namespace
}  // namespace adop

using namespace adop;

extern "C" {

size_t adop_photometric_workspace_bytes(int32_t n_cam) {
  if (n_cam < 1 || n_cam > ADOP_MAX_CAMERAS) return 0;
  return (size_t)n_cam * kPhotoBlocks * kPhotoParams * sizeof(float) + 256;
}

adop_status adop_photometric_backward(const adop_camera* cams, int32_t n_cam, const adop_params* params, int32_t c,
                                      const adop_frame* frames, const float* const* grad_image0, float* grad_photo,
                                      float* grad_crf, void* workspace, size_t workspace_bytes, adop_stream stream) {
  if (!cams || !params || !frames || !grad_photo) return fail(ADOP_ERR_INVALID_ARG, "NULL argument");
  if (n_cam < 1 || n_cam > ADOP_MAX_CAMERAS) return fail(ADOP_ERR_INVALID_ARG, "n_cam outside [1, 64]");
  if (!channels_supported(c)) return fail(ADOP_ERR_UNSUPPORTED, "channel count has no kernels");
  if (params->levels < 1 || params->levels > ADOP_MAX_LEVELS) return fail(ADOP_ERR_INVALID_ARG, "levels outside [1, 8]");
  if (params->grad_dtype != ADOP_F32)
    return fail(ADOP_ERR_UNSUPPORTED, "this call reads FP32 upstream gradients only (params->grad_dtype = ADOP_F32)");
  if (params->env && !env_size_ok(params->env_w, params->env_h))
    return fail(ADOP_ERR_INVALID_ARG, "env_w / env_h outside [1, 16384]");
  if (workspace_bytes < adop_photometric_workspace_bytes(n_cam) || !workspace || ((uintptr_t)workspace & 255))
    return fail(ADOP_ERR_INVALID_ARG, "workspace too small or not 256-byte aligned");
  size_t crf_off = 0;
  for (int k = 0; k < n_cam; ++k) {
    if (cams[k].K.w < 1 || cams[k].K.h < 1 || cams[k].K.w > 16384 || cams[k].K.h > 16384)
      return fail(ADOP_ERR_INVALID_ARG, "image size outside [1, 16384]");
    if (!frames[k].count[0] || !frames[k].acc)
      return fail(ADOP_ERR_INVALID_ARG, "photometric gradients need the forward's kept count/acc");
    if (cams[k].ph.crf_lut && (cams[k].ph.crf_n < 2 || cams[k].ph.crf_n > kMaxLut))
      return fail(ADOP_ERR_INVALID_ARG, "crf_n outside [2, 4000]");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* partials = reinterpret_cast<float*>(((uintptr_t)workspace + 255) / 256 * 256);
  cudaError_t e;
  for (int k0 = 0; k0 < n_cam; k0 += kMaxCamsPerLaunch) {
    const int nc = (n_cam - k0) < kMaxCamsPerLaunch ? (n_cam - k0) : kMaxCamsPerLaunch;
    LaunchCams lc;
    PhotoArgs pa{};
    int max_lut = 0;
    for (int j = 0; j < nc; ++j) {
      const int k = k0 + j;
      set_camera_constants(lc.c[j], cams[k], params->levels, params->flags);
      lc.c[j].cnt[0] = frames[k].count[0];
      lc.c[j].acc = frames[k].acc;
      lc.c[j].grad[0] = grad_image0 ? grad_image0[k] : nullptr;
      const int n = cams[k].ph.crf_lut ? cams[k].ph.crf_n : 0;
      pa.gcrf[j] = (grad_crf && n) ? grad_crf + crf_off : nullptr;
      crf_off += (size_t)3 * (n ? n : 0);
      max_lut = n > max_lut ? n : max_lut;
    }
    pa.partials = partials;
    PointArgs a{};
    a.background = params->background;
    a.env = params->env;
    a.env_w = params->env_w;
    a.env_h = params->env_h;
    a.levels = params->levels;
    a.ncam = nc;
    const size_t smem = sizeof(float) * 3 * (size_t)max_lut;
    if ((e = timed("photo_grad", s, [&] { return launch_photo(lc, a, pa, c, smem, s); })) != cudaSuccess)
      return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
    if ((e = launch_pdl(k_photo_reduce, dim3(nc), dim3(32 * kPhotoParams), 0, s, partials, (int)kPhotoBlocks,
                        grad_photo + (size_t)k0 * kPhotoParams)) != cudaSuccess)
      return fail(ADOP_ERR_CUDA, cudaGetErrorString(e));
  }
  return ADOP_OK;
}

}  // extern "C"
