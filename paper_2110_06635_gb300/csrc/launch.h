// Host-side launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "adop_device.cuh"

namespace adop {

// Screen-tile binning of the backward's visible points: block-local counts in
// shared memory up to kBinSmemTiles tiles per camera; the count kernel keeps
// each block's first slot within every tile's range in a [block][tile] table
// of bin_table_rows(n_cam) rows per camera (kBinTableBlocks blocks over all
// cameras at most), so that the scatter reads the layer masks only once.
constexpr int kBinSmemTiles = 8192;
constexpr int kBinTableBlocks = 1536;
inline int bin_table_rows(int ncam) { return (kBinTableBlocks + ncam - 1) / ncam; }

// Whether launch_pdl launches programmatically on the calling thread (default
// on); a PdlScope sets it for the launches of one API call.  Every kernel
// triggers its dependents as it starts, so the next grid is placed on the SMs
// during this grid's last wave and waits there.  That hides the launch gaps
// of a step of short kernels (5M-point view: 0.4240 -> 0.4193 ms), but where
// every block runs many grid-stride iterations the waiting blocks sit through
// a long, uneven last wave (120M-point frame: 2.305 -> 2.513 ms), so calls
// with more than kPdlMaxPointWork point-camera pairs launch in plain stream
// order.
bool& pdl_on();
struct PdlScope {
  bool prev;
  explicit PdlScope(bool on) : prev(pdl_on()) { pdl_on() = on; }
  ~PdlScope() { pdl_on() = prev; }
};
constexpr int64_t kPdlMaxPointWork = (int64_t)1 << 25;
inline bool pdl_for_points(int64_t n, int ncam) { return n * (int64_t)ncam <= kPdlMaxPointWork; }

// Launches kernel k on stream s as a programmatic dependent of the work before
// it in the stream (while pdl_on()).  The kernel must call pdl_entry() before
// its first memory access (a CPU test checks every kernel launched this way);
// it then runs in stream order, while its launch overlaps the end of the
// previous kernel.  In a captured CUDA graph the dependency becomes a
// programmatic edge.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_on() ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Arguments shared by the point kernels of one launch.  (The forward depth
// and accumulate passes read each camera's cloud from its DevCam instead of
// xyz/feat/normals/n here, so that a server batch can mix clouds.)
struct PointArgs {
  const float* xyz;
  const void* feat;
  const float* normals;  // non-NULL only when normal culling is on
  const float* background;
  const float* env;     // environment map (NULL = background): env_h x env_w texels of c floats
  int32_t env_w, env_h;
  const float* radius;  // stochastic discarding (NULL = off): world radius per point
  const float* beta;    // and uniform draw per point
  float g2;             // f32(gamma * gamma)
  int32_t log_desc;     // descriptors are stored as log values: blend exp(tau)
  int64_t n;
  int32_t levels;
  int32_t ncam;         // cameras in this launch (<= kMaxCamsPerLaunch)
  float znear;
  float a1;             // f32(1 + alpha)
  uint32_t flags;
  int32_t grad_dtype;   // adop_dtype of the upstream gradients (DevCam::grad)
};

// Backward outputs of one launch.
enum GradMode : int32_t { kGradAssign = 0, kGradAccumulate = 1, kGradAtomic = 2 };

struct BwdArgs {
  float* grad_feat;
  float* grad_xyz;
  float* partials;      // [ncam][12][blocks_x] pose (6) + intrinsics (6) block sums
  int32_t mode;         // GradMode
  int32_t all_projected;
  int32_t feat_out;     // adop_dtype of grad_feat (16-bit types only with kGradAssign)
};

int num_sms();
// Blocks for a point kernel's items pass: 8 per SM (two waves of its 4
// resident blocks), shared by the ncam cameras of grid.y.
int point_blocks(int64_t n, int ncam);
// Most pyramid pixels of any camera in the launch.
int64_t most_pixels(const LaunchCams& cams, const PointArgs& a);
// Most points of any camera's cloud in the launch (the forward point passes
// take each camera's cloud from its DevCam).
int64_t most_points(const LaunchCams& cams, const PointArgs& a);
// Grid of a grid-stride kernel k (kThreads threads, smem bytes of dynamic
// shared memory) over `work` items per camera: enough blocks for the work, at
// most `waves` whole waves of the kernel's resident blocks over all SMs,
// shared by the ncam cameras of grid.y.  Whole waves: a grid of 8 blocks per
// SM for a kernel that holds 5 ran its last 0.6 wave on 60% of the block
// slots.  Many waves rather than one: the work per item varies widely (a
// point outside the view costs a projection, a visible one up to four key
// reads and atomics), and with one long-lived block per slot the SMs whose
// blocks drew cheap items idle while the slowest block finishes; with many
// short blocks the block scheduler refills them.  (5M-point 1080p step: depth
// 72 -> 64 us and accumulate 100 -> 91 us at unchanged DRAM traffic and L2
// hit rate; more waves than these were slower again.)
constexpr int kPointWaves = 10;  // k_depth, k_accum
constexpr int kPixelWaves = 6;   // k_clear, k_normalize, k_bwd_prepass, k_env_*
dim3 stride_grid(const void* k, int64_t work, int ncam, int waves, size_t smem);

// launch_pdl of a grid-stride kernel over `work` items per camera, on the
// stride_grid() of that kernel.
template <typename... KArgs, typename... Args>
cudaError_t launch_strided(void (*k)(KArgs...), int64_t work, int ncam, int waves, size_t smem, cudaStream_t s,
                           Args&&... args) {
  return launch_pdl(k, stride_grid((const void*)k, work, ncam, waves, smem), dim3(kThreads), smem, s,
                    std::forward<Args>(args)...);
}

cudaError_t launch_clear(const LaunchCams& cams, const PointArgs& a, int c, cudaStream_t s);
cudaError_t launch_depth(const LaunchCams& cams, const PointArgs& a, cudaStream_t s);
cudaError_t launch_accum(const LaunchCams& cams, const PointArgs& a, int c, adop_dtype fd, cudaStream_t s);
cudaError_t launch_normalize(const LaunchCams& cams, const PointArgs& a, int c, adop_dtype od, cudaStream_t s);
cudaError_t launch_bwd_prepass(const LaunchCams& cams, const PointArgs& a, int c, cudaStream_t s);
cudaError_t launch_bwd_points(const LaunchCams& cams, const PointArgs& a, const BwdArgs& b, int c,
                              adop_dtype fd, int blocks_x, cudaStream_t s);
// Screen-tile binning of the visible points (backward): count, scan, scatter.
// (The binned point pass then also writes the zero gradients of the points
// that are in no Lambda when the mode is kGradAssign.)
cudaError_t launch_bin(const LaunchCams& cams, const PointArgs& a, const BwdArgs& b, int c, cudaStream_t s);
cudaError_t launch_bwd_reduce(const float* partials, int ncam, int blocks_x, float* grad_pose,
                              float* grad_intr, cudaStream_t s);

// Environment map (a.env non-NULL): k_env_fill samples it for every empty
// pixel, stores the value in acc (where the backward pass and the
// photometric gradients read it) and, where image[l] is set, writes the
// pixel (through the epilogue at layer 0); k_env_grad scatters dL/dE.
cudaError_t launch_env_fill(const LaunchCams& cams, const PointArgs& a, int c, adop_dtype od, cudaStream_t s);
cudaError_t launch_env_grad(const LaunchCams& cams, const PointArgs& a, int c, float* grad_env, cudaStream_t s);

// Pixels of a w x h pyramid of `levels` layers (w_l = w >> l, h_l = h >> l);
// off (if given) receives the first pixel of every layer and the total.
inline int64_t pyramid_pixels(int32_t w, int32_t h, int levels, int64_t* off) {
  int64_t o = 0;
  for (int l = 0; l < levels; ++l) {
    if (off) off[l] = o;
    o += (int64_t)(w >> l) * (int64_t)(h >> l);
  }
  if (off)
    for (int l = levels; l <= ADOP_MAX_LEVELS; ++l) off[l] = o;
  return o;
}

// Camera constants of a DevCam (pose, intrinsics, layer offsets, photometric
// epilogue); buffer pointers are left to the caller.
void set_camera_constants(DevCam& d, const adop_camera& cam, int levels, uint32_t flags);

// Set the calling thread's adop_last_error() message.
void set_last_error(const char* msg);

// Kernel timing for adop_profile_enable / adop_profile_collect: events on the
// launch stream around one launch (prof_begin returns -1 when timing is off).
int prof_begin(const char* name, cudaStream_t s);
void prof_end(int rec, cudaStream_t s);

template <class F>
cudaError_t timed(const char* name, cudaStream_t s, F&& launch) {
  const int rec = prof_begin(name, s);
  const cudaError_t e = launch();
  prof_end(rec, s);
  return e;
}

// Environment map sizes the lookup accepts (texel indices stay in int32).
inline bool env_size_ok(int32_t w, int32_t h) { return w >= 1 && h >= 1 && w <= 16384 && h <= 16384; }

// Channel counts with compiled kernels.
inline bool channels_supported(int c) { return c == 1 || c == 2 || c == 3 || c == 4 || c == 8 || c == 16; }

}  // namespace adop

// Dispatch a runtime channel count to a compile-time constant kC.
#define ADOP_DISPATCH_C(c, ...)                     \
  switch (c) {                                      \
    case 1: { constexpr int kC = 1; __VA_ARGS__; break; }  \
    case 2: { constexpr int kC = 2; __VA_ARGS__; break; }  \
    case 3: { constexpr int kC = 3; __VA_ARGS__; break; }  \
    case 4: { constexpr int kC = 4; __VA_ARGS__; break; }  \
    case 8: { constexpr int kC = 8; __VA_ARGS__; break; }  \
    case 16: { constexpr int kC = 16; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;          \
  }

#define ADOP_DISPATCH_T(dt, T, ...)                                   \
  switch (dt) {                                                       \
    case ADOP_F32: { using T = float; __VA_ARGS__; break; }           \
    case ADOP_BF16: { using T = __nv_bfloat16; __VA_ARGS__; break; }  \
    case ADOP_F16: { using T = __half; __VA_ARGS__; break; }          \
    default: return cudaErrorInvalidValue;                            \
  }
