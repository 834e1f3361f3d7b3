// The extern "C" entry points declared in include/adop.h: argument
// validation (all on the host, before any launch), the workspace layout, and
// the sequence of kernel launches for the forward and backward passes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"

namespace adop {
namespace {

thread_local std::string g_last_error;

adop_status fail(adop_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
adop_status fail(adop_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

adop_status cuda_fail(cudaError_t e, const char* what) {
  return fail(ADOP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// kernel timing (adop_profile_enable / adop_profile_collect)
// ---------------------------------------------------------------------------
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;
std::vector<std::string> g_prof_names;

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_id(const char* name) {
  for (size_t i = 0; i < g_prof_names.size(); ++i)
    if (g_prof_names[i] == name) return (int)i;
  g_prof_names.emplace_back(name);
  return (int)g_prof_names.size() - 1;
}


constexpr size_t kAlign = 256;
constexpr int kMaxPartialBlocks = 4096;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool finite(float v) { return std::isfinite(v); }

// Workspace: per camera [keys | counts | sums | point layer masks | backward
// pixel info | pixel-major upstream gradient | tile counts | tile offsets |
// tile-ordered point list | the depth pass's per-point layer bytes], then the
// pose/intrinsics block partials.
struct WsLayout {
  size_t key[ADOP_MAX_CAMERAS], cnt[ADOP_MAX_CAMERAS], acc[ADOP_MAX_CAMERAS], vis[ADOP_MAX_CAMERAS];
  size_t info[ADOP_MAX_CAMERAS], gpm[ADOP_MAX_CAMERAS];
  size_t bin_count[ADOP_MAX_CAMERAS], bin_off[ADOP_MAX_CAMERAS], bin_list[ADOP_MAX_CAMERAS];
  size_t early[ADOP_MAX_CAMERAS], bin_table[ADOP_MAX_CAMERAS];
  int32_t bin_rows;
  bool binning;
  size_t partials;
  size_t total;
};

WsLayout layout(const adop_points* pts, const adop_camera* cams, int32_t n_cam, const adop_params* prm) {
  WsLayout L{};
  size_t o = 0;
  const int c = pts->c;
  for (int k = 0; k < n_cam; ++k) {
    const int64_t px = pyramid_pixels(cams[k].K.w, cams[k].K.h, prm->levels, nullptr);
    L.key[k] = o;
    o = align_up(o + (size_t)px * 8);
    L.cnt[k] = o;
    o = align_up(o + (size_t)px * 4);
    L.acc[k] = o;
    o = align_up(o + (size_t)px * c * 4);
    L.vis[k] = o;
    o = align_up(o + (size_t)pts->n * 4);
    L.info[k] = o;
    o = align_up(o + (size_t)px * 16);
    L.gpm[k] = o;
    o = align_up(o + (size_t)px * g_stride(c) * 4);
    const size_t tiles = (size_t)tiles_along(cams[k].K.w) * (size_t)tiles_along(cams[k].K.h);
    L.bin_count[k] = o;
    o = align_up(o + tiles * 4);
    L.bin_off[k] = o;
    o = align_up(o + (tiles + 1) * 4);
    L.bin_list[k] = o;
    o = align_up(o + (size_t)pts->n * 4);
    L.early[k] = o;
    o = align_up(o + (size_t)pts->n);
    L.bin_table[k] = o;
    if (tiles <= (size_t)kBinSmemTiles) o = align_up(o + (size_t)bin_table_rows(n_cam) * tiles * 4);
  }
  L.bin_rows = bin_table_rows(n_cam);
  L.binning = true;
  L.partials = o;
  o = align_up(o + (size_t)n_cam * kMaxPartialBlocks * 12 * 4);
  L.total = o;
  return L;
}

adop_status validate_common(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                            const adop_params* prm) {
  if (!pts || !cams || !prm) return fail(ADOP_ERR_INVALID_ARG, "points, cameras and params must not be NULL");
  if (n_cam < 1 || n_cam > ADOP_MAX_CAMERAS)
    return fail(ADOP_ERR_INVALID_ARG, "n_cam = %d outside [1, %d]", n_cam, ADOP_MAX_CAMERAS);
  if (pts->n < 0 || pts->n >= ((int64_t)1 << 31))
    return fail(ADOP_ERR_INVALID_ARG, "point count %lld outside [0, 2^31)", (long long)pts->n);
  if (pts->c < 1 || pts->c > 16) return fail(ADOP_ERR_INVALID_ARG, "channel count %d outside [1, 16]", pts->c);
  if (!channels_supported(pts->c))
    return fail(ADOP_ERR_UNSUPPORTED, "channel count %d has no kernels (use 1, 2, 3, 4, 8 or 16)", pts->c);
  if (pts->feat_dtype != ADOP_F32 && pts->feat_dtype != ADOP_BF16 && pts->feat_dtype != ADOP_F16)
    return fail(ADOP_ERR_INVALID_ARG, "unknown feature dtype %d", (int)pts->feat_dtype);
  if (pts->n > 0) {
    if (!pts->xyz || !pts->feat) return fail(ADOP_ERR_INVALID_ARG, "xyz and feat must not be NULL");
    if (((uintptr_t)pts->xyz & 3) != 0) return fail(ADOP_ERR_INVALID_ARG, "xyz must be 4-byte aligned");
    if (((uintptr_t)pts->feat & 15) != 0) return fail(ADOP_ERR_INVALID_ARG, "feat must be 16-byte aligned");
  }
  if (prm->levels < 1 || prm->levels > ADOP_MAX_LEVELS)
    return fail(ADOP_ERR_INVALID_ARG, "levels = %d outside [1, %d]", prm->levels, ADOP_MAX_LEVELS);
  if (!finite(prm->alpha) || prm->alpha < 0.0f) return fail(ADOP_ERR_INVALID_ARG, "alpha must be finite and >= 0");
  if (!finite(prm->znear) || prm->znear < 0.0f) return fail(ADOP_ERR_INVALID_ARG, "znear must be finite and >= 0");
  if (prm->flags & ~(uint32_t)(ADOP_FLAG_NORMAL_CULL | ADOP_FLAG_GRAD_ALL_PROJECTED | ADOP_FLAG_EPILOGUE |
                               ADOP_FLAG_GRAD_ASSIGN | ADOP_FLAG_DISCARD | ADOP_FLAG_LEAKY_CRF |
                               ADOP_FLAG_LOG_DESCRIPTORS))
    return fail(ADOP_ERR_INVALID_ARG, "unknown flag bits 0x%x", prm->flags);
  for (adop_dtype d : {prm->grad_dtype, prm->grad_feat_dtype})
    if (d != ADOP_F32 && d != ADOP_BF16 && d != ADOP_F16)
      return fail(ADOP_ERR_INVALID_ARG, "unknown gradient dtype %d", (int)d);
  if (prm->flags & ADOP_FLAG_DISCARD) {
    if (!(prm->gamma > 0.0f) || !finite(prm->gamma))
      return fail(ADOP_ERR_INVALID_ARG, "ADOP_FLAG_DISCARD needs a finite gamma > 0");
    if (pts->n > 0 && (!pts->radius || !pts->beta))
      return fail(ADOP_ERR_INVALID_ARG, "ADOP_FLAG_DISCARD needs per-point radius and beta");
  }
  if (prm->env) {
    if (!env_size_ok(prm->env_w, prm->env_h))
      return fail(ADOP_ERR_INVALID_ARG, "environment map %dx%d outside [1, 16384]^2", prm->env_w, prm->env_h);
    if (((uintptr_t)prm->env & 15) != 0) return fail(ADOP_ERR_INVALID_ARG, "env must be 16-byte aligned");
  }
  if ((prm->flags & ADOP_FLAG_NORMAL_CULL) && pts->n > 0 && !pts->normals)
    return fail(ADOP_ERR_INVALID_ARG, "ADOP_FLAG_NORMAL_CULL needs normals");
  for (int k = 0; k < n_cam; ++k) {
    const adop_intrinsics& K = cams[k].K;
    if (K.w < 1 || K.h < 1 || K.w > 16384 || K.h > 16384)
      return fail(ADOP_ERR_INVALID_ARG, "camera %d: image size %dx%d outside [1, 16384]", k, K.w, K.h);
    if ((K.w >> (prm->levels - 1)) < 1 || (K.h >> (prm->levels - 1)) < 1)
      return fail(ADOP_ERR_INVALID_ARG, "camera %d: %dx%d too small for %d levels", k, K.w, K.h, prm->levels);
    if (K.model != 0 && K.model != 1)
      return fail(ADOP_ERR_INVALID_ARG, "camera %d: unknown camera model %d", k, K.model);
    const float kv[9] = {K.fx, K.fy, K.cx, K.cy, K.k1, K.k2, K.k3, K.p1, K.p2};
    for (float v : kv)
      if (!finite(v)) return fail(ADOP_ERR_INVALID_ARG, "camera %d: non-finite intrinsics", k);
    for (int j = 0; j < 9; ++j)
      if (!finite(cams[k].T.R[j])) return fail(ADOP_ERR_INVALID_ARG, "camera %d: non-finite rotation", k);
    for (int j = 0; j < 3; ++j)
      if (!finite(cams[k].T.t[j])) return fail(ADOP_ERR_INVALID_ARG, "camera %d: non-finite translation", k);
    const adop_photometric& ph = cams[k].ph;
    if ((prm->flags & ADOP_FLAG_EPILOGUE) && ph.enabled) {
      if (ph.crf_lut && ph.crf_n < 2) return fail(ADOP_ERR_INVALID_ARG, "camera %d: crf_n must be >= 2", k);
      const float pv[9] = {ph.ev, ph.wb[0], ph.wb[1], ph.wb[2], ph.vig_c[0], ph.vig_c[1], ph.vig_a[0], ph.vig_a[1],
                           ph.vig_a[2]};
      for (float v : pv)
        if (!finite(v)) return fail(ADOP_ERR_INVALID_ARG, "camera %d: non-finite photometric parameter", k);
    }
  }
  return ADOP_OK;
}

// state_given: 1 if key/count/acc are all set, 0 if all NULL, -1 if mixed.
int state_given(const adop_frame& f, int levels) {
  int set = 0, unset = 0;
  for (int l = 0; l < levels; ++l) {
    (f.key[l] ? set : unset)++;
    (f.count[l] ? set : unset)++;
  }
  (f.acc ? set : unset)++;
  if (unset == 0) return 1;
  if (set == 0) return 0;
  return -1;
}

adop_status validate_frames(const adop_frame* frames, int32_t n_cam, const adop_params* prm, bool need_out) {
  if (!frames) return fail(ADOP_ERR_INVALID_ARG, "frames must not be NULL");
  for (int k = 0; k < n_cam; ++k) {
    const adop_frame& f = frames[k];
    const int sg = state_given(f, prm->levels);
    if (sg < 0) return fail(ADOP_ERR_INVALID_ARG, "camera %d: key/count/acc must be all set or all NULL", k);
    if (sg == 1 && ((uintptr_t)f.acc & 15) != 0)
      return fail(ADOP_ERR_INVALID_ARG, "camera %d: acc must be 16-byte aligned", k);
    if (sg == 0 && f.vis)
      return fail(ADOP_ERR_INVALID_ARG, "camera %d: vis needs key/count/acc", k);
    if (sg == 1)
      for (int l = 0; l < prm->levels; ++l)
        if (((uintptr_t)f.key[l] & 7) != 0 || ((uintptr_t)f.count[l] & 3) != 0 || ((uintptr_t)f.vis & 3) != 0)
          return fail(ADOP_ERR_INVALID_ARG, "camera %d: misaligned key/count buffer", k);
    if (need_out && f.out_dtype != ADOP_F32 && f.out_dtype != ADOP_BF16 && f.out_dtype != ADOP_F16)
      return fail(ADOP_ERR_INVALID_ARG, "camera %d: unknown output dtype %d", k, (int)f.out_dtype);
  }
  return ADOP_OK;
}

adop_status validate_ws(void* ws, size_t ws_bytes, size_t need) {
  if (ws_bytes < need)
    return fail(ADOP_ERR_OUT_OF_MEMORY, "workspace has %zu bytes, %zu needed", ws_bytes, need);
  if (!ws) return fail(ADOP_ERR_INVALID_ARG, "workspace must not be NULL");
  if (((uintptr_t)ws & (kAlign - 1)) != 0) return fail(ADOP_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  return ADOP_OK;
}

// Fill the device-side camera description.  State buffers come from the
// frame if given, else from the workspace.
void fill_cam(DevCam& d, const adop_camera& cam, const adop_frame* f, bool use_frame_state, const WsLayout& L,
              int k, char* ws, const adop_points* pts, const adop_params* prm) {
  set_camera_constants(d, cam, prm->levels, prm->flags);
  d.xyz = pts->xyz;
  d.feat = pts->feat;
  d.normals = (prm->flags & ADOP_FLAG_NORMAL_CULL) ? pts->normals : nullptr;
  d.n = pts->n;
  for (int l = 0; l < prm->levels; ++l) {
    if (use_frame_state) {
      d.key[l] = reinterpret_cast<unsigned long long*>(f->key[l]);
      d.cnt[l] = f->count[l];
    } else {
      d.key[l] = reinterpret_cast<unsigned long long*>(ws + L.key[k]) + d.off[l];
      d.cnt[l] = reinterpret_cast<uint32_t*>(ws + L.cnt[k]) + d.off[l];
    }
    d.image[l] = f ? f->image[l] : nullptr;
  }
  d.acc = use_frame_state ? f->acc : reinterpret_cast<float*>(ws + L.acc[k]);
  d.vis = use_frame_state ? f->vis : reinterpret_cast<uint32_t*>(ws + L.vis[k]);
  d.early = reinterpret_cast<uint8_t*>(ws + L.early[k]);
  d.info = reinterpret_cast<float*>(ws + L.info[k]);
  d.gpm = reinterpret_cast<float*>(ws + L.gpm[k]);
  if (L.binning) {
    d.bin_count = reinterpret_cast<int32_t*>(ws + L.bin_count[k]);
    d.bin_off = reinterpret_cast<int32_t*>(ws + L.bin_off[k]);
    d.bin_list = reinterpret_cast<int32_t*>(ws + L.bin_list[k]);
    d.bin_table = reinterpret_cast<int32_t*>(ws + L.bin_table[k]);
    d.bin_rows = L.bin_rows;
  }
}

PointArgs point_args(const adop_points* pts, const adop_params* prm, int ncam) {
  PointArgs a{};
  a.xyz = pts->xyz;
  a.feat = pts->feat;
  a.normals = (prm->flags & ADOP_FLAG_NORMAL_CULL) ? pts->normals : nullptr;
  a.background = prm->background;
  a.env = prm->env;
  a.env_w = prm->env_w;
  a.env_h = prm->env_h;
  a.radius = (prm->flags & ADOP_FLAG_DISCARD) ? pts->radius : nullptr;
  a.beta = (prm->flags & ADOP_FLAG_DISCARD) ? pts->beta : nullptr;
  a.g2 = prm->gamma * prm->gamma;
  a.log_desc = (prm->flags & ADOP_FLAG_LOG_DESCRIPTORS) ? 1 : 0;
  a.n = pts->n;
  a.levels = prm->levels;
  a.ncam = ncam;
  a.znear = prm->znear;
  a.a1 = 1.0f + prm->alpha;
  a.flags = prm->flags;
  a.grad_dtype = prm->grad_dtype;
  return a;
}

// The storage type of grad_feat: 16-bit types only where each point's dL/dtau
// is complete before its one store (assigned, one camera).
adop_status check_grad_feat_dtype(const adop_params* prm, int32_t n_cam) {
  if (prm->grad_feat_dtype != ADOP_F32 && (!(prm->flags & ADOP_FLAG_GRAD_ASSIGN) || n_cam != 1))
    return fail(ADOP_ERR_UNSUPPORTED,
                "a 16-bit grad_feat needs ADOP_FLAG_GRAD_ASSIGN and one camera (several cameras and += sum in FP32)");
  return ADOP_OK;
}

// Forward passes (clear, depth, accumulate[, normalize]) for cameras [k0, k0+nc).
adop_status render_chunk(const adop_points* pts, const adop_camera* cams, int k0, int nc, const adop_params* prm,
                         const adop_frame* frames, bool frames_state, const WsLayout& L, char* ws, bool normalize,
                         cudaStream_t s) {
  LaunchCams lc;
  for (int j = 0; j < nc; ++j) {
    const int k = k0 + j;
    const bool use_frame = frames_state && state_given(frames[k], prm->levels) == 1;
    fill_cam(lc.c[j], cams[k], frames ? &frames[k] : nullptr, use_frame, L, k, ws, pts, prm);
    if (!normalize)
      for (int l = 0; l < ADOP_MAX_LEVELS; ++l) lc.c[j].image[l] = nullptr;
  }
  const PointArgs a = point_args(pts, prm, nc);
  cudaError_t e;
  if ((e = timed("clear", s, [&] { return launch_clear(lc, a, pts->c, s); })) != cudaSuccess)
    return cuda_fail(e, "clear launch");
  if ((e = timed("depth", s, [&] { return launch_depth(lc, a, s); })) != cudaSuccess)
    return cuda_fail(e, "depth pass launch");
  if ((e = timed("accumulate", s, [&] { return launch_accum(lc, a, pts->c, pts->feat_dtype, s); })) != cudaSuccess)
    return cuda_fail(e, "accumulate launch");
  if (normalize) {
    // all cameras of a launch share one output dtype: group by dtype
    for (int dt = 0; dt < 3; ++dt) {
      LaunchCams sub;
      int m = 0;
      for (int j = 0; j < nc; ++j)
        if ((int)frames[k0 + j].out_dtype == dt) sub.c[m++] = lc.c[j];
      if (m == 0) continue;
      PointArgs sa = a;
      sa.ncam = m;
      if ((e = timed("normalize", s, [&] { return launch_normalize(sub, sa, pts->c, (adop_dtype)dt, s); })) !=
          cudaSuccess)
        return cuda_fail(e, "normalize launch");
      if (prm->env &&
          (e = timed("env_fill", s, [&] { return launch_env_fill(sub, sa, pts->c, (adop_dtype)dt, s); })) !=
              cudaSuccess)
        return cuda_fail(e, "environment map launch");
    }
  }
  return ADOP_OK;
}

// ---------------------------------------------------------------------------
// scratch of adop_render_backward_noalloc: one static device array
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

void set_last_error(const char* msg) { g_last_error = msg; }

bool& pdl_on() {
  static thread_local bool on = true;
  return on;
}

int prof_begin(const char* name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return -1;
  ProfRec r{prof_id(name), prof_event(), prof_event()};
  cudaEventRecord(r.a, s);
  g_prof_recs.push_back(r);
  return (int)g_prof_recs.size() - 1;
}

void prof_end(int rec, cudaStream_t s) {
  if (rec < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (rec < (int)g_prof_recs.size()) cudaEventRecord(g_prof_recs[rec].b, s);
}

void set_camera_constants(DevCam& d, const adop_camera& cam, int levels, uint32_t flags) {
  memset(&d, 0, sizeof(d));
  memcpy(d.R, cam.T.R, sizeof(d.R));
  memcpy(d.t, cam.T.t, sizeof(d.t));
  d.fx = cam.K.fx; d.fy = cam.K.fy; d.cx = cam.K.cx; d.cy = cam.K.cy;
  d.k1 = cam.K.k1; d.k2 = cam.K.k2; d.k3 = cam.K.k3; d.p1 = cam.K.p1; d.p2 = cam.K.p2;
  d.ifx = (float)(1.0 / (double)cam.K.fx);
  d.ify = (float)(1.0 / (double)cam.K.fy);
  d.w = cam.K.w;
  d.h = cam.K.h;
  d.model = cam.K.model;
  pyramid_pixels(d.w, d.h, levels, d.off);
  d.tiles_x = tiles_along(d.w);
  d.tiles = d.tiles_x * tiles_along(d.h);
  const adop_photometric& ph = cam.ph;
  d.epi = ((flags & ADOP_FLAG_EPILOGUE) && ph.enabled) ? 1 : 0;
  d.leaky = (flags & ADOP_FLAG_LEAKY_CRF) ? 1 : 0;
  d.ev_scale = (float)std::exp2(-(double)ph.ev);
  for (int j = 0; j < 3; ++j) {
    d.wb[j] = ph.wb[j];
    d.vig_a[j] = ph.vig_a[j];
  }
  d.vig_c[0] = ph.vig_c[0];
  d.vig_c[1] = ph.vig_c[1];
  d.crf = ph.crf_lut;
  d.crf_n = ph.crf_n;
}

}  // namespace adop

// File scope, as the entry point's contract states: every device that loads
// the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ADOP_NOALLOC_SCRATCH_BYTES];

namespace adop {
namespace {

// Device address of the static scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
adop_status noalloc_scratch(char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(ADOP_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<char*>(g_scratch_ptr[dev]);
  return ADOP_OK;
}

// Scratch layout of the no-allocation backward: records of every camera,
// then the block partials of one launch chunk.
WsLayout noalloc_layout(const adop_points* pts, const adop_camera* cams, int32_t n_cam, const adop_params* prm) {
  WsLayout L{};
  size_t o = 0;
  for (int k = 0; k < n_cam; ++k) {
    const int64_t px = pyramid_pixels(cams[k].K.w, cams[k].K.h, prm->levels, nullptr);
    L.info[k] = o;
    o = align_up(o + (size_t)px * 16);
    L.gpm[k] = o;
    o = align_up(o + (size_t)px * g_stride(pts->c) * 4);
  }
  L.partials = o;
  const int chunk = n_cam < kMaxCamsPerLaunch ? n_cam : kMaxCamsPerLaunch;
  o = align_up(o + (size_t)chunk * kMaxPartialBlocks * 12 * 4);
  L.total = o;
  return L;
}

}  // namespace
}  // namespace adop

using namespace adop;

extern "C" {

const char* adop_last_error(void) { return g_last_error.c_str(); }

int32_t adop_abi_version(void) { return ADOP_ABI_VERSION; }

adop_status adop_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return ADOP_OK;
}

int32_t adop_profile_collect(adop_kernel_stat* out, int32_t max) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::vector<int64_t> launches(g_prof_names.size(), 0);
  std::vector<double> ms(g_prof_names.size(), 0.0);
  cudaError_t err = cudaSuccess;
  for (const ProfRec& r : g_prof_recs) {
    float t = 0.0f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) err = e;
    launches[r.id] += 1;
    ms[r.id] += t;
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_recs.clear();
  if (err != cudaSuccess) {
    cuda_fail(err, "profile collect");
    return -1;
  }
  int32_t m = 0;
  for (size_t i = 0; i < g_prof_names.size() && m < max; ++i) {
    if (launches[i] == 0) continue;
    if (out) {
      memset(out[m].name, 0, sizeof(out[m].name));
      strncpy(out[m].name, g_prof_names[i].c_str(), sizeof(out[m].name) - 1);
      out[m].launches = launches[i];
      out[m].total_ms = ms[i];
    }
    ++m;
  }
  return m;
}

size_t adop_workspace_bytes(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                            const adop_params* params) {
  if (validate_common(pts, cams, n_cam, params) != ADOP_OK) return 0;
  return layout(pts, cams, n_cam, params).total;
}

adop_status adop_render_forward(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                                const adop_params* params, adop_frame* frames, void* workspace,
                                size_t workspace_bytes, adop_stream stream) {
  adop_status st;
  if ((st = validate_common(pts, cams, n_cam, params)) != ADOP_OK) return st;
  if ((st = validate_frames(frames, n_cam, params, true)) != ADOP_OK) return st;
  const WsLayout L = layout(pts, cams, n_cam, params);
  if ((st = validate_ws(workspace, workspace_bytes, L.total)) != ADOP_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const PdlScope pdl(pdl_for_points(pts->n, n_cam < kMaxCamsPerLaunch ? n_cam : kMaxCamsPerLaunch));
  char* ws = static_cast<char*>(workspace);
  for (int k0 = 0; k0 < n_cam; k0 += kMaxCamsPerLaunch) {
    const int nc = (n_cam - k0) < kMaxCamsPerLaunch ? (n_cam - k0) : kMaxCamsPerLaunch;
    if ((st = render_chunk(pts, cams, k0, nc, params, frames, true, L, ws, true, s)) != ADOP_OK) return st;
  }
  g_last_error.clear();
  return ADOP_OK;
}

adop_status adop_render_backward(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                                 const adop_params* params, const adop_frame* frames,
                                 const float* const* grad_image, float* grad_feat, float* grad_xyz,
                                 float* grad_pose, float* grad_intr, void* workspace, size_t workspace_bytes,
                                 adop_stream stream) {
  adop_status st;
  if ((st = validate_common(pts, cams, n_cam, params)) != ADOP_OK) return st;
  if ((st = validate_frames(frames, n_cam, params, false)) != ADOP_OK) return st;
  const WsLayout L = layout(pts, cams, n_cam, params);
  if ((st = validate_ws(workspace, workspace_bytes, L.total)) != ADOP_OK) return st;
  if (pts->n > 0 && grad_feat && ((uintptr_t)grad_feat & 15) != 0)
    return fail(ADOP_ERR_INVALID_ARG, "grad_feat must be 16-byte aligned");
  if (pts->n > 0 && grad_xyz && ((uintptr_t)grad_xyz & 3) != 0)
    return fail(ADOP_ERR_INVALID_ARG, "grad_xyz must be 4-byte aligned");
  if ((st = check_grad_feat_dtype(params, n_cam)) != ADOP_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const PdlScope pdl(pdl_for_points(pts->n, n_cam < kMaxCamsPerLaunch ? n_cam : kMaxCamsPerLaunch));
  char* ws = static_cast<char*>(workspace);
  const bool assign = (params->flags & ADOP_FLAG_GRAD_ASSIGN) != 0;
  int mode = (n_cam == 1) ? (assign ? kGradAssign : kGradAccumulate) : kGradAtomic;
  cudaError_t e;
  if (assign && n_cam > 1 && pts->n > 0) {
    if (grad_feat && (e = cudaMemsetAsync(grad_feat, 0, (size_t)pts->n * pts->c * 4, s)) != cudaSuccess)
      return cuda_fail(e, "clear grad_feat");
    if (grad_xyz && (e = cudaMemsetAsync(grad_xyz, 0, (size_t)pts->n * 12, s)) != cudaSuccess)
      return cuda_fail(e, "clear grad_xyz");
  }
  const bool want_pose = grad_pose || grad_intr;
  for (int k0 = 0; k0 < n_cam; k0 += kMaxCamsPerLaunch) {
    const int nc = (n_cam - k0) < kMaxCamsPerLaunch ? (n_cam - k0) : kMaxCamsPerLaunch;
    // re-render cameras whose forward state was not kept (the paper's backward
    // re-renders all points since Lambda is never stored)
    {
      LaunchCams rc;
      int m = 0;
      int idx[kMaxCamsPerLaunch];
      for (int j = 0; j < nc; ++j)
        if (state_given(frames[k0 + j], params->levels) == 0) idx[m++] = k0 + j;
      if (m > 0) {
        for (int j = 0; j < m; ++j) fill_cam(rc.c[j], cams[idx[j]], nullptr, false, L, idx[j], ws, pts, params);
        const PointArgs a = point_args(pts, params, m);
        if ((e = timed("clear", s, [&] { return launch_clear(rc, a, pts->c, s); })) != cudaSuccess)
          return cuda_fail(e, "clear launch");
        if ((e = timed("depth", s, [&] { return launch_depth(rc, a, s); })) != cudaSuccess)
          return cuda_fail(e, "depth pass launch");
        if ((e = timed("accumulate", s, [&] { return launch_accum(rc, a, pts->c, pts->feat_dtype, s); })) !=
            cudaSuccess)
          return cuda_fail(e, "accumulate launch");
        if (params->env &&
            (e = timed("env_fill", s, [&] { return launch_env_fill(rc, a, pts->c, ADOP_F32, s); })) != cudaSuccess)
          return cuda_fail(e, "environment map launch");
      }
    }
    LaunchCams lc;
    for (int j = 0; j < nc; ++j) {
      const int k = k0 + j;
      const bool use_frame = state_given(frames[k], params->levels) == 1;
      fill_cam(lc.c[j], cams[k], &frames[k], use_frame, L, k, ws, pts, params);
      for (int l = 0; l < params->levels; ++l) {
        lc.c[j].grad[l] = grad_image ? grad_image[k * params->levels + l] : nullptr;
        lc.c[j].image[l] = nullptr;
      }
    }
    const PointArgs a = point_args(pts, params, nc);
    if ((e = timed("bwd_prepass", s, [&] { return launch_bwd_prepass(lc, a, pts->c, s); })) != cudaSuccess)
      return cuda_fail(e, "backward prepass launch");
    if (pts->n == 0) continue;
    const int bx = point_blocks(pts->n, nc) < kMaxPartialBlocks ? point_blocks(pts->n, nc) : kMaxPartialBlocks;
    BwdArgs b{};
    b.grad_feat = grad_feat;
    b.grad_xyz = grad_xyz;
    b.partials = want_pose ? reinterpret_cast<float*>(ws + L.partials) : nullptr;
    b.mode = mode;
    b.all_projected = (params->flags & ADOP_FLAG_GRAD_ALL_PROJECTED) ? 1 : 0;
    b.feat_out = params->grad_feat_dtype;
    bool dense = !b.all_projected;
    for (int j = 0; j < nc; ++j) dense = dense && lc.c[j].vis != nullptr;
    if (dense) {
      if ((e = timed("bwd_bin", s, [&] { return launch_bin(lc, a, b, pts->c, s); })) != cudaSuccess)
        return cuda_fail(e, "backward binning launch");
    } else {
      for (int j = 0; j < nc; ++j) lc.c[j].bin_list = nullptr;
    }
    if ((e = timed("bwd_points", s, [&] { return launch_bwd_points(lc, a, b, pts->c, pts->feat_dtype, bx, s); })) !=
        cudaSuccess)
      return cuda_fail(e, "backward point pass launch");
    if (want_pose && (e = timed("bwd_reduce", s, [&] {
                        return launch_bwd_reduce(b.partials, nc, bx, grad_pose ? grad_pose + 6 * k0 : nullptr,
                                                 grad_intr ? grad_intr + 6 * k0 : nullptr, s);
                      })) != cudaSuccess)
      return cuda_fail(e, "backward reduce launch");
  }
  g_last_error.clear();
  return ADOP_OK;
}

adop_status adop_render_backward_noalloc(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                                         const adop_params* params, const adop_frame* frames,
                                         const float* const* grad_image, float* grad_feat, float* grad_xyz,
                                         float* grad_pose, float* grad_intr, adop_stream stream) {
  adop_status st;
  if ((st = validate_common(pts, cams, n_cam, params)) != ADOP_OK) return st;
  if ((st = validate_frames(frames, n_cam, params, false)) != ADOP_OK) return st;
  for (int k = 0; k < n_cam; ++k)
    if (state_given(frames[k], params->levels) != 1)
      return fail(ADOP_ERR_INVALID_ARG,
                  "camera %d: the no-allocation backward needs the forward's kept key/count/acc", k);
  const WsLayout L = noalloc_layout(pts, cams, n_cam, params);
  if (L.total > ADOP_NOALLOC_SCRATCH_BYTES)
    return fail(ADOP_ERR_OUT_OF_MEMORY,
                "the no-allocation backward needs %zu bytes of scratch, its static array holds %zu; "
                "use adop_render_backward with a workspace",
                L.total, (size_t)ADOP_NOALLOC_SCRATCH_BYTES);
  if (pts->n > 0 && grad_feat && ((uintptr_t)grad_feat & 15) != 0)
    return fail(ADOP_ERR_INVALID_ARG, "grad_feat must be 16-byte aligned");
  if (pts->n > 0 && grad_xyz && ((uintptr_t)grad_xyz & 3) != 0)
    return fail(ADOP_ERR_INVALID_ARG, "grad_xyz must be 4-byte aligned");
  if ((st = check_grad_feat_dtype(params, n_cam)) != ADOP_OK) return st;
  char* ws = nullptr;
  if ((st = noalloc_scratch(&ws)) != ADOP_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const PdlScope pdl(pdl_for_points(pts->n, n_cam < kMaxCamsPerLaunch ? n_cam : kMaxCamsPerLaunch));
  const bool assign = (params->flags & ADOP_FLAG_GRAD_ASSIGN) != 0;
  const int mode = (n_cam == 1) ? (assign ? kGradAssign : kGradAccumulate) : kGradAtomic;
  cudaError_t e;
  if (assign && n_cam > 1 && pts->n > 0) {
    if (grad_feat && (e = cudaMemsetAsync(grad_feat, 0, (size_t)pts->n * pts->c * 4, s)) != cudaSuccess)
      return cuda_fail(e, "clear grad_feat");
    if (grad_xyz && (e = cudaMemsetAsync(grad_xyz, 0, (size_t)pts->n * 12, s)) != cudaSuccess)
      return cuda_fail(e, "clear grad_xyz");
  }
  const bool want_pose = grad_pose || grad_intr;
  for (int k0 = 0; k0 < n_cam; k0 += kMaxCamsPerLaunch) {
    const int nc = (n_cam - k0) < kMaxCamsPerLaunch ? (n_cam - k0) : kMaxCamsPerLaunch;
    LaunchCams lc;
    for (int j = 0; j < nc; ++j) {
      const int k = k0 + j;
      fill_cam(lc.c[j], cams[k], &frames[k], true, L, k, ws, pts, params);
      for (int l = 0; l < params->levels; ++l) {
        lc.c[j].grad[l] = grad_image ? grad_image[k * params->levels + l] : nullptr;
        lc.c[j].image[l] = nullptr;
      }
    }
    const PointArgs a = point_args(pts, params, nc);
    if ((e = launch_bwd_prepass(lc, a, pts->c, s)) != cudaSuccess) return cuda_fail(e, "backward prepass launch");
    if (pts->n == 0) continue;
    const int bx = point_blocks(pts->n, nc) < kMaxPartialBlocks ? point_blocks(pts->n, nc) : kMaxPartialBlocks;
    BwdArgs b{};
    b.grad_feat = grad_feat;
    b.grad_xyz = grad_xyz;
    b.partials = want_pose ? reinterpret_cast<float*>(ws + L.partials) : nullptr;
    b.mode = mode;
    b.all_projected = (params->flags & ADOP_FLAG_GRAD_ALL_PROJECTED) ? 1 : 0;
    b.feat_out = params->grad_feat_dtype;
    if ((e = launch_bwd_points(lc, a, b, pts->c, pts->feat_dtype, bx, s)) != cudaSuccess)
      return cuda_fail(e, "backward point pass launch");
    if (want_pose && (e = launch_bwd_reduce(b.partials, nc, bx, grad_pose ? grad_pose + 6 * k0 : nullptr,
                                            grad_intr ? grad_intr + 6 * k0 : nullptr, s)) != cudaSuccess)
      return cuda_fail(e, "backward reduce launch");
  }
  g_last_error.clear();
  return ADOP_OK;
}

}  // extern "C"
