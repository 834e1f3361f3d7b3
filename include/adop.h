/*
 * adop.h -- C ABI of a GB300 (sm_103a) implementation of ADOP's
 * differentiable one-pixel point rasterizer.
 *
 * Paper: D. Rueckert, L. Franke, M. Stamminger, "ADOP: Approximate
 * Differentiable One-Pixel Point Rendering" (arXiv 2110.06635), Sec. 3.1
 * (rasterizer, forward and backward), Sec. 3.3 (photometric camera model).
 *
 * Conventions shared by every call
 *   - All array arguments are DEVICE pointers owned by the caller (for
 *     example memory allocated by PyTorch), except the structs themselves,
 *     which are read on the host during the call and may be freed when it
 *     returns.  The library allocates no device memory in these calls.
 *   - Calls are asynchronous on the given CUDA stream (`adop_stream` is
 *     ABI-compatible with cudaStream_t; NULL = the legacy default stream).
 *     Argument errors are detected on the host, before anything is
 *     launched, and returned synchronously.  A launch failure returns
 *     ADOP_ERR_CUDA.  No call aborts or traps.
 *   - adop_last_error() returns a thread-local description of the last
 *     non-OK status returned on the calling thread.
 *   - Layer l of the image pyramid has w_l = w >> l, h_l = h >> l pixels;
 *     pixel (pu, pv) of layer l has id pv * w_l + pu.
 */
#ifndef ADOP_H
#define ADOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADOP_MAX_LEVELS 8          /* pyramid layers per camera (the paper uses 4) */
#define ADOP_MAX_CAMERAS 64        /* cameras per call */
#define ADOP_ABI_VERSION 3

struct CUstream_st;
typedef struct CUstream_st* adop_stream; /* == cudaStream_t */

typedef enum {
    ADOP_OK = 0,
    ADOP_ERR_INVALID_ARG = 1,  /* a pointer, size, shape or flag is invalid */
    ADOP_ERR_UNSUPPORTED = 2,  /* valid, but not implemented (e.g. channel count) */
    ADOP_ERR_OUT_OF_MEMORY = 3,/* workspace too small / server budget exhausted */
    ADOP_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
    ADOP_ERR_TIMEOUT = 5,      /* a bounded wait ran out */
    ADOP_ERR_BUSY = 6,         /* not finished yet (polling) */
    ADOP_ERR_CANCELLED = 7     /* the request was cancelled */
} adop_status;

typedef enum { ADOP_F32 = 0, ADOP_BF16 = 1, ADOP_F16 = 2 } adop_dtype;

/* Camera model C of Eq. render.
 * model 0, pinhole with Brown-Conrady distortion ("Pinhole + Dist."):
 *   xn = X/Z, yn = Y/Z, r2 = xn^2 + yn^2, d = 1 + r2 (k1 + r2 (k2 + r2 k3))
 *   xd = xn d + 2 p1 xn yn + p2 (r2 + 2 xn^2), yd = yn d + p1 (r2 + 2 yn^2) + 2 p2 xn yn
 *   depth = Z.
 * model 1, fisheye (the paper's Office scene; no formula is given -- read as
 * the stereographic projection, r = 2 tan(theta / 2)):
 *   a = 2 / (|X| + Z), (xn, yn) = a (X, Y), xd = xn d, yd = yn d (d as above,
 *   p1, p2 unused); depth = |X| (the paper's rule for a model without z);
 *   undefined on the negative optical axis.
 * Then u0 = fx xd + cx, v0 = fy yd + cy, and layer l uses (u0, v0) / 2^l.
 * w, h: layer-0 image size in pixels (1 .. 16384). */
typedef struct {
    int32_t w, h;
    float fx, fy, cx, cy, k1, k2, k3, p1, p2;
    int32_t model;
} adop_intrinsics;

/* World-to-camera rigid transform (R, t) of Eq. render; X = R x + t, R row-major. */
typedef struct {
    float R[9];
    float t[3];
} adop_pose;

/* Per-image photometric model of Sec. 3.3, applied to channels 0..2 of
 * layer 0 when enabled (and ADOP_FLAG_EPILOGUE is set):
 *   I_e = I / 2^ev; I_w = I_e * wb[ch]; I_v = I_w (1 + a2 r^2 + a4 r^4 + a6 r^6)
 *   with r = |(u / w, v / h) - vig_c|; out = R_ch(I_v), R_ch a piecewise-linear
 *   LUT of crf_n samples on [0,1] (input clamped to [0,1]) at
 *   crf_lut[ch * crf_n ...] (device pointer, 3 x crf_n floats), or the identity
 *   if crf_lut is NULL.  With ADOP_FLAG_LEAKY_CRF (training) the LUT response
 *   leaks outside [0,1] as in Eq. resonseleak, alpha = 0.01: 0.01 x below 0,
 *   -0.01 / sqrt(x) + 1.01 above 1. */
typedef struct {
    float ev;
    float wb[3];
    float vig_c[2];
    float vig_a[3];
    const float* crf_lut;
    int32_t crf_n;
    int32_t enabled;
} adop_photometric;

typedef struct {
    adop_intrinsics K;
    adop_pose T;
    adop_photometric ph;
} adop_camera;

/* The point cloud: positions x (n x 3 FP32, 16-byte aligned), neural
 * descriptors tau (n x c, feat_dtype, 16-byte aligned), optional normals
 * (n x 3 FP32, used only with ADOP_FLAG_NORMAL_CULL).  c in {1,2,3,4,8,16};
 * n < 2^31.  radius and beta (n FP32 each, used only with
 * ADOP_FLAG_DISCARD): the world radius r_world of each point (e.g. from
 * adop_point_radius) and its uniform draw beta in [0, 1) for stochastic
 * point discarding (Sec. 3.1, Eq. discard). */
typedef struct {
    int64_t n;
    int32_t c;
    adop_dtype feat_dtype;
    const float* xyz;
    const void* feat;
    const float* normals;
    const float* radius;
    const float* beta;
} adop_points;

#define ADOP_FLAG_NORMAL_CULL (1u << 0)       /* Eq. normalculling; needs normals */
#define ADOP_FLAG_GRAD_ALL_PROJECTED (1u << 1)/* spatial gradients also for occluded points */
#define ADOP_FLAG_EPILOGUE (1u << 2)          /* apply the photometric model (fwd and bwd) */
#define ADOP_FLAG_GRAD_ASSIGN (1u << 3)       /* grad_feat / grad_xyz are overwritten, not += */
#define ADOP_FLAG_DISCARD (1u << 4)           /* stochastic point discarding, Eq. discard */
#define ADOP_FLAG_LEAKY_CRF (1u << 5)         /* training response curve, Eq. resonseleak */
#define ADOP_FLAG_LOG_DESCRIPTORS (1u << 6)   /* tau stored as log values: exp(tau) is blended (Sec. 3.2);
                                                 grad_feat is then dL/dtau of the stored values */

/* levels: pyramid layers L (1..ADOP_MAX_LEVELS); alpha: fuzzy depth-test
 * threshold of Eq. depthtest (the paper uses 0.01); znear: points with
 * depth z <= znear are discarded; background: c FP32 values (device) shown
 * where no point lands when there is no environment map, NULL = zeros.
 * env (Sec. 3.1, environment map; NULL = none): env_h x env_w texels of c
 * FP32 each, texel-major (texel (i, j) at env[(j env_w + i) c], channels
 * contiguous; device, 16-byte aligned), an equirectangular map of world
 * directions.  A pixel
 * where no point lands shows E(R^T C^-1(u0, v0)) instead of the background:
 * the ray through the pixel centre (layer-l pixel (p, q) at layer-0
 * coordinates (p 2^l, q 2^l)), C^-1 the inverse camera model (pinhole:
 * fixed-point inversion of the distortion; fisheye: Newton on the radial
 * polynomial, then the inverse stereographic map), looked up at longitude
 * phi = atan2(d_x, d_z), colatitude theta = acos(d_y), texel coordinates
 * ((phi + pi) / (2 pi) env_w - 1/2, theta / pi env_h - 1/2), bilinear,
 * wrapping in longitude and clamped in colatitude (FP32).  The empty-target
 * case of the spatial gradient then uses that value; the pose gets no
 * gradient through the lookup.  env_w, env_h in [1, 16384].  A pixel beyond
 * the fold of a non-monotone radial polynomial has no ray; it still samples
 * in-range texels, but which ones is unspecified.
 * gamma (> 0, the paper uses 1.5): with ADOP_FLAG_DISCARD a point is
 * rendered at layer l only if r_screen / sqrt(1 - beta) > 1 / gamma, where
 * r_screen = fx r_world / (z 2^l); evaluated in FP32 as
 * (t * t) * f32(gamma * gamma) > 1 - beta with t = (f32(fx 2^-l) * r_world) / z.
 * A discarded (point, layer) pair takes no part in the depth test, the blend
 * or the gradients of that layer.
 * grad_dtype: storage type of the upstream gradients grad_image of
 * adop_render_backward(_noalloc) (ADOP_F32, the zero default, or ADOP_BF16 /
 * ADOP_F16, read and widened to FP32; adop_env_backward and
 * adop_photometric_backward take ADOP_F32 only).  grad_feat_dtype: storage
 * type of their grad_feat: ADOP_F32 (default), or ADOP_BF16 / ADOP_F16 with
 * ADOP_FLAG_GRAD_ASSIGN and one camera, where each point's dL/dtau is summed
 * in FP32 and rounded once when stored (rows of c 16-bit values, 16-byte
 * aligned); otherwise ADOP_ERR_UNSUPPORTED.  The forward pass ignores both. */
typedef struct {
    int32_t levels;
    float alpha;
    float znear;
    const float* background;
    uint32_t flags;
    float gamma;
    const float* env;
    int32_t env_w, env_h;
    adop_dtype grad_dtype;
    adop_dtype grad_feat_dtype;
} adop_params;

/* Per-camera frame.  image[l]: output, c x h_l x w_l planar in out_dtype
 * (NULL = layer not written).  key[l] (uint64 per pixel: bits(z_min) << 32 |
 * index of the nearest point; UINT64_MAX when empty), count[l] (|Lambda|
 * per pixel) and acc (FP32 feature sums, pixel-major: pixel p of layer l at
 * acc[(off_l + p) * c], off_l = sum_{k<l} w_k h_k; with an environment map,
 * an empty pixel's acc holds the value the forward sampled for it) are the
 * per-pixel state that the backward pass re-uses.  Either all of key/count/acc are given
 * (the forward fills them; the backward reads them) or all are NULL (the
 * forward keeps them in the workspace; the backward re-renders them there,
 * as the paper's backward pass does).
 * vis (optional, n uint32, only with key/count/acc): per point, bit l
 * (l < 8) is set iff the point passed the fuzzy depth test at its layer-l
 * pixel, i.e. is in Lambda of that pixel; bits 8..31 hold, for such points,
 * the 32x32-pixel screen tile of its layer-0 position (row-major over
 * ceil(w/32) tiles per row, position clamped to the image).  The forward
 * writes it; the backward then skips the layers where a point is not in
 * Lambda without looking at any pixel, and visits the points tile by tile.
 * It is the result of the same FP32 comparisons, so results do not change. */
typedef struct {
    void* image[ADOP_MAX_LEVELS];
    uint64_t* key[ADOP_MAX_LEVELS];
    uint32_t* count[ADOP_MAX_LEVELS];
    float* acc;
    uint32_t* vis;
    adop_dtype out_dtype;
} adop_frame;

/* Bytes of device workspace that forward/backward need for these arguments
 * (256-byte aligned pointer required).  Returns 0 on invalid arguments. */
size_t adop_workspace_bytes(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                            const adop_params* params);

/*
 * Forward pass, Sec. 3.1 (Eqs. render, round, boundscheck, normalculling,
 * depthtest, blend): for every camera and layer, project every point,
 * keep the nearest depth per pixel (packed 64-bit (depth, index) key, ties
 * to the smallest index), blend the mean descriptor of all points within
 * the fuzzy threshold z <= (1 + alpha) z_min, write background where no
 * point lands, then the optional photometric epilogue (Sec. 3.3).
 * The projection and depth are evaluated as a fixed sequence of FP32
 * operations (no contraction), rounding ties to even; sums are FP32.
 */
adop_status adop_render_forward(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                                const adop_params* params, adop_frame* frames, void* workspace,
                                size_t workspace_bytes, adop_stream stream);

/*
 * Backward pass, Sec. 3.1 (Eqs. partial, induce, gradp, spatialderiv,
 * tangent).  grad_image[k * levels + l]: dL/dI of camera k, layer l (c x h_l
 * x w_l values of params->grad_dtype, FP32 by default; NULL = zero).
 * Outputs (FP32 -- grad_feat in params->grad_feat_dtype --, accumulated with
 * += unless ADOP_FLAG_GRAD_ASSIGN):
 *   grad_feat n x c   dL/dtau = sum over cameras/layers of G(p)/|Lambda(p)| for
 *                     points in Lambda(p)
 *   grad_xyz  n x 3   dL/dx from the one-pixel approximate spatial gradient
 *                     (NULL = not computed)
 *   grad_pose n_cam x 6  dL/dxi of the left increment exp(xi)(R,t), xi = (nu, omega)
 *   grad_intr n_cam x 6  dL/d(fx, fy, cx, cy, k1, k2)
 * (grad_pose / grad_intr always accumulate, NULL = not computed.)
 * The induced change at a neighbour q of the point's pixel is: tau - I(q) if q
 * is empty or the point is in front (z (1+alpha) < z_min(q)), 0 if it is
 * behind (z > (1+alpha) z_min(q)), (tau - I(q)) / (1 + |Lambda(q)|) otherwise;
 * g_u = (<G(u+1,v), D(u+1,v)> - <G(u-1,v), D(u-1,v)>) / 2, g_v likewise.
 * frames: the forward's frames (key/count/acc NULL => re-rendered here).
 */
adop_status adop_render_backward(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                                 const adop_params* params, const adop_frame* frames,
                                 const float* const* grad_image, float* grad_feat, float* grad_xyz,
                                 float* grad_pose, float* grad_intr, void* workspace,
                                 size_t workspace_bytes, adop_stream stream);

/*
 * Backward pass that allocates nothing and takes no workspace.
 * The paper has no counterpart: this is a deployment variant of
 * adop_render_backward for callers that cannot call cudaMalloc -- for
 * example a renderer embedded in a host application that owns all device
 * memory through its own pool and forbids allocations on its frame loop
 * (cudaMalloc can synchronise the device and stall a frame), or a process
 * whose device-memory budget is fixed before it starts.
 *
 * Same arguments, results and error behaviour as adop_render_backward,
 * except:
 *   - Its scratch (the per-pixel backward records and the pose/intrinsics
 *     block partials) lives in one library-owned static device array of
 *     ADOP_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU which loads the
 *     library keeps until the process exits.  Calls needing more (16 + 4 * c'
 *     bytes per pyramid pixel, c' = c rounded up to a multiple of 4 from 3
 *     on, summed over cameras) return ADOP_ERR_OUT_OF_MEMORY before launching.
 *   - Every frame must carry the forward's kept state (key, count, acc);
 *     re-rendering would need further scratch (ADOP_ERR_INVALID_ARG).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture.
 *   - Under lazy module loading (the CUDA default), the first adop_* call
 *     on a device that launches a kernel loads the library's device code,
 *     and that load places this array in device memory and may
 *     synchronise.  Callers that must not allocate on their frame loop make
 *     one warm-up call of this entry point outside it (or run with
 *     CUDA_MODULE_LOADING=EAGER, which places the array when the context is
 *     created).
 *   - The looked-up address is kept for the life of the process: do not use
 *     the library across a cudaDeviceReset of that device.
 *   - All calls share the array and it keeps the previous call's contents
 *     (every call overwrites what it reads).  Calls that overlap on the GPU
 *     (on different streams, or from different threads) race: serialise them.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define ADOP_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

adop_status adop_render_backward_noalloc(const adop_points* pts, const adop_camera* cams, int32_t n_cam,
                                         const adop_params* params, const adop_frame* frames,
                                         const float* const* grad_image, float* grad_feat,
                                         float* grad_xyz, float* grad_pose, float* grad_intr,
                                         adop_stream stream);

/*
 * Tangent-space pose update (Sec. 3.1, implementation details, Eq. tangent):
 * the pose is optimised through a tangent xi = (nu, omega) in se(3) that
 * starts at zero; after each optimiser step the increment is applied as
 * (R', t') = exp(xi) (R, t) and the tangent is reset.  For k < n:
 * poses[k] <- exp(xi[6k .. 6k+5]) poses[k] (host memory, in place), with
 * exp the closed-form SE(3) exponential:
 *   E = I + a [omega]x + b [omega]x^2,  e = (I + b [omega]x + c [omega]x^2) nu,
 *   a = sin(th)/th, b = (1 - cos(th))/th^2, c = (th - sin(th))/th^3,
 *   th = |omega|;  R' = E R, t' = E t + e.
 * Evaluated in FP64 from the FP32 pose and rounded to FP32 once.  Host only:
 * no device memory, no stream.  ADOP_ERR_INVALID_ARG for n < 0, NULL
 * pointers (n > 0) or a non-finite tangent (then no pose is changed).
 */
adop_status adop_pose_apply_tangent(const double* xi, adop_pose* poses, int32_t n);

/* ------------------------------------------------------------------------
 * Render server: continuous batching of forward renders.
 *
 * A server keeps point clouds resident (it borrows their device pointers,
 * which must stay valid until adop_serve_destroy) and renders requests --
 * one camera each, any resolution -- into caller-owned device buffers.  The
 * only device memory it allocates is one block of mem_budget_bytes at
 * create, from which every admitted request reserves its pixel state
 * (keys, counts, sums: (12 + 4 c) bytes per pyramid pixel).  A scheduler
 * thread admits queued requests in FIFO order whenever a slot and memory are
 * free, groups the oldest admitted requests (up to max_batch, of any of the
 * resident clouds: each camera of a launch renders its own cloud) into one
 * launch sequence, and runs batches concurrently on `streams` CUDA streams;
 * requests that arrive while others run join the next batch.  With
 * batch_window_us > 0, a batch smaller than max_batch is held back while its
 * oldest request has waited less than that long, so that more can join.  The
 * render itself is adop_render_forward's (forward pass of Sec. 3.1 plus the
 * photometric epilogue of Sec. 3.3 when ADOP_FLAG_EPILOGUE is set and the
 * camera enables it), so a result is the same alone and in a batch.
 * Latency = submit to completion of the request's batch on the device.
 * Not part of the paper: the deployment side of the method.
 * ---------------------------------------------------------------------- */
typedef struct adop_server adop_server;

typedef struct {
    size_t mem_budget_bytes;   /* device memory for pixel state (>= 1 MiB) */
    int32_t max_slots;         /* requests admitted at once (1..4096) */
    int32_t streams;           /* batches in flight at once (1..16) */
    int32_t max_batch;         /* cameras per launch (1..16) */
    int32_t levels;            /* pyramid layers of every request */
    float alpha, znear;        /* as in adop_params */
    uint32_t flags;            /* ADOP_FLAG_EPILOGUE | ADOP_FLAG_NORMAL_CULL */
    adop_dtype out_dtype;      /* output image type */
    const float* background;   /* c FP32 (device) or NULL */
    const float* env;          /* environment map as in adop_params, or NULL */
    int32_t env_w, env_h;
    int32_t batch_window_us;   /* dynamic batching window, 0 .. 10^6 microseconds (0: launch at once) */
} adop_serve_config;

typedef struct {
    int64_t submitted, completed, cancelled, failed, queued, active, batches;
    double mean_batch;         /* requests per launched batch */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency since the last reset */
    double req_per_s, points_per_s;          /* completed since the last reset */
    size_t mem_in_use, mem_peak;
    int64_t mixed_batches;     /* batches whose cameras render more than one cloud */
} adop_serve_stats;

/* Create a server (allocates the budget and the streams, starts the scheduler). */
adop_status adop_serve_create(const adop_serve_config* cfg, adop_server** out);
/* Register a resident cloud; all clouds share c and feat_dtype. */
adop_status adop_serve_load_cloud(adop_server* s, const adop_points* pts, int32_t* cloud_id);
/* Queue a render of cloud_id through cam into out_image (device, caller-owned:
 * all layers concatenated, layer l = c x h_l x w_l planar in out_dtype).
 * ADOP_ERR_OUT_OF_MEMORY if the request could never fit the budget. */
adop_status adop_serve_submit(adop_server* s, int32_t cloud_id, const adop_camera* cam, void* out_image,
                              uint64_t* ticket);
/* ADOP_OK when done, ADOP_ERR_BUSY while queued or running, or the request's error. */
adop_status adop_serve_poll(adop_server* s, uint64_t ticket);
/* Block until the request is done or timeout_ms passes (ADOP_ERR_TIMEOUT). */
adop_status adop_serve_wait(adop_server* s, uint64_t ticket, int32_t timeout_ms);
/* Cancel a request still in the queue (ADOP_ERR_BUSY once admitted). */
adop_status adop_serve_cancel(adop_server* s, uint64_t ticket);
/* Latency of a finished request in milliseconds. */
adop_status adop_serve_latency(adop_server* s, uint64_t ticket, double* ms);
adop_status adop_serve_get_stats(adop_server* s, adop_serve_stats* out);
adop_status adop_serve_reset_stats(adop_server* s);
/* Cancel queued requests, finish admitted ones, free everything. */
adop_status adop_serve_destroy(adop_server* s);

/*
 * Gradients of the photometric parameters (Sec. 3.3) of every camera whose
 * epilogue is enabled (ADOP_FLAG_EPILOGUE and ph.enabled), from dL/d(out) of
 * layer 0 (grad_image0[k]: c x h x w FP32, NULL = zero) and the layer-0 image
 * before the epilogue, which is the forward's kept state (frames must carry
 * key/count/acc).  Accumulated (+=):
 *   grad_photo  n_cam x 9: dL/d(ev, wb[0..2], vig_c[0..1], vig_a[0..2])
 *   grad_crf    dL/d(crf_lut): for each camera in order, 3 x its crf_n floats
 *               (no entries for a camera without a LUT); NULL = not computed
 * crf_n <= 4000.  Workspace: adop_photometric_workspace_bytes(n_cam).
 */
/*
 * Gradient of the environment map (Sec. 3.1), accumulated (+=) into
 * grad_env (laid out like params->env, 16-byte aligned): every pixel of every
 * layer where no point landed adds its upstream gradient to the four texels
 * it sampled, with the bilinear weights.  grad_image[k * levels + l] as in
 * adop_render_backward (at layer 0 it is chained through the photometric
 * epilogue when that is on, at the value kept in frames[k].acc if given, else
 * at a new sample); frames must carry the forward's count[l] of every layer.
 * params->env must be the map the forward sampled.  Needs no workspace.
 * Texel sums use FP32 atomics: their order, and so the last bits, vary
 * between runs.
 */
adop_status adop_env_backward(const adop_camera* cams, int32_t n_cam, const adop_params* params, int32_t c,
                              const adop_frame* frames, const float* const* grad_image, float* grad_env,
                              adop_stream stream);

size_t adop_photometric_workspace_bytes(int32_t n_cam);
adop_status adop_photometric_backward(const adop_camera* cams, int32_t n_cam, const adop_params* params,
                                      int32_t c, const adop_frame* frames, const float* const* grad_image0,
                                      float* grad_photo, float* grad_crf, void* workspace,
                                      size_t workspace_bytes, adop_stream stream);

/* Kernel timing.  While enabled, every kernel the library launches is
 * bracketed by a pair of CUDA events recorded on the launch's stream (a few
 * microseconds of host time per launch, no device synchronisation).
 * adop_profile_collect waits for the recorded events, adds each kernel's
 * launches and device time into out[] (one entry per kernel name, at most
 * max entries), clears the record and returns the number of entries
 * (negative on a CUDA error).  Not part of the paper: instrumentation. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} adop_kernel_stat;

adop_status adop_profile_enable(int32_t on);
int32_t adop_profile_collect(adop_kernel_stat* out, int32_t max);

/*
 * World radius of every point for stochastic discarding (Sec. 3.1): the
 * distance to its k-th nearest other point (the paper uses k = 4), by a
 * uniform-grid search on the GPU with cells of 1.5x the median k-NN distance
 * of 256 sampled points; +inf if the cloud has fewer than k + 1 points.
 * Exact (FP32 distances) when the k-th neighbour lies within 8 cells and at
 * most 65536 candidates are scanned for the point; otherwise an upper bound
 * (isolated outliers, which discarding keeps anyway).  xyz: n x 3 FP32
 * (device); radius: n FP32 (device, output); 1 <= k <= 16.  A preprocess: it
 * synchronises `stream` once (to size the grid).  Workspace from
 * adop_point_radius_workspace_bytes(n).
 */
size_t adop_point_radius_workspace_bytes(int64_t n);
adop_status adop_point_radius(const float* xyz, int64_t n, int32_t k, float* radius, void* workspace,
                              size_t workspace_bytes, adop_stream stream);

/* Thread-local message of the last error on this thread ("" if none). */
const char* adop_last_error(void);

/*
 * Measurement aid, not part of the paper: launch `ops` atomics of one kind at
 * uniformly random elements of buf (device, elems elements of the kind's
 * size, elems < 2^32; hash of seed + op index): kind 0 = 64-bit unsigned
 * atomicMin (the depth pass's key update), 1 = 32-bit integer add (|Lambda|),
 * 2 = 16-byte float4 add (the accumulate pass's vector atomics), 3 = 32-bit
 * float add.  The caller times the launch on `stream`; the result in buf is
 * meaningless.  Used for the L2-atomic ceiling of the depth and accumulate
 * passes.
 */
adop_status adop_atomic_probe(int32_t kind, void* buf, int64_t elems, int64_t ops, uint64_t seed,
                              adop_stream stream);

/* ADOP_ABI_VERSION of the loaded library. */
int32_t adop_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ADOP_H */
