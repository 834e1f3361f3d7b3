/*
 * Plain CPU oracle of ADOP's differentiable one-pixel point rasterizer
 * (Rueckert, Franke, Stamminger: "ADOP: Approximate Differentiable One-Pixel
 * Point Rendering", Sec. 3.1, Eqs. render, round, boundscheck, normalculling,
 * depthtest, blend, induce, gradp, spatialderiv, tangent; Sec. 3.3 for the
 * photometric epilogue).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path must compute.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only in
 * the written FP32 projection contract below and in seeded inputs.
 *
 * Precision rules
 *   - The projection that decides a pixel and a depth is an FP32 contract:
 *     every step is one IEEE binary32 operation in the order written below,
 *     no fused multiply-add (compile with -ffp-contract=off), rounding to
 *     the nearest integer with ties to even (nearbyintf under the default
 *     rounding mode).  The paper leaves the precision open; this reading is
 *     what makes depth/index buffers comparable bit for bit.
 *   - Everything after the pixel/depth decision (blend sums, means, the
 *     induced changes of Eq. spatialderiv, Jacobians, the chain rule and all
 *     reductions) is FP64.
 *   - Decisions that compare depths (fuzzy test, the cases of Eq.
 *     spatialderiv) are taken in FP32, the precision of the depth buffer.
 *
 * Layouts (all per camera)
 *   xyz     n x 3 float, world space
 *   feat    n x c double (features upcast exactly from their storage type)
 *   layers  l = 0..levels-1, w_l = w >> l, h_l = h >> l, pixel id within a
 *           layer = pv * w_l + pu; per-layer arrays are concatenated in
 *           layer order (offset of layer l = sum_{k<l} w_k h_k pixels)
 *   image   per layer c x h_l x w_l (planar), concatenated
 *   keys    per pixel: (bits(z_min) << 32) | index of the nearest point,
 *           UINT64_MAX for an empty pixel
 *
 * parity pins: projection (closed forms), blend + spatial gradient (hand
 * example, brute force, shift-and-rerender), chain rule (finite differences
 * with an independent SE(3) exponential) -- see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Threads (a timing aid only: results do not depend on them, see the    */
/* forward and backward below)                                           */
/* ------------------------------------------------------------------ */

/* Threads to use for a request of `threads` (<= 0: every core; 1 when the
 * library was built without OpenMP). */
static int team_size(int32_t threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_num_procs();
#else
    (void)threads;
    return 1;
#endif
}

static int thread_id(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

static int threads_in_team(void) {
#ifdef _OPENMP
    return omp_get_num_threads();
#else
    return 1;
#endif
}

/* Threads a request of `threads` gets (exported for the timing legs). */
int32_t orc_threads(int32_t threads) { return team_size(threads); }

/* Camera model C.  model 0: pinhole with Brown-Conrady distortion (k1,k2,k3
 * radial, p1,p2 tangential); the paper's scenes use "Pinhole + Dist." (Table
 * scenes) without stating the polynomial; this is the common
 * five-coefficient model.  model 1: fisheye (the paper's Office scene; its
 * formula is not given), read as the stereographic projection r = 2 tan(theta/2)
 * with the same radial polynomial in r^2 (p1, p2 unused), and -- as the paper
 * prescribes for a model without a z -- the distance to the camera as depth. */
typedef struct {
    int32_t w, h;
    float fx, fy, cx, cy, k1, k2, k3, p1, p2;
    int32_t model;
} orc_intrinsics;

/* World-to-camera rigid transform (R, t), R row-major (Eq. render). */
typedef struct {
    float R[9];
    float t[3];
} orc_pose;

/* ------------------------------------------------------------------ */
/* FP32 projection contract (Sec. 3.1, P_l(C,R,t,x) = 2^-l C(Rx + t))   */
/* ------------------------------------------------------------------ */

/* X = R x + t, each row summed left to right, then t added. */
static void transform_f32(const orc_pose* T, const float* x, float* X) {
    for (int r = 0; r < 3; ++r) {
        float s = T->R[3 * r + 0] * x[0];
        s = s + T->R[3 * r + 1] * x[1];
        s = s + T->R[3 * r + 2] * x[2];
        X[r] = s + T->t[r];
    }
}

/* Camera model C applied to a camera-space point; returns layer-0 pixel
 * coordinates (u0, v0) and the depth of Eq. depthtest (pinhole: z = X[2];
 * fisheye: the distance |X|).  Returns 0 where the model is undefined
 * (fisheye: on the negative optical axis). */
static int camera_f32(const orc_intrinsics* K, const float* X, float* u0, float* v0, float* depth) {
    if (K->model == 1) {
        /* stereographic: normalised radius 2 tan(theta/2) = 2 rho / (|X| + Z) */
        float d = sqrtf((X[0] * X[0] + X[1] * X[1]) + X[2] * X[2]);
        float s = d + X[2];
        *depth = d;
        if (!(s > 0.0f)) return 0;
        float a = 2.0f / s;
        float xn = a * X[0];
        float yn = a * X[1];
        float r2 = xn * xn + yn * yn;
        float dd = 1.0f + r2 * (K->k1 + r2 * (K->k2 + r2 * K->k3));
        *u0 = K->fx * (xn * dd) + K->cx;
        *v0 = K->fy * (yn * dd) + K->cy;
        return 1;
    }
    *depth = X[2];
    float xn = X[0] / X[2];
    float yn = X[1] / X[2];
    float r2 = xn * xn + yn * yn;
    float d = 1.0f + r2 * (K->k1 + r2 * (K->k2 + r2 * K->k3));
    float a = xn * yn;
    float tx = (2.0f * K->p1) * a + K->p2 * (r2 + 2.0f * (xn * xn));
    float ty = K->p1 * (r2 + 2.0f * (yn * yn)) + (2.0f * K->p2) * a;
    float xd = xn * d + tx;
    float yd = yn * d + ty;
    *u0 = K->fx * xd + K->cx;
    *v0 = K->fy * yd + K->cy;
    return 1;
}

/* Exported: the FP32 contract for one point (used by the projection pins).
 * Returns 0 where the camera model is undefined. */
int orc_project_f32(const orc_intrinsics* K, const orc_pose* T, const float* x,
                    float* u0, float* v0, float* z) {
    float X[3];
    transform_f32(T, x, X);
    return camera_f32(K, X, u0, v0, z);
}

/* Eq. round + Eq. boundscheck for layer l.  The layer scale 2^-l is exact.
 * A coordinate outside ]-1, w_l + 1[ (or NaN) is discarded before the
 * integer conversion; nearbyintf rounds half to even.  Returns 1 and the
 * pixel if the point lands inside layer l, else 0. */
int orc_pixel(float u0, float v0, int l, int32_t w, int32_t h, int32_t* pu, int32_t* pv) {
    int32_t wl = w >> l, hl = h >> l;
    float s = ldexpf(1.0f, -l);
    float ul = u0 * s, vl = v0 * s;
    if (!(ul > -1.0f && ul < (float)wl + 1.0f)) return 0;
    if (!(vl > -1.0f && vl < (float)hl + 1.0f)) return 0;
    int32_t iu = (int32_t)nearbyintf(ul);
    int32_t iv = (int32_t)nearbyintf(vl);
    if (iu < 0 || iu >= wl || iv < 0 || iv >= hl) return 0;
    *pu = iu;
    *pv = iv;
    return 1;
}

static uint32_t f32_bits(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

static float bits_f32(uint32_t b) {
    float f;
    memcpy(&f, &b, 4);
    return f;
}

static int64_t layer_offset(int32_t w, int32_t h, int l) {
    int64_t off = 0;
    for (int k = 0; k < l; ++k) off += (int64_t)(w >> k) * (int64_t)(h >> k);
    return off;
}

/* Total pixels over all layers. */
int64_t orc_pyramid_pixels(int32_t w, int32_t h, int levels) {
    return layer_offset(w, h, levels);
}

/* ------------------------------------------------------------------ */
/* Projection of all points, with the discard tests                     */
/* ------------------------------------------------------------------ */

/* For every point and layer: the pixel id (or -1 if discarded) and the FP32
 * depth.  Tests in the order of Sec. 3.1: near plane (z must be a positive
 * depth), normal culling (Eq. normalculling, optional), bounds (Eq.
 * boundscheck).  The normal test is taken literally from the paper:
 * keep iff (R n)^T (R x + t) / |R x + t| > 0; the positive norm does not
 * change the sign, so it is evaluated as an FP32 dot product. */
/* Eq. discard (stochastic point discarding): render the point at layer l
 * only if r_screen / sqrt(1 - beta) > 1 / gamma, with the world radius
 * projected as r_screen = fx r_world / (z 2^l) (a pinhole reading: the paper
 * does not spell the projection out).  Both sides are positive, so the test
 * is evaluated without the square root as (gamma r_screen)^2 > 1 - beta, in
 * this FP32 order: t = (f32(fx 2^-l) * r) / z; keep iff (t * t) * f32(gamma *
 * gamma) > 1 - beta. */
static int discard_keep(const orc_intrinsics* K, float z, float r, float beta, float gamma, int l) {
    float fxl = K->fx * ldexpf(1.0f, -l);
    float t = (fxl * r) / z;
    float g2 = gamma * gamma;
    return (t * t) * g2 > 1.0f - beta;
}

static void project_all(int64_t n, const float* xyz, const float* normals,
                        const orc_intrinsics* K, const orc_pose* T, int levels, float znear,
                        const float* radius, const float* beta, float gamma,
                        int32_t* pix, float* zf, int nt) {
    /* every point on its own: any split over threads gives the same arrays */
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        float X[3], u0 = 0.0f, v0 = 0.0f, z;
        transform_f32(T, xyz + 3 * i, X);
        int defined = camera_f32(K, X, &u0, &v0, &z);
        zf[i] = z;
        int keep = defined && (z > znear);
        if (keep && normals) {
            const float* nn = normals + 3 * i;
            float Rn[3];
            for (int r = 0; r < 3; ++r) {
                float s = T->R[3 * r + 0] * nn[0];
                s = s + T->R[3 * r + 1] * nn[1];
                s = s + T->R[3 * r + 2] * nn[2];
                Rn[r] = s;
            }
            float dot = Rn[0] * X[0];
            dot = dot + Rn[1] * X[1];
            dot = dot + Rn[2] * X[2];
            keep = (dot > 0.0f);
        }
        for (int l = 0; l < levels; ++l) {
            int32_t pu, pv;
            int keep_l = keep && (!radius || discard_keep(K, z, radius[i], beta[i], gamma, l));
            if (keep_l && orc_pixel(u0, v0, l, K->w, K->h, &pu, &pv))
                pix[i * levels + l] = pv * (K->w >> l) + pu;
            else
                pix[i * levels + l] = -1;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Environment map (Sec. 3.1, "Environment Map"; Eq. blend, empty pixels) */
/* ------------------------------------------------------------------ */

/* Inverse camera model C^-1 in FP64: the unit camera-space direction of the
 * ray through layer-0 pixel coordinates (u0, v0).  Pinhole: the distortion is
 * inverted by fixed-point iteration (xn, yn) = ((xd, yd) - tangential) / d(r2)
 * until it no longer moves; fisheye: the radial polynomial r d(r^2) = r_d is
 * inverted by Newton's method, then the stereographic projection. */
void orc_camera_inverse_f64(const orc_intrinsics* K, double u0, double v0, double* dir) {
    const double xd = (u0 - K->cx) / K->fx, yd = (v0 - K->cy) / K->fy;
    const double k1 = K->k1, k2 = K->k2, k3 = K->k3, p1 = K->p1, p2 = K->p2;
    if (K->model == 1) {
        const double rd = sqrt(xd * xd + yd * yd);
        double r = rd;
        for (int it = 0; it < 100; ++it) {
            const double r2 = r * r;
            const double f = r * (1.0 + k1 * r2 + k2 * r2 * r2 + k3 * r2 * r2 * r2) - rd;
            const double fp = 1.0 + 3.0 * k1 * r2 + 5.0 * k2 * r2 * r2 + 7.0 * k3 * r2 * r2 * r2;
            const double step = f / fp;
            r -= step;
            if (fabs(step) <= 1e-15 * (1.0 + r)) break;
        }
        const double xn = rd > 0.0 ? xd * r / rd : 0.0, yn = rd > 0.0 ? yd * r / rd : 0.0;
        const double r2 = xn * xn + yn * yn;
        dir[0] = 4.0 * xn / (4.0 + r2);
        dir[1] = 4.0 * yn / (4.0 + r2);
        dir[2] = (4.0 - r2) / (4.0 + r2);
        return;
    }
    double xn = xd, yn = yd;
    for (int it = 0; it < 500; ++it) {
        const double r2 = xn * xn + yn * yn;
        const double d = 1.0 + k1 * r2 + k2 * r2 * r2 + k3 * r2 * r2 * r2;
        const double tx = 2.0 * p1 * xn * yn + p2 * (r2 + 2.0 * xn * xn);
        const double ty = p1 * (r2 + 2.0 * yn * yn) + 2.0 * p2 * xn * yn;
        const double nx = (xd - tx) / d, ny = (yd - ty) / d;
        const double moved = fabs(nx - xn) + fabs(ny - yn);
        xn = nx;
        yn = ny;
        if (moved <= 1e-16) break;
    }
    const double nrm = sqrt(xn * xn + yn * yn + 1.0);
    dir[0] = xn / nrm;
    dir[1] = yn / nrm;
    dir[2] = 1.0 / nrm;
}

/* Equirectangular lookup of a world direction in E (c x eh x ew): longitude
 * phi = atan2(dx, dz), colatitude theta = acos(dy); texel coordinates
 * (phi + pi) / (2 pi) ew - 1/2 and theta / pi eh - 1/2 (texel centres at
 * integers); bilinear, wrapping in longitude, clamped in colatitude.
 * out (c values, may be NULL) receives the sample; tex[4] and wts[4] (may be
 * NULL) the texels and weights used. */
void orc_env_sample(const double* env, int32_t c, int32_t ew, int32_t eh, const double* d, double* out,
                    int64_t* tex, double* wts) {
    const double pi = 3.14159265358979323846;
    const double phi = atan2(d[0], d[2]);
    const double dy = d[1] < -1.0 ? -1.0 : (d[1] > 1.0 ? 1.0 : d[1]);
    const double theta = acos(dy);
    const double ue = (phi + pi) / (2.0 * pi) * ew - 0.5;
    const double ve = theta / pi * eh - 0.5;
    const double fu0 = floor(ue), fv0 = floor(ve);
    const double fu = ue - fu0, fv = ve - fv0;
    int64_t iu0 = (int64_t)fu0, iv0 = (int64_t)fv0;
    int64_t iu[2] = {((iu0 % ew) + ew) % ew, (((iu0 + 1) % ew) + ew) % ew};
    int64_t iv[2] = {iv0 < 0 ? 0 : (iv0 >= eh ? eh - 1 : iv0), iv0 + 1 < 0 ? 0 : (iv0 + 1 >= eh ? eh - 1 : iv0 + 1)};
    const double w[4] = {(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv};
    const int64_t t[4] = {iv[0] * ew + iu[0], iv[0] * ew + iu[1], iv[1] * ew + iu[0], iv[1] * ew + iu[1]};
    for (int ch = 0; out && ch < c; ++ch) {
        double v = 0.0;
        for (int k = 0; k < 4; ++k) v += w[k] * env[(int64_t)ch * ew * eh + t[k]];
        out[ch] = v;
    }
    if (tex)
        for (int k = 0; k < 4; ++k) {
            tex[k] = t[k];
            wts[k] = w[k];
        }
}

/* World direction of the ray through pixel (pu, pv) of layer l: C^-1 at the
 * layer-0 coordinates (pu 2^l, pv 2^l) of the pixel's centre, then R^T. */
static void pixel_ray(const orc_intrinsics* K, const orc_pose* T, int l, int32_t pu, int32_t pv, double* dw) {
    double dc[3];
    orc_camera_inverse_f64(K, ldexp((double)pu, l), ldexp((double)pv, l), dc);
    for (int k = 0; k < 3; ++k)
        dw[k] = (double)T->R[0 * 3 + k] * dc[0] + (double)T->R[1 * 3 + k] * dc[1] + (double)T->R[2 * 3 + k] * dc[2];
}

/* dL/dE of the environment map: every empty pixel of every layer adds its
 * upstream gradient G (c x h_l x w_l planar, concatenated) to the texels it
 * sampled, with the bilinear weights.  dE (c x eh x ew) is overwritten. */
void orc_env_grad(const orc_intrinsics* K, const orc_pose* T, int32_t levels, int32_t c, const uint32_t* cnt,
                  const double* G, int32_t ew, int32_t eh, double* dE) {
    for (int64_t j = 0; j < (int64_t)c * ew * eh; ++j) dE[j] = 0.0;
    for (int l = 0; l < levels; ++l) {
        const int64_t off = layer_offset(K->w, K->h, l);
        const int32_t wl = K->w >> l, hl = K->h >> l;
        const int64_t np = (int64_t)wl * hl;
        for (int32_t pv = 0; pv < hl; ++pv)
            for (int32_t pu = 0; pu < wl; ++pu) {
                const int64_t p = (int64_t)pv * wl + pu;
                if (cnt[off + p] != 0) continue;
                double dw[3];
                int64_t tex[4];
                double wts[4];
                pixel_ray(K, T, l, pu, pv, dw);
                orc_env_sample(NULL, c, ew, eh, dw, NULL, tex, wts); /* texels and weights only */
                for (int ch = 0; ch < c; ++ch)
                    for (int k = 0; k < 4; ++k)
                        dE[(int64_t)ch * ew * eh + tex[k]] += wts[k] * G[c * off + (int64_t)ch * np + p];
            }
    }
}

/* ------------------------------------------------------------------ */
/* Forward (Eq. render, Eq. depthtest, Eq. blend)                       */
/* ------------------------------------------------------------------ */

/*
 * orc_forward: one camera.
 *   feat       n x c, double
 *   background c doubles or NULL (= 0): the value of an empty pixel when no
 *              environment map is given.
 *   radius, beta, gamma  stochastic discarding (Eq. discard): per-point world
 *              radius and uniform draw in [0,1); radius NULL = no discarding.
 *   env        environment map (c x env_h x env_w, FP64) sampled for empty
 *              pixels instead of the background; NULL = background.
 * Outputs (all over the concatenated pyramid of `levels` layers):
 *   keys  uint64 per pixel; cnt  |Lambda| per pixel; img  c x h_l x w_l;
 *   pix   n x levels pixel id or -1 (may be NULL); zf  n depths (may be NULL).
 * threads: threads to use (<= 0: every core); the results are the same for
 *   any value (see the steps below).
 * Returns 0, or -1 if an allocation fails.
 */
int orc_forward(int64_t n, const float* xyz, int32_t c, const double* feat, const float* normals,
                const orc_intrinsics* K, const orc_pose* T, int32_t levels, float alpha,
                float znear, const double* background,
                const float* radius, const float* beta, float gamma, int32_t log_desc,
                const double* env, int32_t env_w, int32_t env_h,
                uint64_t* keys, uint32_t* cnt, double* img, int32_t* pix_out, float* z_out,
                int32_t threads) {
    int64_t npx = orc_pyramid_pixels(K->w, K->h, levels);
    const int nt = team_size(threads);
    /* Logarithmic descriptors (Sec. 3.2) are converted to linear values before
     * blending. */
    double* lin = NULL;
    if (log_desc) {
        lin = (double*)malloc(sizeof(double) * (size_t)(n * c + 1));
        if (!lin) return -1;
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t j = 0; j < n * c; ++j) lin[j] = exp(feat[j]);
        feat = lin;
    }
    int32_t* pix = pix_out ? pix_out : (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * levels + 1));
    float* zf = z_out ? z_out : (float*)malloc(sizeof(float) * (size_t)(n + 1));
    double* sum = (double*)calloc((size_t)(npx * c + 1), sizeof(double));
    if (!pix || !zf || !sum) return -1;

    /* Step 1: project every point to every layer (Eqs. projection, round,
     * boundscheck, normalculling). */
    project_all(n, xyz, normals, K, T, levels, znear, radius, beta, gamma, pix, zf, nt);

    /* Steps 2-4 visit the (point, layer) pairs in point-index order, layer by
     * layer.  With several threads, each thread owns one contiguous range
     * [g0, g1) of the pyramid's pixels and takes only the pairs that land
     * there, still in that order: every pixel then sees exactly the same
     * sequence of updates as with one thread, so keys, counts and the FP64
     * sums do not depend on the thread count. */
    const float a1 = 1.0f + alpha;
#pragma omp parallel num_threads(nt)
    {
        const int t = thread_id(), tt = threads_in_team();
        const int64_t g0 = npx * t / tt, g1 = npx * (t + 1) / tt;

        /* Step 2: nearest depth per pixel, as a (depth bits, index) key so
         * that equal depths resolve to the smallest point index. */
        for (int64_t g = g0; g < g1; ++g) keys[g] = UINT64_MAX;
        for (int l = 0; l < levels; ++l) {
            int64_t off = layer_offset(K->w, K->h, l);
            for (int64_t i = 0; i < n; ++i) {
                int32_t p = pix[i * levels + l];
                if (p < 0 || off + p < g0 || off + p >= g1) continue;
                uint64_t key = ((uint64_t)f32_bits(zf[i]) << 32) | (uint64_t)(uint32_t)i;
                if (key < keys[off + p]) keys[off + p] = key;
            }
        }

        /* Step 3: fuzzy depth test (Eq. depthtest) against min_z(p), taken
         * in FP32: pass iff z <= f32(min_z * f32(1 + alpha)).  Step 4:
         * Lambda's size and the feature sum, for the mean of Eq. blend. */
        for (int64_t g = g0; g < g1; ++g) cnt[g] = 0;
        for (int l = 0; l < levels; ++l) {
            int64_t off = layer_offset(K->w, K->h, l);
            for (int64_t i = 0; i < n; ++i) {
                int32_t p = pix[i * levels + l];
                if (p < 0 || off + p < g0 || off + p >= g1) continue;
                float minz = bits_f32((uint32_t)(keys[off + p] >> 32));
                float thr = minz * a1;
                if (!(zf[i] <= thr)) continue;
                cnt[off + p] += 1;
                for (int ch = 0; ch < c; ++ch) sum[(off + p) * c + ch] += feat[i * c + ch];
            }
        }
    }

    /* Step 5: Eq. blend -- the mean over Lambda, or, for an empty pixel, the
     * environment map E(R^T C^-1(u, v)) (or the constant background).  Every
     * pixel on its own. */
    int failed = 0;
    for (int l = 0; l < levels; ++l) {
        int64_t off = layer_offset(K->w, K->h, l);
        const int32_t wl = K->w >> l;
        int64_t np = (int64_t)wl * (K->h >> l);
#pragma omp parallel num_threads(nt) reduction(| : failed)
        {
            double* ev = (double*)malloc(sizeof(double) * (size_t)(c + 1));
            if (!ev) failed = 1;
#pragma omp for schedule(static)
            for (int64_t p = 0; p < np; ++p) {
                if (!ev) continue;
                if (cnt[off + p] == 0 && env) {
                    double dw[3];
                    pixel_ray(K, T, l, (int32_t)(p % wl), (int32_t)(p / wl), dw);
                    orc_env_sample(env, c, env_w, env_h, dw, ev, NULL, NULL);
                }
                for (int ch = 0; ch < c; ++ch) {
                    double v;
                    if (cnt[off + p] == 0)
                        v = env ? ev[ch] : (background ? background[ch] : 0.0);
                    else
                        v = sum[(off + p) * c + ch] / (double)cnt[off + p];
                    img[c * off + (int64_t)ch * np + p] = v;
                }
            }
            free(ev);
        }
    }
    free(sum);
    if (failed) {
        free(lin);
        if (!pix_out) free(pix);
        if (!z_out) free(zf);
        return -1;
    }
    free(lin);
    if (!pix_out) free(pix);
    if (!z_out) free(zf);
    return 0;
}

/* ------------------------------------------------------------------ */
/* FP64 projection and its Jacobians (chain rule, Eq. partial)          */
/* ------------------------------------------------------------------ */

/*
 * For the chain rule the continuous projection is re-evaluated in FP64 from
 * the same FP32 inputs.  Outputs:
 *   uv[2]      (u0, v0)
 *   X[3]       camera-space point
 *   J_X[6]     d(u0,v0)/dX, row-major 2 x 3
 *   J_K[12]    d(u0,v0)/d(fx, fy, cx, cy, k1, k2), row-major 2 x 6
 */
/* The camera model C in FP64 with FP64 parameters k9 = (fx, fy, cx, cy, k1,
 * k2, k3, p1, p2), for a camera-space point X.  Exported for the
 * finite-difference pins (intrinsics and pose perturbed in FP64). */
void orc_camera_f64(const double* k9, const double* X, double* uv) {
    const double fx = k9[0], fy = k9[1], cx = k9[2], cy = k9[3];
    const double k1 = k9[4], k2 = k9[5], k3 = k9[6], p1 = k9[7], p2 = k9[8];
    const double xn = X[0] / X[2], yn = X[1] / X[2];
    const double r2 = xn * xn + yn * yn;
    const double d = 1.0 + k1 * r2 + k2 * r2 * r2 + k3 * r2 * r2 * r2;
    const double xd = xn * d + 2.0 * p1 * xn * yn + p2 * (r2 + 2.0 * xn * xn);
    const double yd = yn * d + p1 * (r2 + 2.0 * yn * yn) + 2.0 * p2 * xn * yn;
    uv[0] = fx * xd + cx;
    uv[1] = fy * yd + cy;
}

/* The fisheye model (stereographic + radial polynomial) in FP64, k9 as above. */
void orc_camera_fisheye_f64(const double* k9, const double* X, double* uv) {
    const double d = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    const double a = 2.0 / (d + X[2]);
    const double xn = a * X[0], yn = a * X[1];
    const double r2 = xn * xn + yn * yn;
    const double dd = 1.0 + k9[4] * r2 + k9[5] * r2 * r2 + k9[6] * r2 * r2 * r2;
    uv[0] = k9[0] * xn * dd + k9[2];
    uv[1] = k9[1] * yn * dd + k9[3];
}

/* orc_camera_f64 (model 0) or orc_camera_fisheye_f64 (model 1) over n
 * camera-space points (X: n x 3, uv: n x 2). */
void orc_camera_f64_many(int64_t n, const double* k9, const double* X, double* uv, int32_t model) {
    for (int64_t i = 0; i < n; ++i) {
        if (model == 1)
            orc_camera_fisheye_f64(k9, X + 3 * i, uv + 2 * i);
        else
            orc_camera_f64(k9, X + 3 * i, uv + 2 * i);
    }
}

void orc_project_jac_f64(const orc_intrinsics* K, const orc_pose* T, const float* x,
                         double* uv, double* X, double* J_X, double* J_K) {
    for (int r = 0; r < 3; ++r) {
        X[r] = (double)T->R[3 * r + 0] * x[0] + (double)T->R[3 * r + 1] * x[1] +
               (double)T->R[3 * r + 2] * x[2] + (double)T->t[r];
    }
    const double k9[9] = {K->fx, K->fy, K->cx, K->cy, K->k1, K->k2, K->k3, K->p1, K->p2};
    if (K->model == 1) {
        orc_camera_fisheye_f64(k9, X, uv);
        const double fx = K->fx, fy = K->fy, k1 = K->k1, k2 = K->k2, k3 = K->k3;
        const double d = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
        const double s = d + X[2];
        const double a = 2.0 / s;
        const double xn = a * X[0], yn = a * X[1];
        const double r2 = xn * xn + yn * yn;
        const double dd = 1.0 + k1 * r2 + k2 * r2 * r2 + k3 * r2 * r2 * r2;
        const double ddr = k1 + 2.0 * k2 * r2 + 3.0 * k3 * r2 * r2;
        /* d s / d X = X / d + e_z ; d a / d X = -2 / s^2 * d s / d X */
        double ds[3] = {X[0] / d, X[1] / d, X[2] / d + 1.0};
        double da[3];
        for (int k = 0; k < 3; ++k) da[k] = -2.0 / (s * s) * ds[k];
        double dxn[3], dyn[3];
        for (int k = 0; k < 3; ++k) {
            dxn[k] = X[0] * da[k] + (k == 0 ? a : 0.0);
            dyn[k] = X[1] * da[k] + (k == 1 ? a : 0.0);
        }
        const double dxd_dxn = dd + xn * ddr * 2.0 * xn, dxd_dyn = xn * ddr * 2.0 * yn;
        const double dyd_dxn = yn * ddr * 2.0 * xn, dyd_dyn = dd + yn * ddr * 2.0 * yn;
        for (int k = 0; k < 3; ++k) {
            J_X[k] = fx * (dxd_dxn * dxn[k] + dxd_dyn * dyn[k]);
            J_X[3 + k] = fy * (dyd_dxn * dxn[k] + dyd_dyn * dyn[k]);
        }
        J_K[0] = xn * dd; J_K[1] = 0.0; J_K[2] = 1.0; J_K[3] = 0.0;
        J_K[4] = fx * xn * r2; J_K[5] = fx * xn * r2 * r2;
        J_K[6] = 0.0; J_K[7] = yn * dd; J_K[8] = 0.0; J_K[9] = 1.0;
        J_K[10] = fy * yn * r2; J_K[11] = fy * yn * r2 * r2;
        return;
    }
    orc_camera_f64(k9, X, uv);
    const double fx = K->fx, fy = K->fy;
    const double k1 = K->k1, k2 = K->k2, k3 = K->k3, p1 = K->p1, p2 = K->p2;
    const double xn = X[0] / X[2], yn = X[1] / X[2];
    const double r2 = xn * xn + yn * yn;
    const double d = 1.0 + k1 * r2 + k2 * r2 * r2 + k3 * r2 * r2 * r2;
    const double dd_dr2 = k1 + 2.0 * k2 * r2 + 3.0 * k3 * r2 * r2;
    const double xd = xn * d + 2.0 * p1 * xn * yn + p2 * (r2 + 2.0 * xn * xn);
    const double yd = yn * d + p1 * (r2 + 2.0 * yn * yn) + 2.0 * p2 * xn * yn;

    /* d(xd, yd)/d(xn, yn) */
    const double dxd_dxn = d + xn * dd_dr2 * 2.0 * xn + 2.0 * p1 * yn + p2 * 6.0 * xn;
    const double dxd_dyn = xn * dd_dr2 * 2.0 * yn + 2.0 * p1 * xn + p2 * 2.0 * yn;
    const double dyd_dxn = yn * dd_dr2 * 2.0 * xn + p1 * 2.0 * xn + 2.0 * p2 * yn;
    const double dyd_dyn = d + yn * dd_dr2 * 2.0 * yn + p1 * 6.0 * yn + 2.0 * p2 * xn;
    /* d(xn, yn)/dX */
    const double iz = 1.0 / X[2];
    const double dxn_dX[3] = {iz, 0.0, -X[0] * iz * iz};
    const double dyn_dX[3] = {0.0, iz, -X[1] * iz * iz};
    for (int k = 0; k < 3; ++k) {
        J_X[k] = fx * (dxd_dxn * dxn_dX[k] + dxd_dyn * dyn_dX[k]);
        J_X[3 + k] = fy * (dyd_dxn * dxn_dX[k] + dyd_dyn * dyn_dX[k]);
    }
    /* intrinsics: fx, fy, cx, cy, k1, k2 */
    J_K[0] = xd;  J_K[1] = 0.0; J_K[2] = 1.0; J_K[3] = 0.0;
    J_K[4] = fx * xn * r2;  J_K[5] = fx * xn * r2 * r2;
    J_K[6] = 0.0; J_K[7] = yd;  J_K[8] = 0.0; J_K[9] = 1.0;
    J_K[10] = fy * yn * r2; J_K[11] = fy * yn * r2 * r2;
}

/* ------------------------------------------------------------------ */
/* Backward (Eqs. induce, gradp, spatialderiv; chain rule Eq. partial)  */
/* ------------------------------------------------------------------ */

/*
 * orc_backward: one camera, after orc_forward.
 * Inputs: the forward's keys, cnt, img (FP64), pix, zf; the upstream
 * gradient G = dL/dI over the pyramid (same layout as img).
 * all_projected = 0: spatial gradients only for points in Lambda of their own
 *   pixel (the point "projected at p" that is shown there); 1: for every
 *   point that lands inside the layer.
 * Outputs (overwritten, FP64):
 *   dfeat n x c    dL/dtau: sum over layers of [i in Lambda] G(p)/|Lambda(p)|
 *   dxyz  n x 3    dL/dx
 *   dpose 6        dL/dxi for the left increment exp(xi)(R,t), xi = (nu, omega)
 *   dintr 6        dL/d(fx, fy, cx, cy, k1, k2)
 *   dpose_abs, dintr_abs  sum of |per (point, layer) term| (error scale)
 *   gu, gv  n x levels   the layer-pixel gradients g_u, g_v (may be NULL)
 * sample (NULL = every point): n_sample point indices to visit instead of all
 *   n; the other rows stay zero and the reduced sums cover the sample only.
 *   It restricts which points are visited, not what is computed for one.
 * threads: as in orc_forward.  Per-point outputs do not depend on it; the
 *   reduced sums are added per thread, then over the threads in order, so
 *   with more than one thread they may differ from one thread's in FP64
 *   rounding.
 *
 * Induced change D at a target pixel q one pixel away (Eq. spatialderiv,
 * read with the conditions on the target q):
 *   q outside the layer                     -> 0
 *   Lambda(q) empty                         -> tau - I(q)   (I(q) = background)
 *   z > f32(min_z(q) (1+alpha))             -> 0            (behind)
 *   f32(z (1+alpha)) < min_z(q)             -> tau - I(q)   (in front)
 *   otherwise (fuzzy-equal)                 -> (|Lambda| I(q) + tau)/(1+|Lambda|) - I(q)
 * Eq. gradp with the shift to u-1 having du = -1, contracted with G at the
 * target:  g_u = 1/2 ( <G(u+1,v), D(u+1,v)> - <G(u-1,v), D(u-1,v)> ), and
 * likewise g_v from (u, v+-1).  g is in layer pixels; the layer scale 2^-l
 * maps it to layer-0 pixels.
 */
int orc_backward(int64_t n, const float* xyz, int32_t c, const double* feat,
                 const orc_intrinsics* K, const orc_pose* T, int32_t levels, float alpha,
                 const double* background, int32_t all_projected, int32_t log_desc,
                 const uint64_t* keys, const uint32_t* cnt, const double* img,
                 const int32_t* pix, const float* zf, const double* G,
                 double* dfeat, double* dxyz, double* dpose, double* dintr,
                 double* dpose_abs, double* dintr_abs, double* gu_out, double* gv_out,
                 const int64_t* sample, int64_t n_sample, int32_t threads) {
    const float a1 = 1.0f + alpha;
    const int nt = team_size(threads);
    const double* feat_stored = feat;
    double* lin = NULL;
    if (log_desc) { /* blend and induced changes act on exp(tau) (Sec. 3.2) */
        lin = (double*)malloc(sizeof(double) * (size_t)(n * c + 1));
        if (!lin) return -1;
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t j = 0; j < n * c; ++j) lin[j] = exp(feat_stored[j]);
        feat = lin;
    }
    for (int k = 0; k < 6; ++k) dpose[k] = dintr[k] = dpose_abs[k] = dintr_abs[k] = 0.0;
    for (int64_t i = 0; i < n * c; ++i) dfeat[i] = 0.0;
    for (int64_t i = 0; i < n * 3; ++i) dxyz[i] = 0.0;
    if (gu_out)
        for (int64_t i = 0; i < n * levels; ++i) gu_out[i] = gv_out[i] = 0.0;

    /* The points visited: all of them in index order, or the given sample
     * (point indices; only their rows of dfeat, dxyz, gu, gv are written and
     * only their terms enter the reduced sums).  Every point's own outputs
     * depend on nothing but its own terms; the reduced sums (pose,
     * intrinsics) are summed point by point within each thread's contiguous
     * share of the list, then over the threads in order. */
    const int64_t m = sample ? n_sample : n;
    double* part = (double*)calloc((size_t)nt * 24, sizeof(double));
    if (!part) {
        free(lin);
        return -1;
    }
    int failed = 0;
#pragma omp parallel num_threads(nt) reduction(| : failed)
    {
        const int t = thread_id(), tt = threads_in_team();
        const int64_t j0 = m * t / tt, j1 = m * (t + 1) / tt;
        double* acc = part + 24 * t; /* dpose, dintr, dpose_abs, dintr_abs */
        double* D = (double*)malloc(sizeof(double) * (size_t)(c > 0 ? c : 1));
        if (!D) failed = 1;
        for (int64_t j = j0; D && j < j1; ++j) {
            const int64_t i = sample ? sample[j] : j;
            const double* tau = feat + i * c;
            double dL_du0 = 0.0, dL_dv0 = 0.0;
            double tu[8], tv[8]; /* per layer contributions to du0, dv0 */
            for (int l = 0; l < levels; ++l) {
                tu[l] = tv[l] = 0.0;
                int32_t p = pix[i * levels + l];
                if (p < 0) continue;
                const int32_t wl = K->w >> l, hl = K->h >> l;
                const int64_t np = (int64_t)wl * hl;
                const int64_t off = layer_offset(K->w, K->h, l);
                const double* Il = img + c * off;
                const double* Gl = G + c * off;
                float minz_p = bits_f32((uint32_t)(keys[off + p] >> 32));
                int in_lambda = (zf[i] <= minz_p * a1);

                /* Feature gradient: d mean / d tau_i = 1/|Lambda| for members. */
                if (in_lambda)
                    for (int ch = 0; ch < c; ++ch)
                        dfeat[i * c + ch] += Gl[(int64_t)ch * np + p] / (double)cnt[off + p];

                if (!in_lambda && !all_projected) continue;
                const int32_t pu = p % wl, pv = p / wl;
                const int32_t du[4] = {+1, -1, 0, 0};
                const int32_t dv[4] = {0, 0, +1, -1};
                double contrib[4];
                for (int s = 0; s < 4; ++s) {
                    contrib[s] = 0.0;
                    int32_t qu = pu + du[s], qv = pv + dv[s];
                    if (qu < 0 || qu >= wl || qv < 0 || qv >= hl) continue;
                    int64_t q = (int64_t)qv * wl + qu;
                    uint32_t nq = cnt[off + q];
                    float minz_q = bits_f32((uint32_t)(keys[off + q] >> 32));
                    for (int ch = 0; ch < c; ++ch) {
                        double Iq = Il[(int64_t)ch * np + q];
                        if (nq == 0)
                            D[ch] = tau[ch] - Iq; /* background overwritten */
                        else if (zf[i] > minz_q * a1)
                            D[ch] = 0.0; /* behind the target's surface */
                        else if (zf[i] * a1 < minz_q)
                            D[ch] = tau[ch] - Iq; /* in front: replaces the mean */
                        else
                            D[ch] = ((double)nq * Iq + tau[ch]) / (1.0 + (double)nq) - Iq;
                    }
                    double dot = 0.0;
                    for (int ch = 0; ch < c; ++ch) dot += Gl[(int64_t)ch * np + q] * D[ch];
                    contrib[s] = dot;
                }
                double g_u = 0.5 * (contrib[0] - contrib[1]);
                double g_v = 0.5 * (contrib[2] - contrib[3]);
                if (gu_out) {
                    gu_out[i * levels + l] = g_u;
                    gv_out[i * levels + l] = g_v;
                }
                double sc = ldexp(1.0, -l);
                tu[l] = g_u * sc;
                tv[l] = g_v * sc;
                dL_du0 += tu[l];
                dL_dv0 += tv[l];
            }
            if (dL_du0 == 0.0 && dL_dv0 == 0.0) {
                int any = 0;
                for (int l = 0; l < levels; ++l) any |= (tu[l] != 0.0 || tv[l] != 0.0);
                if (!any) continue;
            }
            double uv[2], X[3], J_X[6], J_K[12];
            orc_project_jac_f64(K, T, xyz + 3 * i, uv, X, J_X, J_K);
            double dX[3];
            for (int k = 0; k < 3; ++k) dX[k] = J_X[k] * dL_du0 + J_X[3 + k] * dL_dv0;
            /* dL/dx = R^T dL/dX */
            for (int k = 0; k < 3; ++k)
                dxyz[i * 3 + k] = (double)T->R[0 * 3 + k] * dX[0] + (double)T->R[1 * 3 + k] * dX[1] +
                                  (double)T->R[2 * 3 + k] * dX[2];
            /* Left increment exp(xi)(R,t): X' = X + nu + omega x X, so
             * dL/dnu = dL/dX and dL/domega = X x dL/dX. */
            double dxi[6] = {dX[0], dX[1], dX[2],
                             X[1] * dX[2] - X[2] * dX[1],
                             X[2] * dX[0] - X[0] * dX[2],
                             X[0] * dX[1] - X[1] * dX[0]};
            for (int k = 0; k < 6; ++k) {
                acc[k] += dxi[k];
                double dk = J_K[k] * dL_du0 + J_K[6 + k] * dL_dv0;
                acc[6 + k] += dk;
            }
            /* error scale: sum of the magnitudes of each layer's own term */
            for (int l = 0; l < levels; ++l) {
                if (tu[l] == 0.0 && tv[l] == 0.0) continue;
                double eX[3];
                for (int k = 0; k < 3; ++k) eX[k] = J_X[k] * tu[l] + J_X[3 + k] * tv[l];
                double exi[6] = {eX[0], eX[1], eX[2],
                                 X[1] * eX[2] - X[2] * eX[1],
                                 X[2] * eX[0] - X[0] * eX[2],
                                 X[0] * eX[1] - X[1] * eX[0]};
                for (int k = 0; k < 6; ++k) {
                    acc[12 + k] += fabs(exi[k]);
                    acc[18 + k] += fabs(J_K[k] * tu[l] + J_K[6 + k] * tv[l]);
                }
            }
        }
        free(D);
    }
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 6; ++k) {
            dpose[k] += part[24 * t + k];
            dintr[k] += part[24 * t + 6 + k];
            dpose_abs[k] += part[24 * t + 12 + k];
            dintr_abs[k] += part[24 * t + 18 + k];
        }
    free(part);
    if (log_desc) /* d exp(tau) / d tau = exp(tau) */
        for (int64_t j = 0; j < n * c; ++j) dfeat[j] *= lin[j];
    free(lin);
    return failed ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Photometric epilogue on layer 0 (Sec. 3.3)                           */
/* ------------------------------------------------------------------ */

/* Response curve R_ch(x) of one channel and its derivative.  crf_n < 2: the
 * identity.  Otherwise a LUT of crf_n samples on [0,1] with linear
 * interpolation; outside [0,1] the input is clamped (inference), or, with
 * leaky != 0, the training response of Eq. resonseleak with alpha = 0.01:
 * alpha x below 0 and -alpha / sqrt(x) + alpha + 1 above 1. */
static double response(const double* lut, int32_t crf_n, int leaky, double x, double* dy, int32_t* seg,
                       double* frac) {
    *seg = -1;
    *frac = 0.0;
    if (crf_n < 2) {
        *dy = 1.0;
        return x;
    }
    const double a = 0.01;
    if (leaky && x < 0.0) {
        *dy = a;
        return a * x;
    }
    if (leaky && x > 1.0) {
        *dy = a / (2.0 * x * sqrt(x));
        return -a / sqrt(x) + a + 1.0;
    }
    double xc = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
    double pos = xc * (crf_n - 1);
    int32_t i0 = (int32_t)floor(pos);
    if (i0 > crf_n - 2) i0 = crf_n - 2;
    double f = pos - i0;
    *seg = i0;
    *frac = f;
    *dy = (x < 0.0 || x > 1.0) ? 0.0 : (lut[i0 + 1] - lut[i0]) * (crf_n - 1);
    return lut[i0] * (1.0 - f) + lut[i0 + 1] * f;
}

/*
 * In-place on the layer-0 planes of img (c x h x w), channels 0..min(c,3)-1:
 *   I_e = I / 2^EV                         (exposure)
 *   I_w = I_e * wb[ch]                     (white balance, multiplicative)
 *   I_v = I_w * (1 + a2 r^2 + a4 r^4 + a6 r^6),
 *         r = |(u/w, v/h) - c_v|           (vignette, normalised coords)
 *   out = R_ch(I_v)                        (response curve, see response())
 * If grad is not NULL it receives d out / d I per element (same layout), for
 * chaining an upstream gradient through the epilogue.
 */
void orc_epilogue(int32_t w, int32_t h, int32_t c, double* img, double ev, const double* wb,
                  const double* vig_c, const double* vig_a, const double* crf_lut, int32_t crf_n,
                  int32_t leaky, double* grad) {
    const int64_t np = (int64_t)w * h;
    const int cc = c < 3 ? c : 3;
    const double e = pow(2.0, -ev);
    for (int ch = 0; ch < cc; ++ch) {
        for (int32_t v = 0; v < h; ++v) {
            for (int32_t u = 0; u < w; ++u) {
                int64_t p = (int64_t)v * w + u;
                double ru = (double)u / w - vig_c[0];
                double rv = (double)v / h - vig_c[1];
                double r2 = ru * ru + rv * rv;
                double vig = 1.0 + vig_a[0] * r2 + vig_a[1] * r2 * r2 + vig_a[2] * r2 * r2 * r2;
                double scale = e * wb[ch] * vig;
                double x = img[(int64_t)ch * np + p] * scale;
                double dy, f;
                int32_t seg;
                double y = response(crf_lut ? crf_lut + (int64_t)ch * crf_n : NULL, crf_n, leaky, x, &dy, &seg, &f);
                img[(int64_t)ch * np + p] = y;
                if (grad) grad[(int64_t)ch * np + p] = dy * scale;
            }
        }
    }
    if (grad)
        for (int ch = cc; ch < c; ++ch)
            for (int64_t p = 0; p < np; ++p) grad[(int64_t)ch * np + p] = 1.0;
}

/*
 * Gradients of L with respect to the photometric parameters of one image
 * (Sec. 3.3), given the layer-0 image before the epilogue (img, c x h x w)
 * and dL/d(out) (G, same layout):
 *   gp[0] dL/dEV, gp[1..3] dL/dwb, gp[4..5] dL/dc_v, gp[6..8] dL/d(a2, a4, a6)
 *   gcrf[ch * crf_n + j] dL/dlut[ch][j] (NULL = not computed)
 *   gp_abs  the sum of |term| of each gp entry (error scale)
 * Overwritten.  Sums in FP64.
 */
void orc_photometric_grad(int32_t w, int32_t h, int32_t c, const double* img, const double* G, double ev,
                          const double* wb, const double* vig_c, const double* vig_a, const double* crf_lut,
                          int32_t crf_n, int32_t leaky, double* gp, double* gcrf, double* gp_abs) {
    const int64_t np = (int64_t)w * h;
    const int cc = c < 3 ? c : 3;
    const double e = pow(2.0, -ev);
    for (int k = 0; k < 9; ++k) gp[k] = gp_abs[k] = 0.0;
    if (gcrf)
        for (int64_t j = 0; j < 3 * (int64_t)crf_n; ++j) gcrf[j] = 0.0;
    for (int ch = 0; ch < cc; ++ch) {
        for (int32_t v = 0; v < h; ++v) {
            for (int32_t u = 0; u < w; ++u) {
                int64_t p = (int64_t)v * w + u;
                double ru = (double)u / w - vig_c[0];
                double rv = (double)v / h - vig_c[1];
                double r2 = ru * ru + rv * rv;
                double vig = 1.0 + vig_a[0] * r2 + vig_a[1] * r2 * r2 + vig_a[2] * r2 * r2 * r2;
                double I = img[(int64_t)ch * np + p];
                double x = I * e * wb[ch] * vig;
                double dy, f;
                int32_t seg;
                response(crf_lut ? crf_lut + (int64_t)ch * crf_n : NULL, crf_n, leaky, x, &dy, &seg, &f);
                double g = G[(int64_t)ch * np + p];
                double gx = g * dy; /* dL/dx */
                /* dvig/dr2 and dr2/dc_v = -2 (p - c_v) */
                double dvig = vig_a[0] + 2.0 * vig_a[1] * r2 + 3.0 * vig_a[2] * r2 * r2;
                double base = gx * I * e * wb[ch];
                double t[9] = {gx * x * (-log(2.0)), 0.0, 0.0, 0.0, base * dvig * (-2.0 * ru),
                               base * dvig * (-2.0 * rv), base * r2, base * r2 * r2, base * r2 * r2 * r2};
                t[1 + ch] = gx * I * e * vig;
                for (int k = 0; k < 9; ++k) {
                    gp[k] += t[k];
                    gp_abs[k] += fabs(t[k]);
                }
                if (gcrf && crf_n >= 2) {
                    if (seg >= 0) {
                        gcrf[ch * crf_n + seg] += g * (1.0 - f);
                        gcrf[ch * crf_n + seg + 1] += g * f;
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* World radius for stochastic discarding (Sec. 3.1)                   */
/* ------------------------------------------------------------------ */

/* r_world[i] = distance from point i to its k-th nearest other point (the
 * paper uses k = 4), by exhaustive search in FP64; +inf if fewer than k
 * other points exist.  O(n^2): for test-sized clouds. */
void orc_knn_radius(int64_t n, const float* xyz, int32_t k, double* radius) {
    double best[64];
    for (int64_t i = 0; i < n; ++i) {
        int m = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = (double)xyz[3 * j] - xyz[3 * i];
            double dy = (double)xyz[3 * j + 1] - xyz[3 * i + 1];
            double dz = (double)xyz[3 * j + 2] - xyz[3 * i + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (m < k) {
                int q = m++;
                while (q > 0 && best[q - 1] > d2) { best[q] = best[q - 1]; --q; }
                best[q] = d2;
            } else if (d2 < best[k - 1]) {
                int q = k - 1;
                while (q > 0 && best[q - 1] > d2) { best[q] = best[q - 1]; --q; }
                best[q] = d2;
            }
        }
        radius[i] = m < k ? INFINITY : sqrt(best[k - 1]);
    }
}
