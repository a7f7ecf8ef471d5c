/*
 * FP64 CPU oracle for the NVGS per-frame render pass — TEST INFRASTRUCTURE ONLY.
 *
 * This file is a plain, slow, obviously-correct restatement of what the render pass computes
 * (NVGS, "Neural Visibility for Occlusion Culling in 3D Gaussian Splatting"), used by the tests,
 * by the package smoke check and by the bench's CPU-baseline leg.  It shares no code, header,
 * table or constant generator with the CUDA library and must never be linked into it.
 *
 * Every quantity is double precision.  Steps follow the paper's order:
 *   Sec. 3.1, Eq. 1        per-asset distance bounds d = r / (tan(theta/2) p)
 *   Sec. 3.3               frustum culling on the Gaussian mean, MLP gating by the minimum
 *                          distance, global-to-local transform of the MLP inputs
 *   Sec. 3.3, Eq. 2        distance correction d_t = d_r (f_t / f_r) / s, min-max normalised
 *   Sec. 3.2               the visibility MLP (shape fixed by the workload: 32-64-64-64-1)
 *   Sec. 3.3 (3DGS)        EWA projection, SH colour, tiled rasterisation
 *   Sec. 4.1               blending: skip alpha < 1/255, stop once T < 1e-4
 *   Sec. 3.1               contribution C = alpha * T; a Gaussian is visible iff it blends
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - alpha is clamped at 0.99 and 0.3 px^2 is added to the 2D covariance (3DGS convention);
 *   - a fragment whose T (1 - alpha) would drop below t_stop is not blended and ends the pixel;
 *   - the support of a splat is the exact ellipse {alpha >= alpha_min}; its axis-aligned bounding
 *     box selects candidate pixels and tiles, so binning never changes the image;
 *   - the frustum keeps z > z_near and |x|, |y| within 1.3x the half field of view;
 *   - depth ties are broken by (instance, gaussian) index;
 *   - MLP inputs: [p, sin(2^k pi p), cos(2^k pi p) (k = 0..3), view dir, normalised log d_t, 0].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t pad_;
    const double* means;          /* n*3 */
    const double* log_scales;     /* n*3 */
    const double* quats;          /* n*4, (w, x, y, z), not necessarily normalised */
    const double* opacity_logits; /* n */
    const double* sh;             /* n*K*3, K = (deg+1)^2, coefficient-major, RGB innermost */
    double bbox_min[3];
    double bbox_max[3];
    double d_min, d_max;          /* Eq. 1 distance bounds (asset-local units) */
    double train_focal;           /* f_t = 1 / tan(theta_t / 2) */
} or_asset;

typedef struct {
    int32_t asset_id;
    int32_t pad_;
    double R[9];   /* row-major, orthonormal */
    double t[3];
    double s;
} or_instance;

typedef struct {
    double R[9];   /* world -> camera rotation, row-major */
    double t[3];
    double fx, fy, cx, cy;
    int32_t width, height;
    double z_near;
} or_camera;

typedef struct {
    double alpha_min;      /* 1/255 */
    double alpha_max;      /* 0.99 */
    double t_stop;         /* 1e-4 */
    double dilation;       /* 0.3 px^2 */
    double guard_band;     /* 1.3 */
    double bg[3];
    int32_t tile_size;
    int32_t pad_;
    /* half-widths of the ambiguity bands (relative unless stated) */
    double eps_alpha;      /* |alpha - alpha_min| <= eps_alpha * alpha_min */
    double eps_t;          /* |T(1-alpha) - t_stop| <= eps_t * t_stop */
    double eps_depth;      /* |z1 - z2| <= eps_depth * z1 between neighbours in depth order */
    double eps_frustum;    /* |margin| <= eps_frustum * z */
    double eps_px;         /* support bounding box within eps_px pixels of a pixel/tile edge */
    double swap_tol;       /* a near-tie in depth only counts if swapping changes a channel by more */
    double radius_clip_area; /* Sec. 4.4 radius clipping: drop a splat whose 1-sigma ellipse area
                                pi sqrt(det Sigma_2D) is below this (px^2); 0: off */
    double eps_clip;       /* |det - threshold| <= eps_clip * threshold: the clip decision is ambiguous */
} or_opts;

typedef struct {
    int32_t valid;         /* in frustum, kept, non-empty support */
    int32_t ambiguous;     /* some decision lies inside its ambiguity band */
    int32_t instance, gaussian;
    double u, v, depth;
    double cov[3];         /* 2D covariance incl. dilation: (a, b, c) = [[a, b], [b, c]] */
    double conic[3];       /* its inverse, same packing */
    double opacity;
    double rgb[3];
    double x_ext, y_ext;   /* half-extents of the {alpha >= alpha_min} ellipse's bounding box */
    int32_t px_min[2], px_max[2];       /* inclusive pixel bbox, clamped; empty if min > max */
    int32_t tile_min[2], tile_max[2];   /* inclusive tile rect; empty if min > max */
} or_splat;

/* ------------------------------------------------------------------ small linear algebra */
static void mat3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
static void mat3_transpose(const double* A, double* T) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * j + i] = A[3 * i + j];
}
static void mat3_vec(const double* A, const double* x, double* y) {
    for (int i = 0; i < 3; i++) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}

/* Rotation matrix of the normalised quaternion q = (w, x, y, z). */
void or_quat_to_rot(const double* q_in, double* R) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* 3D covariance Sigma = R(q) diag(exp(2 ls)) R(q)^T (3DGS parameterisation), row-major 3x3. */
void or_cov3d(const double* log_scale, const double* quat, double* Sigma) {
    double R[9], M[9];
    or_quat_to_rot(quat, R);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[3 * i + j] = R[3 * i + j] * exp(log_scale[j]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += M[3 * i + k] * M[3 * j + k];
            Sigma[3 * i + j] = s;
        }
}

/* ------------------------------------------------------------------ Sec. 3.1, Eq. 1 */
/* Camera distance at which the asset's bounding-box diagonal (half-length r) covers the
 * fraction p of a view with field of view theta. */
double or_distance_bound(double r, double theta, double p) { return r / (tan(theta / 2.0) * p); }

/* Per-asset constants of Sec. 3.1: the bounding box of the means, the near / far camera
 * distances by Eq. 1 (r = half the box diagonal, p = p_near / p_far of the view covered at the
 * training field of view theta_t), and the training focal f_t = 1 / tan(theta_t / 2).  A
 * positive override replaces the Eq. 1 value. */
void or_asset_prepare(or_asset* a, double theta_t, double p_near, double p_far,
                      double d_min_override, double d_max_override) {
    for (int k = 0; k < 3; k++) { a->bbox_min[k] = INFINITY; a->bbox_max[k] = -INFINITY; }
    for (int64_t g = 0; g < a->n; g++)
        for (int k = 0; k < 3; k++) {
            double v = a->means[3 * g + k];
            if (v < a->bbox_min[k]) a->bbox_min[k] = v;
            if (v > a->bbox_max[k]) a->bbox_max[k] = v;
        }
    double dd = 0.0;
    for (int k = 0; k < 3; k++) dd += (a->bbox_max[k] - a->bbox_min[k]) * (a->bbox_max[k] - a->bbox_min[k]);
    double r = 0.5 * sqrt(dd);
    a->d_min = d_min_override > 0.0 ? d_min_override : or_distance_bound(r, theta_t, p_near);
    a->d_max = d_max_override > 0.0 ? d_max_override : or_distance_bound(r, theta_t, p_far);
    a->train_focal = 1.0 / tan(theta_t / 2.0);
}

/* ------------------------------------------------------------------ O1: frustum */
/* Returns 1 if the camera-space point is kept; *margin is the smallest signed distance to the
 * guard-band planes (positive inside), in the units of z. */
static int frustum_test(const or_camera* cam, const or_opts* o, const double* xc, double* margin) {
    double tx = o->guard_band * (cam->width / (2.0 * cam->fx));
    double ty = o->guard_band * (cam->height / (2.0 * cam->fy));
    double z = xc[2];
    double m0 = z - cam->z_near;
    double m1 = tx * z - fabs(xc[0]);
    double m2 = ty * z - fabs(xc[1]);
    double m = m0 < m1 ? m0 : m1;
    m = m < m2 ? m : m2;
    *margin = m;
    return (z > cam->z_near) && (fabs(xc[0]) <= tx * z) && (fabs(xc[1]) <= ty * z);
}

static void world_point(const or_instance* in, const double* mu, double* xw) {
    double sm[3] = {in->s * mu[0], in->s * mu[1], in->s * mu[2]};
    mat3_vec(in->R, sm, xw);
    for (int k = 0; k < 3; k++) xw[k] += in->t[k];
}

static void camera_point(const or_camera* cam, const double* xw, double* xc) {
    mat3_vec(cam->R, xw, xc);
    for (int k = 0; k < 3; k++) xc[k] += cam->t[k];
}

static void camera_center(const or_camera* cam, double* c) {
    /* c = -R^T t */
    for (int j = 0; j < 3; j++)
        c[j] = -(cam->R[j] * cam->t[0] + cam->R[3 + j] * cam->t[1] + cam->R[6 + j] * cam->t[2]);
}

/* Camera centre in the instance's local frame: R_i^T (c - t_i) / s_i (Sec. 3.3). */
static void local_camera_center(const or_camera* cam, const or_instance* in, double* cl) {
    double c[3], d[3];
    camera_center(cam, c);
    for (int k = 0; k < 3; k++) d[k] = c[k] - in->t[k];
    for (int j = 0; j < 3; j++)
        cl[j] = (in->R[j] * d[0] + in->R[3 + j] * d[1] + in->R[6 + j] * d[2]) / in->s;
}

static int64_t instance_offset(const or_asset* assets, const or_instance* inst, int i) {
    int64_t off = 0;
    for (int k = 0; k < i; k++) off += assets[inst[k].asset_id].n;
    return off;
}

/* Per instanced Gaussian (instance-major order): frustum decision and ambiguity. */
void or_frustum(const or_asset* assets, const or_instance* inst, int n_inst, const or_camera* cam,
                const or_opts* o, uint8_t* in_frustum, uint8_t* ambiguous) {
    for (int i = 0; i < n_inst; i++) {
        const or_asset* a = &assets[inst[i].asset_id];
        int64_t off = instance_offset(assets, inst, i);
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < a->n; g++) {
            double xw[3], xc[3], m;
            world_point(&inst[i], &a->means[3 * g], xw);
            camera_point(cam, xw, xc);
            in_frustum[off + g] = (uint8_t)frustum_test(cam, o, xc, &m);
            if (ambiguous) ambiguous[off + g] = fabs(m) <= o->eps_frustum * fabs(xc[2]) + 1e-300;
        }
    }
}

/* ------------------------------------------------------------------ O2: MLP input + forward */
#define OR_MLP_IN 32
#define OR_MLP_H 64
#define OR_MLP_NW (64 * 32 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1)

/* Normalised focal length of a pinhole camera: 1 / tan(fov_x / 2) = 2 fx / W. */
static double render_focal(const or_camera* cam) { return 2.0 * cam->fx / cam->width; }

/* Eq. 2 followed by the min-max map of Sec. 3.3, applied to log distance and clamped. */
double or_normalised_distance(double d_local, double f_t, double f_r, double d_min, double d_max) {
    double dt = d_local * (f_t / f_r);   /* the 1/s of Eq. 2 is already inside d_local */
    double x = 2.0 * (log(dt) - log(d_min)) / (log(d_max) - log(d_min)) - 1.0;
    if (x < -1.0) x = -1.0;
    if (x > 1.0) x = 1.0;
    return x;
}

/* The 32 MLP inputs of Gaussian mean mu (asset-local) seen from local camera centre cl. */
void or_mlp_features(const or_asset* a, const double* mu, const double* cl, double f_r,
                     double* f) {
    double p[3];
    for (int k = 0; k < 3; k++) {
        double c = 0.5 * (a->bbox_min[k] + a->bbox_max[k]);
        double e = a->bbox_max[k] - a->bbox_min[k];
        if (!(e > 0.0)) e = 1.0;
        p[k] = 2.0 * (mu[k] - c) / e;
    }
    for (int k = 0; k < 3; k++) f[k] = p[k];
    for (int fr = 0; fr < 4; fr++) {
        double w = ldexp(OR_PI, fr); /* 2^fr * pi */
        for (int k = 0; k < 3; k++) {
            f[3 + 3 * fr + k] = sin(w * p[k]);
            f[15 + 3 * fr + k] = cos(w * p[k]);
        }
    }
    double d[3] = {mu[0] - cl[0], mu[1] - cl[1], mu[2] - cl[2]};
    double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; k++) f[27 + k] = d[k] / dist;
    f[30] = or_normalised_distance(dist, a->train_focal, f_r, a->d_min, a->d_max);
    f[31] = 0.0;
}

/* One dense layer y = W x + b with W stored (out, in), explicit loops. */
static void dense(const double* W, const double* b, const double* x, int n_in, int n_out,
                  int relu, double* y) {
    for (int o = 0; o < n_out; o++) {
        double s = b[o];
        for (int i = 0; i < n_in; i++) s += W[(int64_t)o * n_in + i] * x[i];
        y[o] = (relu && s < 0.0) ? 0.0 : s;
    }
}

/* Visibility logit of one feature vector; weights flat: W1 b1 W2 b2 W3 b3 W4 b4. */
double or_mlp_forward_one(const double* w, const double* f) {
    const double *W1 = w, *b1 = W1 + 64 * 32, *W2 = b1 + 64, *b2 = W2 + 64 * 64,
                 *W3 = b2 + 64, *b3 = W3 + 64 * 64, *W4 = b3 + 64, *b4 = W4 + 64;
    double h1[64], h2[64], h3[64], out;
    dense(W1, b1, f, 32, 64, 1, h1);
    dense(W2, b2, h1, 64, 64, 1, h2);
    dense(W3, b3, h2, 64, 64, 1, h3);
    dense(W4, b4, h3, 64, 1, 0, &out);
    return out;
}

void or_mlp_forward(const double* w, int64_t n, const double* feats, double* logits) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) logits[i] = or_mlp_forward_one(w, &feats[32 * i]);
}

/* Per instanced Gaussian: the MLP logit (NaN-free) and whether the instance bypasses the MLP
 * because its corrected centre distance is below d_min (Sec. 3.3 gating).  Features are
 * returned too when feats != NULL (32 per Gaussian). */
/* Per instance: the camera centre in its local frame and whether it bypasses the MLP (Sec. 3.3:
 * its bounding-box centre is closer than the asset's minimum distance, with the Eq. 2 focal
 * correction). */
static int instance_gate(const or_asset* a, const or_instance* in, const or_camera* cam, double f_r,
                         int gate, double* cl) {
    local_camera_center(cam, in, cl);
    double bc[3], dd = 0.0;
    for (int k = 0; k < 3; k++) {
        bc[k] = 0.5 * (a->bbox_min[k] + a->bbox_max[k]);
        dd += (bc[k] - cl[k]) * (bc[k] - cl[k]);
    }
    double d_centre = sqrt(dd) * (a->train_focal / f_r);
    return gate && (d_centre < a->d_min);
}

void or_visibility(const or_asset* assets, const or_instance* inst, int n_inst,
                   const or_camera* cam, const double* weights, int gate, double* logits,
                   uint8_t* gated, double* feats) {
    double f_r = render_focal(cam);
    for (int i = 0; i < n_inst; i++) {
        const or_asset* a = &assets[inst[i].asset_id];
        int64_t off = instance_offset(assets, inst, i);
        double cl[3];
        int bypass = instance_gate(a, &inst[i], cam, f_r, gate, cl);
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < a->n; g++) {
            double f[32];
            or_mlp_features(a, &a->means[3 * g], cl, f_r, f);
            if (feats) memcpy(&feats[32 * (off + g)], f, sizeof f);
            logits[off + g] = weights ? or_mlp_forward_one(weights, f) : 0.0;
            if (gated) gated[off + g] = (uint8_t)bypass;
        }
    }
}

/* or_visibility at sampled instanced Gaussians: entry s of the outputs is Gaussian idx[s] of the
 * instance-major order, computed exactly as or_visibility computes it (feats: 32 per entry,
 * nullable).  For checks at scene sizes where evaluating every Gaussian in FP64 takes minutes.
 * Returns 0, or -1 for an index outside [0, total) or a failed allocation. */
int or_visibility_at(const or_asset* assets, const or_instance* inst, int n_inst,
                     const or_camera* cam, const double* weights, int gate, const int64_t* idx,
                     int64_t n_idx, double* logits, uint8_t* gated, double* feats) {
    double f_r = render_focal(cam);
    int64_t* offs = (int64_t*)malloc(((size_t)n_inst + 1) * sizeof *offs);
    if (!offs) return -1;
    offs[0] = 0;
    for (int i = 0; i < n_inst; i++) offs[i + 1] = offs[i] + assets[inst[i].asset_id].n;
    for (int64_t s = 0; s < n_idx; s++)
        if (idx[s] < 0 || idx[s] >= offs[n_inst]) { free(offs); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n_idx; s++) {
        int lo = 0, hi = n_inst - 1;   /* last instance whose first index is <= idx[s] */
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (offs[mid] <= idx[s]) lo = mid; else hi = mid - 1;
        }
        const or_asset* a = &assets[inst[lo].asset_id];
        const int64_t g = idx[s] - offs[lo];
        double cl[3], f[32];
        int bypass = instance_gate(a, &inst[lo], cam, f_r, gate, cl);
        or_mlp_features(a, &a->means[3 * g], cl, f_r, f);
        if (feats) memcpy(&feats[32 * s], f, sizeof f);
        logits[s] = weights ? or_mlp_forward_one(weights, f) : 0.0;
        if (gated) gated[s] = (uint8_t)bypass;
    }
    free(offs);
    return 0;
}

/* ------------------------------------------------------------------ O4: SH colour */
/* Real spherical harmonics up to degree 3 at unit direction (x, y, z), in the sign convention of
 * the original 3DGS code (real parts of the Condon-Shortley complex harmonics).  The constants
 * are the normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0),
 * written out from that formula. */
void or_sh_basis(int degree, double x, double y, double z, double* Y) {
    const double pi = OR_PI;
    Y[0] = 0.5 / sqrt(pi);
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (degree < 2) return;
    double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    if (degree < 3) return;
    double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi),
           c3c = 0.25 * sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * sqrt(7.0 / pi),
           c3e = 0.25 * sqrt(105.0 / pi);
    Y[9] = -c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3.0 * y * y);
}

/* rgb = max(0, 0.5 + sum_k Y_k(dir) sh_k), dir = unit vector from camera to the mean in the
 * asset's local frame (the instance rotation is undone). */
static void sh_color(const or_asset* a, int64_t g, const double* dir, double* rgb) {
    double Y[16];
    int K = (a->sh_degree + 1) * (a->sh_degree + 1);
    or_sh_basis(a->sh_degree, dir[0], dir[1], dir[2], Y);
    const double* c = &a->sh[(int64_t)g * K * 3];
    for (int ch = 0; ch < 3; ch++) {
        double s = 0.5;
        for (int k = 0; k < K; k++) s += Y[k] * c[3 * k + ch];
        rgb[ch] = s < 0.0 ? 0.0 : s;
    }
}

/* ------------------------------------------------------------------ O3: EWA projection */
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

/* Project instanced Gaussian (i, g).  keep_flag is the culling decision made before projection
 * (frustum and, optionally, MLP); the record is filled even when it is not valid, so that
 * ambiguous splats still know their footprint. */
static void project_one(const or_asset* a, const or_instance* in, const or_camera* cam,
                        const or_opts* o, int i, int64_t g, int keep, int keep_amb,
                        or_splat* sp) {
    memset(sp, 0, sizeof *sp);
    sp->instance = i;
    sp->gaussian = (int32_t)g;
    const double* mu = &a->means[3 * g];
    double xw[3], xc[3], margin;
    world_point(in, mu, xw);
    camera_point(cam, xw, xc);
    int inside = frustum_test(cam, o, xc, &margin);
    int amb = keep_amb || fabs(margin) <= o->eps_frustum * fabs(xc[2]);
    sp->px_min[0] = sp->px_min[1] = 1;
    sp->px_max[0] = sp->px_max[1] = 0;
    sp->tile_min[0] = sp->tile_min[1] = 1;
    sp->tile_max[0] = sp->tile_max[1] = 0;
    if (xc[2] <= 1e-6) { sp->ambiguous = amb; return; }

    /* Sigma_c = s^2 (W R_i) Sigma (W R_i)^T */
    double S[9], M[9], MT[9], T1[9], Sc[9];
    or_cov3d(&a->log_scales[3 * g], &a->quats[4 * g], S);
    mat3_mul(cam->R, in->R, M);
    mat3_transpose(M, MT);
    mat3_mul(M, S, T1);
    mat3_mul(T1, MT, Sc);
    for (int k = 0; k < 9; k++) Sc[k] *= in->s * in->s;

    /* Jacobian of the perspective map at the mean, x/z and y/z clamped to the guard band */
    double z = xc[2];
    double limx = o->guard_band * (cam->width / (2.0 * cam->fx));
    double limy = o->guard_band * (cam->height / (2.0 * cam->fy));
    double tx = xc[0] / z, ty = xc[1] / z;
    tx = tx < -limx ? -limx : (tx > limx ? limx : tx);
    ty = ty < -limy ? -limy : (ty > limy ? limy : ty);
    double J[6] = {cam->fx / z, 0.0, -cam->fx * tx / z, 0.0, cam->fy / z, -cam->fy * ty / z};
    /* Sigma_2D = J Sigma_c J^T + dilation I */
    double JS[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            JS[3 * r + c] = J[3 * r] * Sc[c] + J[3 * r + 1] * Sc[3 + c] + J[3 * r + 2] * Sc[6 + c];
    double ca = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + o->dilation;
    double cb = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
    double cc = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + o->dilation;
    double det = ca * cc - cb * cb;
    sp->cov[0] = ca; sp->cov[1] = cb; sp->cov[2] = cc;
    if (!(det > 0.0)) { sp->ambiguous = amb; return; }
    sp->conic[0] = cc / det; sp->conic[1] = -cb / det; sp->conic[2] = ca / det;
    sp->u = cam->fx * xc[0] / z + cam->cx;
    sp->v = cam->fy * xc[1] / z + cam->cy;
    sp->depth = z;
    sp->opacity = sigmoid(a->opacity_logits[g]);

    /* colour at the local-frame viewing direction */
    double cl[3], dir[3], nrm = 0.0;
    local_camera_center(cam, in, cl);
    for (int k = 0; k < 3; k++) { dir[k] = mu[k] - cl[k]; nrm += dir[k] * dir[k]; }
    nrm = sqrt(nrm);
    for (int k = 0; k < 3; k++) dir[k] /= nrm;
    sh_color(a, g, dir, sp->rgb);

    /* radius clipping (Sec. 4.4): the 1-sigma ellipse {d : d^T Sigma_2D^-1 d <= 1} has area
       pi sqrt(det Sigma_2D); below the given area the splat is dropped */
    int clipped = 0;
    if (o->radius_clip_area > 0.0) {
        double thr = o->radius_clip_area / OR_PI;
        thr *= thr;
        clipped = det < thr;
        if (fabs(det - thr) <= o->eps_clip * thr) amb = 1;
    }

    /* exact support: {d : d^T conic d <= 2 ln(255 o)}; its bounding box */
    double kk = 2.0 * log(sp->opacity / o->alpha_min);
    if (fabs(sp->opacity - o->alpha_min) <= o->eps_alpha * o->alpha_min) amb = 1;
    int valid = inside && keep && kk > 0.0 && !clipped;
    if (kk > 0.0 && !clipped) {
        sp->x_ext = sqrt(kk * ca);
        sp->y_ext = sqrt(kk * cc);
        double lo_x = sp->u - sp->x_ext - 0.5, hi_x = sp->u + sp->x_ext - 0.5;
        double lo_y = sp->v - sp->y_ext - 0.5, hi_y = sp->v + sp->y_ext - 0.5;
        int x0 = (int)ceil(lo_x), x1 = (int)floor(hi_x);
        int y0 = (int)ceil(lo_y), y1 = (int)floor(hi_y);
        /* a bbox edge within eps_px of an integer may round the other way in FP32 */
        double e = o->eps_px;
        if (fabs(lo_x - rint(lo_x)) <= e || fabs(hi_x - rint(hi_x)) <= e ||
            fabs(lo_y - rint(lo_y)) <= e || fabs(hi_y - rint(hi_y)) <= e)
            sp->ambiguous |= 2; /* footprint (tile-list) ambiguity only */
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > cam->width - 1) x1 = cam->width - 1;
        if (y1 > cam->height - 1) y1 = cam->height - 1;
        sp->px_min[0] = x0; sp->px_min[1] = y0;
        sp->px_max[0] = x1; sp->px_max[1] = y1;
        if (x0 <= x1 && y0 <= y1) {
            int ts = o->tile_size;
            sp->tile_min[0] = floor_div(x0, ts); sp->tile_min[1] = floor_div(y0, ts);
            sp->tile_max[0] = floor_div(x1, ts); sp->tile_max[1] = floor_div(y1, ts);
        } else {
            valid = 0;
        }
    }
    sp->valid = valid;
    sp->ambiguous |= amb;
}

/* Project every instanced Gaussian (instance-major).  keep/keep_amb are nullable per-instanced
 * culling decisions (e.g. from MLP logits); NULL keeps everything in the frustum. */
void or_project(const or_asset* assets, const or_instance* inst, int n_inst, const or_camera* cam,
                const or_opts* o, const uint8_t* keep, const uint8_t* keep_amb, or_splat* out) {
    for (int i = 0; i < n_inst; i++) {
        const or_asset* a = &assets[inst[i].asset_id];
        int64_t off = instance_offset(assets, inst, i);
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < a->n; g++)
            project_one(a, &inst[i], cam, o, i, g, keep ? keep[off + g] : 1,
                        keep_amb ? keep_amb[off + g] : 0, &out[off + g]);
    }
}

/* ------------------------------------------------------------------ O5: exact compositing */
typedef struct {
    double z;
    int32_t inst, g;
    int64_t idx;      /* index into the splat array */
    double alpha;
    int ghost;        /* not blended (alpha just below alpha_min, or a culled ambiguous splat) */
    int amb;          /* reaching this fragment makes the pixel ambiguous */
} fragment;

static int frag_cmp(const void* pa, const void* pb) {
    const fragment* a = (const fragment*)pa;
    const fragment* b = (const fragment*)pb;
    if (a->z < b->z) return -1;
    if (a->z > b->z) return 1;
    if (a->inst != b->inst) return a->inst < b->inst ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return 0;
}

/* alpha of splat sp at pixel centre (px + 0.5, py + 0.5); *power_out receives the exponent. */
static double splat_alpha(const or_splat* sp, const or_opts* o, int px, int py, double* power_out) {
    double dx = (px + 0.5) - sp->u, dy = (py + 0.5) - sp->v;
    double power = -0.5 * (sp->conic[0] * dx * dx + sp->conic[2] * dy * dy) -
                   sp->conic[1] * dx * dy;
    *power_out = power;
    double al = sp->opacity * exp(power);
    return al < o->alpha_max ? al : o->alpha_max;
}

/* Front-to-back compositing of one pixel's fragments (Sec. 4.1).  Returns whether a decision
 * that FP32 could take the other way was reached before the pixel stopped. */
static int blend_pixel(fragment* fr, size_t nf, const or_splat* splats, const or_opts* o,
                       double* C, double* T_io, int32_t* n_contrib) {
    qsort(fr, nf, sizeof(fragment), frag_cmp);
    double T = 1.0;
    int amb = 0;
    for (size_t k = 0; k < nf; k++) {
        if (fr[k].amb) amb = 1;
        if (fr[k].ghost) continue;
        double al = fr[k].alpha;
        /* next blended neighbour in depth order */
        size_t k2 = k + 1;
        while (k2 < nf && fr[k2].ghost) k2++;
        if (k2 < nf && fr[k2].z - fr[k].z <= o->eps_depth * fr[k].z) {
            /* FP32 depths may order this pair the other way: blend the pair both ways from the
             * current T (stop rule included) and count the pixel as ambiguous only if the
             * colour or the transmittance handed on differs by more than swap_tol. */
            const double* ca = splats[fr[k].idx].rgb;
            const double* cb = splats[fr[k2].idx].rgb;
            double ab[2] = {al, fr[k2].alpha};
            const double* cc[2] = {ca, cb};
            double res[2][4];
            for (int ord = 0; ord < 2; ord++) {
                double t = T, c3[3] = {0.0, 0.0, 0.0};
                for (int q = 0; q < 2; q++) {
                    int e = ord ? 1 - q : q;
                    double ntq = t * (1.0 - ab[e]);
                    if (ntq < o->t_stop) { t = 0.0; break; }  /* stopped: nothing passes on */
                    for (int ch = 0; ch < 3; ch++) c3[ch] += ab[e] * t * cc[e][ch];
                    t = ntq;
                }
                res[ord][0] = c3[0]; res[ord][1] = c3[1]; res[ord][2] = c3[2]; res[ord][3] = t;
            }
            double d = 0.0;
            for (int ch = 0; ch < 4; ch++) d = fmax(d, fabs(res[0][ch] - res[1][ch]));
            if (d > o->swap_tol) amb = 1;
        }
        double nt = T * (1.0 - al);
        if (fabs(nt - o->t_stop) <= o->eps_t * o->t_stop) amb = 1;
        if (nt < o->t_stop) break;
        const double* c = splats[fr[k].idx].rgb;
        for (int ch = 0; ch < 3; ch++) C[ch] += al * T * c[ch];
        T = nt;
        if (n_contrib) {
#pragma omp atomic
            n_contrib[fr[k].idx]++;
        }
    }
    *T_io = T;
    return amb;
}

/* Composite the listed splats front to back at every requested pixel row.
 *   splats, n_splats : candidates (valid or merely ambiguous); only valid ones are blended
 *   rows, n_rows     : the image rows to produce (all rows if rows == NULL)
 *   image            : n_rows * W * 3 (bg applied)
 *   T_final          : nullable, n_rows * W
 *   n_contrib        : nullable, per splat: number of pixels where it was blended (Sec. 3.1)
 *   amb_px           : nullable, n_rows * W, 1 where a decision that FP32 arithmetic could take
 *                      the other way is reached before the pixel stops
 *   brute_force      : 1 = ignore the support bbox and test every splat at every pixel
 * Candidates are bucketed by row and, inside a row, by 16-pixel column; both only skip pixels
 * outside a splat's exact-support bounding box (pinned against brute force). */
void or_composite(const or_splat* splats, int64_t n_splats, const or_camera* cam,
                  const or_opts* o, const int32_t* rows, int n_rows, double* image,
                  double* T_final, int32_t* n_contrib, uint8_t* amb_px, int brute_force) {
    int W = cam->width;
    int nr = rows ? n_rows : cam->height;
    const int CW = 16;
    int ncol = (W + CW - 1) / CW;
    /* row buckets: which splats have a (possibly ambiguous) footprint on row y */
    int32_t* row_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)cam->height);
    for (int y = 0; y < cam->height; y++) row_of[y] = -1;
    for (int r = 0; r < nr; r++) row_of[rows ? rows[r] : r] = r;
    int64_t* cnt = (int64_t*)calloc((size_t)nr + 1, sizeof(int64_t));
    for (int64_t s = 0; s < n_splats; s++) {
        const or_splat* sp = &splats[s];
        if (!sp->valid && !(sp->ambiguous & 1)) continue;
        int y0 = brute_force ? 0 : sp->px_min[1], y1 = brute_force ? cam->height - 1 : sp->px_max[1];
        for (int y = y0; y <= y1; y++)
            if (row_of[y] >= 0) cnt[row_of[y] + 1]++;
    }
    for (int r = 0; r < nr; r++) cnt[r + 1] += cnt[r];
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt[nr] > 0 ? cnt[nr] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nr > 0 ? nr : 1));
    for (int r = 0; r < nr; r++) fill[r] = cnt[r];
    for (int64_t s = 0; s < n_splats; s++) {
        const or_splat* sp = &splats[s];
        if (!sp->valid && !(sp->ambiguous & 1)) continue;
        int y0 = brute_force ? 0 : sp->px_min[1], y1 = brute_force ? cam->height - 1 : sp->px_max[1];
        for (int y = y0; y <= y1; y++)
            if (row_of[y] >= 0) list[fill[row_of[y]]++] = s;
    }

#pragma omp parallel
    {
        size_t cap = 256;
        fragment* fr = (fragment*)malloc(sizeof(fragment) * cap);
        int64_t* ccnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncol + 1));
        int64_t* cfill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncol + 1));
        size_t clist_cap = 1024;
        int64_t* clist = (int64_t*)malloc(sizeof(int64_t) * clist_cap);
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < nr; r++) {
            int y = rows ? rows[r] : r;
            /* column buckets of this row's candidates */
            for (int c = 0; c <= ncol; c++) ccnt[c] = 0;
            for (int64_t q = cnt[r]; q < cnt[r + 1]; q++) {
                const or_splat* sp = &splats[list[q]];
                int c0 = brute_force ? 0 : sp->px_min[0] / CW;
                int c1 = brute_force ? ncol - 1 : sp->px_max[0] / CW;
                for (int c = c0; c <= c1; c++) ccnt[c + 1]++;
            }
            for (int c = 0; c < ncol; c++) ccnt[c + 1] += ccnt[c];
            if ((size_t)ccnt[ncol] > clist_cap) {
                clist_cap = (size_t)ccnt[ncol];
                clist = (int64_t*)realloc(clist, sizeof(int64_t) * clist_cap);
            }
            for (int c = 0; c < ncol; c++) cfill[c] = ccnt[c];
            for (int64_t q = cnt[r]; q < cnt[r + 1]; q++) {
                const or_splat* sp = &splats[list[q]];
                int c0 = brute_force ? 0 : sp->px_min[0] / CW;
                int c1 = brute_force ? ncol - 1 : sp->px_max[0] / CW;
                for (int c = c0; c <= c1; c++) clist[cfill[c]++] = list[q];
            }
            for (int x = 0; x < W; x++) {
                size_t nf = 0;
                int col = x / CW;
                for (int64_t q = ccnt[col]; q < ccnt[col + 1]; q++) {
                    const or_splat* sp = &splats[clist[q]];
                    if (!brute_force && (x < sp->px_min[0] || x > sp->px_max[0])) continue;
                    double power;
                    double al = splat_alpha(sp, o, x, y, &power);
                    int near_thr = (sp->valid || (sp->ambiguous & 1)) &&
                                   fabs(al - o->alpha_min) <= o->eps_alpha * o->alpha_min;
                    int blend = sp->valid && power <= 0.0 && al >= o->alpha_min;
                    if (!blend && !near_thr && !((sp->ambiguous & 1) && al >= o->alpha_min)) continue;
                    if (nf == cap) { cap *= 2; fr = (fragment*)realloc(fr, sizeof(fragment) * cap); }
                    fr[nf].z = sp->depth; fr[nf].inst = sp->instance; fr[nf].g = sp->gaussian;
                    fr[nf].idx = clist[q]; fr[nf].alpha = al;
                    fr[nf].ghost = !blend;
                    fr[nf].amb = near_thr || (sp->ambiguous & 1);
                    nf++;
                }
                double T = 1.0, C[3] = {0.0, 0.0, 0.0};
                int amb = blend_pixel(fr, nf, splats, o, C, &T, n_contrib);
                int64_t p = (int64_t)r * W + x;
                for (int ch = 0; ch < 3; ch++) image[3 * p + ch] = C[ch] + T * o->bg[ch];
                if (T_final) T_final[p] = T;
                if (amb_px) amb_px[p] = (uint8_t)amb;
            }
        }
        free(fr); free(ccnt); free(cfill); free(clist);
    }
    free(row_of); free(cnt); free(list); free(fill);
}

/* Exact render of selected pixel rows of a large scene without materialising every splat:
 * each instanced Gaussian is projected (in parallel); only those whose footprint reaches one of
 * the rows are kept, then composited as in or_composite.  Returns the number of kept splats, or
 * -1 on allocation failure.  keep / keep_amb are nullable per-instanced culling decisions. */
int64_t or_render_rows(const or_asset* assets, const or_instance* inst, int n_inst,
                       const or_camera* cam, const or_opts* o, const uint8_t* keep,
                       const uint8_t* keep_amb, const int32_t* rows, int n_rows, double* image,
                       double* T_final, uint8_t* amb_px) {
    uint8_t* on_row = (uint8_t*)calloc((size_t)cam->height, 1);
    for (int r = 0; r < n_rows; r++) on_row[rows[r]] = 1;
    int64_t total = 0;
    for (int i = 0; i < n_inst; i++) total += assets[inst[i].asset_id].n;
    uint8_t* hit = (uint8_t*)calloc((size_t)(total > 0 ? total : 1), 1);
    if (!hit) { free(on_row); return -1; }
    for (int i = 0; i < n_inst; i++) {
        const or_asset* a = &assets[inst[i].asset_id];
        int64_t off = instance_offset(assets, inst, i);
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t g = 0; g < a->n; g++) {
            or_splat sp;
            project_one(a, &inst[i], cam, o, i, g, keep ? keep[off + g] : 1,
                        keep_amb ? keep_amb[off + g] : 0, &sp);
            if (!sp.valid && !(sp.ambiguous & 1)) continue;
            for (int y = sp.px_min[1]; y <= sp.px_max[1]; y++)
                if (on_row[y]) { hit[off + g] = 1; break; }
        }
    }
    int64_t n_hit = 0;
    for (int64_t k = 0; k < total; k++) n_hit += hit[k];
    or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (size_t)(n_hit > 0 ? n_hit : 1));
    if (!sp) { free(on_row); free(hit); return -1; }
    int64_t w = 0;
    for (int i = 0; i < n_inst; i++) {
        const or_asset* a = &assets[inst[i].asset_id];
        int64_t off = instance_offset(assets, inst, i);
        for (int64_t g = 0; g < a->n; g++)
            if (hit[off + g])
                project_one(a, &inst[i], cam, o, i, g, keep ? keep[off + g] : 1,
                            keep_amb ? keep_amb[off + g] : 0, &sp[w++]);
    }
    or_composite(sp, n_hit, cam, o, rows, n_rows, image, T_final, NULL, amb_px, 0);
    free(sp); free(hit); free(on_row);
    return n_hit;
}

/* Contributions alpha_k T_k of every blended fragment at one pixel, in blend order, plus the
 * final T.  Returns the number of blended fragments (at most cap). */
int or_pixel_weights(const or_splat* splats, int64_t n_splats, const or_camera* cam,
                     const or_opts* o, int x, int y, double* weights, int cap, double* T_out) {
    fragment* fr = (fragment*)malloc(sizeof(fragment) * (size_t)(n_splats > 0 ? n_splats : 1));
    size_t nf = 0;
    (void)cam;
    for (int64_t s = 0; s < n_splats; s++) {
        const or_splat* sp = &splats[s];
        if (!sp->valid) continue;
        double power;
        double al = splat_alpha(sp, o, x, y, &power);
        if (power > 0.0 || al < o->alpha_min) continue;
        fr[nf].z = sp->depth; fr[nf].inst = sp->instance; fr[nf].g = sp->gaussian;
        fr[nf].idx = s; fr[nf].alpha = al; fr[nf].amb = 0; fr[nf].ghost = 0;
        nf++;
    }
    qsort(fr, nf, sizeof(fragment), frag_cmp);
    double T = 1.0;
    int n = 0;
    for (size_t k = 0; k < nf; k++) {
        double nt = T * (1.0 - fr[k].alpha);
        if (nt < o->t_stop) break;
        if (n < cap) weights[n] = fr[k].alpha * T;
        n++;
        T = nt;
    }
    *T_out = T;
    free(fr);
    return n;
}

/* ------------------------------------------------------------------ MLP training (Sec. 3.2, 4.1) */
/* Batch loss of the class-balanced binary cross-entropy and (if grad != NULL) its gradient with
 * respect to the flat weights.  Sample k is Gaussian sg[k] seen from training view sv[k]; views
 * holds, per view, the camera centre in the asset frame and its normalised focal length f_view.
 * A sample of class c weighs B / (2 N_c), N_c = the batch count of class c (the class-frequency
 * weighting of Sec. 4.1, read as class balancing); the loss is the weighted mean over the batch. */
double or_train_loss_grad(const or_asset* a, const double* views, const uint8_t* labels,
                          int64_t n_gauss, const int32_t* sv, const int32_t* sg, int64_t B,
                          const double* w, double* grad) {
    const double *W1 = w, *b1 = W1 + 64 * 32, *W2 = b1 + 64, *b2 = W2 + 64 * 64,
                 *W3 = b2 + 64, *b3 = W3 + 64 * 64, *W4 = b3 + 64, *b4 = W4 + 64;
    int64_t n_pos = 0;
    for (int64_t k = 0; k < B; k++) n_pos += labels[(int64_t)sv[k] * n_gauss + sg[k]] != 0;
    double w_pos = 1.0, w_neg = 1.0;
    if (n_pos > 0 && n_pos < B) { w_pos = (double)B / (2.0 * n_pos); w_neg = (double)B / (2.0 * (B - n_pos)); }
    if (grad) memset(grad, 0, sizeof(double) * OR_MLP_NW);
    double loss = 0.0;
    for (int64_t k = 0; k < B; k++) {
        const double* vw = &views[4 * sv[k]];
        double f[32], h1[64], h2[64], h3[64], z;
        or_mlp_features(a, &a->means[3 * (int64_t)sg[k]], vw, vw[3], f);
        dense(W1, b1, f, 32, 64, 1, h1);
        dense(W2, b2, h1, 64, 64, 1, h2);
        dense(W3, b3, h2, 64, 64, 1, h3);
        dense(W4, b4, h3, 64, 1, 0, &z);
        const int y = labels[(int64_t)sv[k] * n_gauss + sg[k]] != 0;
        const double wy = y ? w_pos : w_neg;
        const double p = 1.0 / (1.0 + exp(-z));
        /* -[y log p + (1 - y) log(1 - p)], written stably */
        loss += wy * ((z > 0 ? z : 0.0) - (y ? z : 0.0) + log1p(exp(-fabs(z)))) / (double)B;
        if (!grad) continue;
        double *gW1 = grad, *gb1 = gW1 + 64 * 32, *gW2 = gb1 + 64, *gb2 = gW2 + 64 * 64,
               *gW3 = gb2 + 64, *gb3 = gW3 + 64 * 64, *gW4 = gb3 + 64, *gb4 = gW4 + 64;
        const double dz = wy * (p - y) / (double)B;
        double d3[64], d2[64], d1[64];
        gb4[0] += dz;
        for (int j = 0; j < 64; j++) {
            gW4[j] += dz * h3[j];
            d3[j] = h3[j] > 0.0 ? dz * W4[j] : 0.0;
        }
        for (int j = 0; j < 64; j++) {
            gb3[j] += d3[j];
            for (int i = 0; i < 64; i++) gW3[64 * j + i] += d3[j] * h2[i];
        }
        for (int i = 0; i < 64; i++) {
            double s = 0.0;
            for (int j = 0; j < 64; j++) s += d3[j] * W3[64 * j + i];
            d2[i] = h2[i] > 0.0 ? s : 0.0;
        }
        for (int j = 0; j < 64; j++) {
            gb2[j] += d2[j];
            for (int i = 0; i < 64; i++) gW2[64 * j + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < 64; i++) {
            double s = 0.0;
            for (int j = 0; j < 64; j++) s += d2[j] * W2[64 * j + i];
            d1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        for (int j = 0; j < 64; j++) {
            gb1[j] += d1[j];
            for (int i = 0; i < 32; i++) gW1[32 * j + i] += d1[j] * f[i];
        }
    }
    return loss;
}

/* One Adam step (bias-corrected moments; step is 0-based) on the batch gradient above. */
double or_train_step(const or_asset* a, const double* views, const uint8_t* labels, int64_t n_gauss,
                     const int32_t* sv, const int32_t* sg, int64_t B, double* w, double* m,
                     double* v, double lr, double beta1, double beta2, double eps, int step) {
    double* g = (double*)malloc(sizeof(double) * OR_MLP_NW);
    double loss = or_train_loss_grad(a, views, labels, n_gauss, sv, sg, B, w, g);
    const double bc1 = 1.0 - pow(beta1, step + 1), bc2 = 1.0 - pow(beta2, step + 1);
    for (int i = 0; i < OR_MLP_NW; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        w[i] -= lr * (m[i] / bc1) / (sqrt(v[i] / bc2) + eps);
    }
    free(g);
    return loss;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
