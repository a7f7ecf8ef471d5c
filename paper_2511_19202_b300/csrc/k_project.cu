// S4: EWA projection of the surviving instanced Gaussians to 2D conics plus SH colour
// (NVGS Sec. 3.3 hands the survivors to the original 3DGS tiled pipeline).
//
// One thread per survivor.  Per survivor it reads 16 B mean/opacity + 16 B log-scale + 16 B
// quaternion + 16..192 B of SH (all 16-byte vector loads) and writes one 64-byte record (the
// splat with its 16-byte tile rectangle, one aligned 64-byte access for the depth-ordered
// gathers of the binning and the compositing), a 4-byte tile count and the depth sort's key.
// The SH loads are issued together with the mean, scale and quaternion loads, before the
// covariance arithmetic, so that ~250 B per thread are in flight at once (126 registers, two
// CTAs of 256 threads per SM: measured 3 % faster than four CTAs that load the SH after the
// covariance).
//
// Conventions (3DGS):  Sigma = R(q) diag(e^{2 ls}) R(q)^T;  Sigma_cam = s^2 W Sigma W^T with
// W = R_cam R_inst;  J is the pinhole Jacobian at the mean with x/z, y/z clamped to the guard
// band;  Sigma_2D = J Sigma_cam J^T + dilation I.  The support is the exact ellipse where
// opacity * exp(power) >= alpha_min, i.e. d^T Sigma_2D^{-1} d <= 2 ln(opacity / alpha_min); its
// axis-aligned half-extents are sqrt(k Sigma_2D,xx) and sqrt(k Sigma_2D,yy), so a splat is
// binned to exactly the tiles whose pixel centres it can reach.
#include <algorithm>

#include "nvgs_internal.cuh"

namespace nvgs {

// kMV (multi-view batches): each survivor takes its view's camera, and the rect's w carries the
// view in its high 16 bits (tile rows stay below 2^16).
template <bool kMV>
__global__ void __launch_bounds__(256, 2) k_project(const uint2* __restrict__ surv, uint32_t n,
                                                 const uint32_t* __restrict__ n_dev,
                                                 const FrameInst* __restrict__ fis,
                                                 const AssetDev* __restrict__ assets, const CamParams* __restrict__ camp,
                                                 float4* __restrict__ rec,
                                                 uint32_t* __restrict__ counts,
                                                 uint32_t* __restrict__ dkey,
                                                 uint32_t* __restrict__ didx) {
    const CamParams cam0 = *camp;
    if (n_dev) n = min(n, *n_dev);   // device-side count (n is then the capacity)
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint2 e = surv[i];
        const FrameInst& fi = fis[e.x];
        const CamParams cam = kMV ? camp[fi.view] : cam0;
        const AssetDev& a = assets[fi.asset];
        const uint32_t g = e.y;
        const float4 m = __ldg(&a.mean_op[g]);
        const float4 ls = __ldg(&a.scale_quat[2 * (size_t)g]);
        const float4 qr = __ldg(&a.scale_quat[2 * (size_t)g + 1]);
        // the SH coefficients (16 bytes at a time: coefficient j / 3, channel j % 3 of float j),
        // fetched only for a splat that can reach the image: early on a cheap conservative bound
        // (below), else once its support box is known to meet the image
        const int n_floats = 3 * (a.sh_degree + 1) * (a.sh_degree + 1);
        const float4* __restrict__ shp = reinterpret_cast<const float4*>(a.sh + (size_t)g * a.sh_stride);
        float4 shv[12];

        const float3 pc = cam_point(fi, m.x, m.y, m.z);
        const float x = pc.x, y = pc.y, z = pc.z;
        const float iz = 1.0f / z;
        const float tx = fminf(cam.lim_x, fmaxf(-cam.lim_x, x * iz));
        const float ty = fminf(cam.lim_y, fmaxf(-cam.lim_y, y * iz));
        // a cheap bound on the support's pixel radius: the largest 3D scale through the Jacobian's
        // Frobenius norm at the clamped ray, the level 2 ln(1 / alpha_min) at full opacity, the
        // dilation; a splat certainly outside the image fetches no SH here
        bool sh_loaded = false;
        {
            const float smax = fi.s * expf(fmaxf(ls.x, fmaxf(ls.y, ls.z)));
            const float rad = 3.4f * (fmaxf(cam.fx, cam.fy) * iz * sqrtf(2.0f + tx * tx + ty * ty) * smax + 0.6f) + 2.0f;
            const float uc = fmaf(cam.fx, x * iz, cam.cx), vc = fmaf(cam.fy, y * iz, cam.cy);
            if (uc + rad >= -0.5f && uc - rad <= (float)cam.W && vc + rad >= -0.5f && vc - rad <= (float)cam.H) {
#pragma unroll
                for (int q = 0; q < 12; q++)
                    shv[q] = 4 * q < n_floats ? __ldg(&shp[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
                sh_loaded = true;
            }
        }
        // A = J W (2 x 3)
        const float jx = cam.fx * iz, jy = cam.fy * iz;
        float A0[3], A1[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            A0[k] = jx * fmaf(-tx, fi.W[6 + k], fi.W[k]);
            A1[k] = jy * fmaf(-ty, fi.W[6 + k], fi.W[3 + k]);
        }
        // R(q) with q normalised
        const float qn = rsqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
        const float qw = qr.x * qn, qx = qr.y * qn, qy = qr.z * qn, qz = qr.w * qn;
        const float Rq[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                             2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                             2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
        const float sc[3] = {fi.s * expf(ls.x), fi.s * expf(ls.y), fi.s * expf(ls.z)};
        // B = A R(q) diag(s e^ls);  Sigma_2D = B B^T + dilation I
        float B0[3], B1[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            B0[k] = (A0[0] * Rq[k] + A0[1] * Rq[3 + k] + A0[2] * Rq[6 + k]) * sc[k];
            B1[k] = (A1[0] * Rq[k] + A1[1] * Rq[3 + k] + A1[2] * Rq[6 + k]) * sc[k];
        }
        const float ca = fmaf(B0[0], B0[0], fmaf(B0[1], B0[1], B0[2] * B0[2])) + cam.dilation;
        const float cb = fmaf(B0[0], B1[0], fmaf(B0[1], B1[1], B0[2] * B1[2]));
        const float cc = fmaf(B1[0], B1[0], fmaf(B1[1], B1[1], B1[2] * B1[2])) + cam.dilation;
        float det = ca * cc - cb * cb;
        if (!(det > 1e-3f * ca * cc))   // near-degenerate: cancellation guard in FP64
            det = (float)((double)ca * (double)cc - (double)cb * (double)cb);

        const float op = 1.0f / (1.0f + expf(-m.w));
        const float kk = 2.0f * (logf(op) - logf(cam.alpha_min));
        int4 r = make_int4(1, 1, 0, 0);
        uint32_t cnt = 0;
        const float u = fmaf(cam.fx, x * iz, cam.cx);
        const float v = fmaf(cam.fy, y * iz, cam.cy);
        const float xe = sqrtf(kk * ca), ye = sqrtf(kk * cc);
        const float cA = cc / det, cB = -cb / det, cC = ca / det;   // conic, as stored
        const float kw = -0.5f * kk;                                  // stored ln(alpha_min / o)
        // non-finite geometry (degenerate input) is never binned; neither is a splat that radius
        // clipping (Sec. 4.4) drops by the determinant of its 2D covariance
        const bool clipped = cam.clip_det > 0.0f && det < cam.clip_det;
        if (kk > 0.0f && det > 0.0f && !clipped && isfinite(u) && isfinite(v) && isfinite(xe) &&
            isfinite(ye) && isfinite(det)) {
            float x0 = fmaxf(ceilf(u - xe - 0.5f), 0.0f);
            float x1 = fminf(floorf(u + xe - 0.5f), (float)(cam.W - 1));
            float y0 = fmaxf(ceilf(v - ye - 0.5f), 0.0f);
            float y1 = fminf(floorf(v + ye - 0.5f), (float)(cam.H - 1));
            if (x0 <= x1 && y0 <= y1) {
                // the colour's inputs (if the bound above did not already fetch them)
                if (!sh_loaded) {
#pragma unroll
                    for (int q = 0; q < 12; q++)
                        shv[q] = 4 * q < n_floats ? __ldg(&shp[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const int ts = cam.tile_size;
                r = make_int4((int)x0 / ts, (int)y0 / ts, (int)x1 / ts, (int)y1 / ts);
                cnt = (uint32_t)((r.z - r.x + 1) * (r.w - r.y + 1));
                if (cnt > 1) {
                    // row by row, from the values the record stores (as k_duplicate reads them)
                    const SplatEllipse el = splat_ellipse(u, v, cA, cB, cC, det, -2.0f * kw);
                    const float rts = 1.0f / (float)ts;
                    cnt = 0;
                    for (int ty = r.y; ty <= r.w; ty++) {
                        int t0, t1;
                        row_tile_span(el, ty, ts, rts, t0, t1);
                        t0 = max(t0, r.x);
                        t1 = min(t1, r.z);
                        if (t0 <= t1) cnt += (uint32_t)(t1 - t0 + 1);
                    }
                }
            }
        }
        // a splat without tiles (its support box outside the image -- the guard band keeps ~15-20 %
        // of the survivors there -- or every row pruned) gets an empty rectangle and nothing else:
        // no pair ever reads the rest of its record, so neither its colour nor its SH are fetched
        if (cnt == 0) r = make_int4(1, 1, 0, 0);
        if (kMV) r.w |= fi.view << 16;
        counts[i] = cnt;
        dkey[i] = __float_as_uint(z);   // z > z_near > 0: the bit pattern orders like the value
        didx[i] = i;
        float4* out = rec + kRecF4 * (size_t)i;
        reinterpret_cast<int4*>(out)[3] = r;
        if (cnt == 0) continue;
        out[0] = make_float4(u, v, cA, cB);
        // z: det Sigma_2D (the binning's row spans recover Sigma_2D from it and the conic);
        // w: ln(alpha_min / opacity), the exponent below which a fragment cannot reach alpha_min
        out[1] = make_float4(cC, op, det, kw);

        // colour at the local-frame direction from the camera to the mean
        float dx = m.x - fi.cam_local[0], dy = m.y - fi.cam_local[1], dz = m.z - fi.cam_local[2];
        const float dn = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        dx *= dn; dy *= dn; dz *= dn;
        float Y[16];
        sh_eval(a.sh_degree, dx, dy, dz, Y);
        float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int q = 0; q < 12; q++) {
            if (4 * q < n_floats) {
                const float4 t = shv[q];
                const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int j = 4 * q + e;
                    if (j < n_floats) col[j % 3] = fmaf(Y[j / 3], tv[e], col[j % 3]);
                }
            }
        }
        out[2] = make_float4(fmaxf(col[0], 0.0f), fmaxf(col[1], 0.0f), fmaxf(col[2], 0.0f), z);
    }
}

cudaError_t launch_project(const uint2* surv, uint32_t n, const uint32_t* n_dev, const FrameInst* fi,
                           const AssetDev* assets, const CamParams* cam_dev, float4* rec,
                           uint32_t* tile_counts, uint32_t* dkey, uint32_t* didx, int num_sms,
                           cudaStream_t s, LaunchLog* log, int multi_view) {
    if (n == 0) return cudaSuccess;
    // grid-stride over two waves of the two resident CTAs per SM
    const uint32_t grid = std::min<uint32_t>((n + 255) / 256, (uint32_t)num_sms * 2 * 2);
    if (multi_view)
        NVGS_LAUNCH(log, s, "k_project_views", k_project<true><<<grid, 256, 0, s>>>(surv, n, n_dev, fi, assets, cam_dev, rec, tile_counts, dkey, didx));
    else
        NVGS_LAUNCH(log, s, "k_project", k_project<false><<<grid, 256, 0, s>>>(surv, n, n_dev, fi, assets, cam_dev, rec, tile_counts, dkey, didx));
    return cudaGetLastError();
}

}  // namespace nvgs
