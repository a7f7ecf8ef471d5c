// N2: gradients of the render pass (compositing and EWA projection) with respect to the asset
// parameters -- means, log-scales, quaternions, opacity logits and SH coefficients -- for a loss
// L(image).  The same algebra as the original 3DGS backward, written for this pipeline:
//
//   k_blend_bwd    per tile and pixel, the tile's sorted Gaussians are walked back to front from
//                  the last fragment the forward blended (kept per pixel, with the final T); the
//                  forward quantities are recomputed on the fly (no per-pixel lists are stored)
//                  and T before each fragment is recovered as T / (1 - alpha).  Per fragment:
//                    dL/dc     = alpha T dL/dC
//                    dL/dalpha = T (c - C_behind) . dL/dC - T_final / (1 - alpha) bg . dL/dC
//                  (C_behind: colour of everything behind, per unit transmittance), then through
//                  alpha = opacity e^power (zero past the 0.99 clamp) to the 2D mean, the conic
//                  and the opacity.  The nine values are summed over each warp before one atomic
//                  add per value into the survivor's accumulator.
//   k_project_bwd  per survivor, chains those through the conic inversion, Sigma_2D = B B^T with
//                  B = J W R(q) diag(s e^ls), the quaternion (and its normalisation), the clamped
//                  pinhole Jacobian and mean projection, the camera transform, the sigmoid and the
//                  SH basis (coefficients and viewing direction), and adds them to the asset's
//                  gradient arrays (instances of one asset accumulate).
#include "nvgs_internal.cuh"

namespace nvgs {

namespace {
constexpr int kG = 9;   // per-survivor accumulators: u, v, conic A, B, C, opacity, r, g, b
}

template <int TS>
__global__ void __launch_bounds__(TS* TS) k_blend_bwd(const uint32_t* __restrict__ ranges,
                                                      const uint32_t* __restrict__ values,
                                                      const float4* __restrict__ rec, const CamParams* __restrict__ camp,
                                                      const float* __restrict__ final_T,
                                                      const int32_t* __restrict__ last_pair,
                                                      const float* __restrict__ dL_dimg,
                                                      float* __restrict__ gsurv) {
    const CamParams cam = *camp;
    constexpr int B = TS * TS;
    __shared__ float4 s_a[B];
    __shared__ float4 s_b[B];
    __shared__ float4 s_c[B];
    __shared__ uint32_t s_id[B];
    const int tile = blockIdx.x;
    const uint32_t start = ranges[2 * tile];
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int px = tx * TS + (threadIdx.x % TS), py = ty * TS + (threadIdx.x / TS);
    const bool inside = px < cam.W && py < cam.H;
    const size_t p = inside ? (size_t)py * cam.W + px : 0;
    const uint32_t last = inside ? (uint32_t)last_pair[p] : 0u;
    const float T_final = inside ? final_T[p] : 1.0f;
    float T = T_final;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) { g0 = dL_dimg[3 * p]; g1 = dL_dimg[3 * p + 1]; g2 = dL_dimg[3 * p + 2]; }
    const float bg_dot = cam.bg[0] * g0 + cam.bg[1] * g1 + cam.bg[2] * g2;
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;        // colour behind, per unit transmittance
    float la = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;  // the fragment just behind
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    // walk [start, max over the tile's pixels of last) back to front
    __shared__ uint32_t s_end;
    if (threadIdx.x == 0) s_end = start;
    __syncthreads();
    if (last > start) atomicMax(&s_end, last);
    __syncthreads();
    const uint32_t end = s_end;
    const int lane = threadIdx.x & 31;
    for (uint32_t hi = end; hi > start;) {
        const uint32_t lo = hi - start > (uint32_t)B ? hi - B : start;
        __syncthreads();   // the previous batch is fully consumed
        const uint32_t k = lo + threadIdx.x;
        if (k < hi) {
            const uint32_t id = values[k];
            s_id[threadIdx.x] = id;
            s_a[threadIdx.x] = __ldg(&rec[kRecF4 * (size_t)id]);
            s_b[threadIdx.x] = __ldg(&rec[kRecF4 * (size_t)id + 1]);
            s_c[threadIdx.x] = __ldg(&rec[kRecF4 * (size_t)id + 2]);
        }
        __syncthreads();
        for (int j = (int)(hi - lo) - 1; j >= 0; j--) {
            float gr[kG] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool any = false;
            if (lo + j < last) {
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                const float dx = fx - a.x, dy = fy - a.y;
                float4 sa, sb;
                stage_splat(a, b, sa, sb);   // the forward's exponent, bit for bit
                const float p2 = splat_exponent2(sa, sb, dx, dy);
                if (!(p2 > 0.0f || p2 < sb.z)) {   // the forward's pre-test
                    const float G = ex2_approx(p2);
                    const float og = __fmul_rn(b.y, G);
                    const float alpha = fminf(cam.alpha_max, og);
                    if (alpha >= cam.alpha_min) {
                        any = true;
                        const float4 c = s_c[j];
                        const float om = 1.0f - alpha;
                        T = T / om;                       // transmittance in front of it
                        const float w = alpha * T;
                        gr[6] = w * g0; gr[7] = w * g1; gr[8] = w * g2;
                        acc0 = la * lc0 + (1.0f - la) * acc0;
                        acc1 = la * lc1 + (1.0f - la) * acc1;
                        acc2 = la * lc2 + (1.0f - la) * acc2;
                        la = alpha; lc0 = c.x; lc1 = c.y; lc2 = c.z;
                        float dl_da = ((c.x - acc0) * g0 + (c.y - acc1) * g1 + (c.z - acc2) * g2) * T;
                        dl_da += -T_final / om * bg_dot;
                        if (og <= cam.alpha_max) {        // past the clamp alpha is constant
                            const float gpow = alpha * dl_da;
                            gr[5] = G * dl_da;
                            gr[0] = gpow * (a.z * dx + a.w * dy);
                            gr[1] = gpow * (b.x * dy + a.w * dx);
                            gr[2] = gpow * (-0.5f * dx * dx);
                            gr[3] = gpow * (-dx * dy);
                            gr[4] = gpow * (-0.5f * dy * dy);
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int q = 0; q < kG; q++) {
                    float v = gr[q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    gr[q] = v;
                }
                if (lane < kG) {
                    float v = 0.f;
#pragma unroll
                    for (int q = 0; q < kG; q++) v = q == lane ? gr[q] : v;
                    if (v != 0.0f) atomicAdd(&gsurv[(size_t)s_id[j] * kG + lane], v);
                }
            }
        }
        hi = lo;
    }
}

// Derivative of the real SH basis (the 3DGS signs) with respect to an unnormalised direction's
// components, contracted with w[k] = sum_ch dL/dcolour_ch sh_k,ch: returns dL/d(x, y, z).
__device__ __forceinline__ float3 sh_dir_grad(int deg, float x, float y, float z, const float* w) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (deg < 1) return make_float3(0.f, 0.f, 0.f);
    const float C1 = 0.4886025119029199f;
    gy += -C1 * w[1];
    gz += C1 * w[2];
    gx += -C1 * w[3];
    if (deg >= 2) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
        gx += a * y * w[4];            gy += a * x * w[4];
        gy += -a * z * w[5];           gz += -a * y * w[5];
        gx += -2.f * b * x * w[6];     gy += -2.f * b * y * w[6];     gz += 4.f * b * z * w[6];
        gx += -a * z * w[7];           gz += -a * x * w[7];
        gx += 2.f * c * x * w[8];      gy += -2.f * c * y * w[8];
    }
    if (deg >= 3) {
        const float a = 0.5900435899266435f, b = 2.890611442640554f, c = 0.4570457994644658f,
                    d = 0.3731763325901154f, e = 1.445305721320277f;
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += -6.f * a * x * y * w[9];                 gy += -a * (3.f * xx - 3.f * yy) * w[9];
        gx += b * y * z * w[10];  gy += b * x * z * w[10];  gz += b * x * y * w[10];
        gx += 2.f * c * x * y * w[11];  gy += -c * (4.f * zz - xx - 3.f * yy) * w[11];  gz += -8.f * c * y * z * w[11];
        gx += -6.f * d * x * z * w[12];  gy += -6.f * d * y * z * w[12];  gz += d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
        gx += -c * (4.f * zz - 3.f * xx - yy) * w[13];  gy += 2.f * c * x * y * w[13];  gz += -8.f * c * x * z * w[13];
        gx += 2.f * e * x * z * w[14];  gy += -2.f * e * y * z * w[14];  gz += e * (xx - yy) * w[14];
        gx += -a * (3.f * xx - 3.f * yy) * w[15];  gy += 6.f * a * x * y * w[15];
    }
    return make_float3(gx, gy, gz);
}

__global__ void __launch_bounds__(128) k_project_bwd(const uint2* __restrict__ surv, uint32_t n,
                                                     const FrameInst* __restrict__ fis,
                                                     const AssetDev* __restrict__ assets, const CamParams* __restrict__ camp,
                                                     const float* __restrict__ gsurv, int asset_id,
                                                     float* __restrict__ g_means, float* __restrict__ g_ls,
                                                     float* __restrict__ g_quat, float* __restrict__ g_op,
                                                     float* __restrict__ g_sh) {
    const CamParams cam = *camp;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 e = surv[i];
    const FrameInst& fi = fis[e.x];
    if (fi.asset != asset_id) return;
    const float* gs = gsurv + (size_t)i * kG;
    const float gu = gs[0], gv = gs[1], gA = gs[2], gB = gs[3], gC = gs[4], go = gs[5];
    const float gcol[3] = {gs[6], gs[7], gs[8]};
    const AssetDev& a = assets[fi.asset];
    const uint32_t g = e.y;
    const float4 m = a.mean_op[g];
    const float4 ls = a.scale_quat[2 * (size_t)g];
    const float4 qr = a.scale_quat[2 * (size_t)g + 1];
    // ---- forward recomputation (as in k_project)
    const float3 pc = cam_point(fi, m.x, m.y, m.z);
    const float x = pc.x, y = pc.y, z = pc.z;
    const float iz = 1.0f / z;
    const float txr = x * iz, tyr = y * iz;
    const float tx = fminf(cam.lim_x, fmaxf(-cam.lim_x, txr));
    const float ty = fminf(cam.lim_y, fmaxf(-cam.lim_y, tyr));
    const float jx = cam.fx * iz, jy = cam.fy * iz;
    float A0[3], A1[3], U0[3], U1[3];
    for (int k = 0; k < 3; k++) {
        U0[k] = fmaf(-tx, fi.W[6 + k], fi.W[k]);
        U1[k] = fmaf(-ty, fi.W[6 + k], fi.W[3 + k]);
        A0[k] = jx * U0[k];
        A1[k] = jy * U1[k];
    }
    const float qlen = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float qn = 1.0f / qlen;
    const float qw = qr.x * qn, qx = qr.y * qn, qy = qr.z * qn, qz = qr.w * qn;
    const float Rq[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                         2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                         2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    const float sc[3] = {fi.s * expf(ls.x), fi.s * expf(ls.y), fi.s * expf(ls.z)};
    float P0[3], P1[3], B0[3], B1[3];
    for (int k = 0; k < 3; k++) {
        P0[k] = A0[0] * Rq[k] + A0[1] * Rq[3 + k] + A0[2] * Rq[6 + k];
        P1[k] = A1[0] * Rq[k] + A1[1] * Rq[3 + k] + A1[2] * Rq[6 + k];
        B0[k] = P0[k] * sc[k];
        B1[k] = P1[k] * sc[k];
    }
    const float ca = B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2] + cam.dilation;
    const float cb = B0[0] * B1[0] + B0[1] * B1[1] + B0[2] * B1[2];
    const float cc = B1[0] * B1[0] + B1[1] * B1[1] + B1[2] * B1[2] + cam.dilation;
    const float det = ca * cc - cb * cb;
    // ---- conic = inverse(Sigma_2D): to (a, b, c)
    const float d2 = det * det;
    const float g_ca = (-cc * cc * gA + cb * cc * gB - cb * cb * gC) / d2;
    const float g_cb = (2.f * cb * cc * gA - (ca * cc + cb * cb) * gB + 2.f * ca * cb * gC) / d2;
    const float g_cc = (-cb * cb * gA + ca * cb * gB - ca * ca * gC) / d2;
    // ---- B rows -> P, scales, rotation, A
    float gA0[3] = {0.f, 0.f, 0.f}, gA1[3] = {0.f, 0.f, 0.f}, gR[9], g_ls3[3];
    for (int k = 0; k < 3; k++) {
        const float gB0 = 2.f * g_ca * B0[k] + g_cb * B1[k];
        const float gB1 = g_cb * B0[k] + 2.f * g_cc * B1[k];
        g_ls3[k] = (gB0 * P0[k] + gB1 * P1[k]) * sc[k];   // d sc / d ls = sc
        const float gP0 = gB0 * sc[k], gP1 = gB1 * sc[k];
        for (int j = 0; j < 3; j++) {
            gA0[j] += gP0 * Rq[3 * j + k];
            gA1[j] += gP1 * Rq[3 * j + k];
            gR[3 * j + k] = A0[j] * gP0 + A1[j] * gP1;
        }
    }
    // ---- quaternion (normalised), then its normalisation
    const float dw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    const float dxq = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - qw * gR[5] + qz * gR[6] +
                             qw * gR[7] - 2.f * qx * gR[8]);
    const float dyq = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + qw * gR[2] + qx * gR[3] + qz * gR[5] - qw * gR[6] +
                             qz * gR[7] - 2.f * qy * gR[8]);
    const float dzq = 2.f * (-2.f * qz * gR[0] - qw * gR[1] + qx * gR[2] + qw * gR[3] - 2.f * qz * gR[4] +
                             qy * gR[5] + qx * gR[6] + qy * gR[7]);
    const float qdot = qw * dw + qx * dxq + qy * dyq + qz * dzq;
    const float gq[4] = {(dw - qw * qdot) * qn, (dxq - qx * qdot) * qn, (dyq - qy * qdot) * qn,
                         (dzq - qz * qdot) * qn};
    // ---- A = J W: jx, jy, clamped tx, ty -> camera-space point
    float gx = 0.f, gy = 0.f, gz = 0.f;
    float g_jx = 0.f, g_jy = 0.f, g_tx = 0.f, g_ty = 0.f;
    for (int j = 0; j < 3; j++) {
        g_jx += gA0[j] * U0[j];
        g_jy += gA1[j] * U1[j];
        g_tx += -jx * gA0[j] * fi.W[6 + j];
        g_ty += -jy * gA1[j] * fi.W[6 + j];
    }
    gz += -(jx * iz) * g_jx - (jy * iz) * g_jy;
    if (txr > -cam.lim_x && txr < cam.lim_x) { gx += g_tx * iz; gz += -txr * iz * g_tx; }
    if (tyr > -cam.lim_y && tyr < cam.lim_y) { gy += g_ty * iz; gz += -tyr * iz * g_ty; }
    // mean projection u = fx x / z + cx, v = fy y / z + cy
    gx += jx * gu;
    gy += jy * gv;
    gz += -jx * txr * gu - jy * tyr * gv;
    // camera point = M mu + b
    float gmu[3];
    for (int k = 0; k < 3; k++) gmu[k] = fi.M[k] * gx + fi.M[3 + k] * gy + fi.M[6 + k] * gz;
    // ---- opacity
    const float op = 1.0f / (1.0f + expf(-m.w));
    const float g_logit = go * op * (1.0f - op);
    // ---- colour: SH coefficients and the viewing direction
    const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
    float ddx = m.x - fi.cam_local[0], ddy = m.y - fi.cam_local[1], ddz = m.z - fi.cam_local[2];
    const float dlen = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
    const float dx = ddx / dlen, dy = ddy / dlen, dz = ddz / dlen;
    float Y[16];
    sh_eval(a.sh_degree, dx, dy, dz, Y);
    const float* shp = a.sh + (size_t)g * a.sh_stride;
    float raw[3] = {0.5f, 0.5f, 0.5f};
    for (int k = 0; k < K; k++)
        for (int ch = 0; ch < 3; ch++) raw[ch] = fmaf(Y[k], shp[3 * k + ch], raw[ch]);
    float gc[3];
    for (int ch = 0; ch < 3; ch++) gc[ch] = raw[ch] > 0.0f ? gcol[ch] : 0.0f;   // max(0, .)
    const size_t KS = (size_t)K * 3;
    float wk[16];
    for (int k = 0; k < K; k++) {
        wk[k] = gc[0] * shp[3 * k] + gc[1] * shp[3 * k + 1] + gc[2] * shp[3 * k + 2];
        for (int ch = 0; ch < 3; ch++) atomicAdd(&g_sh[(size_t)g * KS + 3 * k + ch], Y[k] * gc[ch]);
    }
    const float3 gd = sh_dir_grad(a.sh_degree, dx, dy, dz, wk);
    const float gdot = gd.x * dx + gd.y * dy + gd.z * dz;
    gmu[0] += (gd.x - dx * gdot) / dlen;
    gmu[1] += (gd.y - dy * gdot) / dlen;
    gmu[2] += (gd.z - dz * gdot) / dlen;
    // ---- accumulate into the asset's gradients
    for (int k = 0; k < 3; k++) {
        atomicAdd(&g_means[3 * (size_t)g + k], gmu[k]);
        atomicAdd(&g_ls[3 * (size_t)g + k], g_ls3[k]);
    }
    for (int k = 0; k < 4; k++) atomicAdd(&g_quat[4 * (size_t)g + k], gq[k]);
    atomicAdd(&g_op[g], g_logit);
}

cudaError_t launch_render_backward(const uint32_t* ranges, const uint32_t* values, const float4* rec,
                                   const CamParams& cam, const CamParams* cam_dev, const float* final_T,
                                   const int32_t* last_pair,
                                   const float* dL_dimg, float* gsurv, const uint2* surv, uint32_t n_surv,
                                   const FrameInst* fi, const AssetDev* assets, int asset_id,
                                   float* g_means, float* g_ls, float* g_quat, float* g_op, float* g_sh,
                                   cudaStream_t s, LaunchLog* log) {
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    cudaError_t e = cudaMemsetAsync(gsurv, 0, (size_t)n_surv * kG * 4 + 4, s);
    if (e != cudaSuccess) return e;
    switch (cam.tile_size) {
        case 8: NVGS_LAUNCH(log, s, "k_blend_bwd<8>", k_blend_bwd<8><<<n_tiles, 64, 0, s>>>(ranges, values, rec, cam_dev, final_T, last_pair, dL_dimg, gsurv)); break;
        case 16: NVGS_LAUNCH(log, s, "k_blend_bwd<16>", k_blend_bwd<16><<<n_tiles, 256, 0, s>>>(ranges, values, rec, cam_dev, final_T, last_pair, dL_dimg, gsurv)); break;
        case 32: NVGS_LAUNCH(log, s, "k_blend_bwd<32>", k_blend_bwd<32><<<n_tiles, 1024, 0, s>>>(ranges, values, rec, cam_dev, final_T, last_pair, dL_dimg, gsurv)); break;
        default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || n_surv == 0) return e;
    NVGS_LAUNCH(log, s, "k_project_bwd", k_project_bwd<<<(n_surv + 127) / 128, 128, 0, s>>>(surv, n_surv, fi, assets, cam_dev, gsurv, asset_id, g_means, g_ls, g_quat, g_op, g_sh));
    return cudaGetLastError();
}

size_t render_backward_scratch_bytes(uint64_t n_surv) { return (size_t)(n_surv * kG * 4 + 256); }

// ------------------------------------------------------------------ asset update on the device
// Repacks structure-of-arrays parameters (device) into the asset's 16-byte layout in place.
__global__ void k_pack_asset(uint32_t n, int K, int stride, const float* __restrict__ means,
                             const float* __restrict__ log_scales, const float* __restrict__ quats,
                             const float* __restrict__ opacity_logits, const float* __restrict__ sh,
                             float4* __restrict__ mean_op, float4* __restrict__ scale_quat,
                             float* __restrict__ sh_out) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    mean_op[g] = make_float4(means[3 * (size_t)g], means[3 * (size_t)g + 1], means[3 * (size_t)g + 2],
                             opacity_logits[g]);
    scale_quat[2 * (size_t)g] = make_float4(log_scales[3 * (size_t)g], log_scales[3 * (size_t)g + 1],
                                            log_scales[3 * (size_t)g + 2], 0.0f);
    scale_quat[2 * (size_t)g + 1] = make_float4(quats[4 * (size_t)g], quats[4 * (size_t)g + 1],
                                                quats[4 * (size_t)g + 2], quats[4 * (size_t)g + 3]);
    for (int k = 0; k < 3 * K; k++) sh_out[(size_t)g * stride + k] = sh[(size_t)g * 3 * K + k];
}

cudaError_t launch_pack_asset(uint32_t n, int K, int stride, const float* means, const float* log_scales,
                              const float* quats, const float* opacity_logits, const float* sh,
                              float4* mean_op, float4* scale_quat, float* sh_out,
                              cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_pack_asset", k_pack_asset<<<(n + 255) / 256, 256, 0, s>>>(n, K, stride, means, log_scales, quats, opacity_logits, sh, mean_op, scale_quat, sh_out));
    return cudaGetLastError();
}

}  // namespace nvgs
