// MLP input encoding shared by the FP32 and tcgen05 visibility-MLP kernels (NVGS Sec. 3.2-3.3).
#pragma once

#include "nvgs_internal.cuh"

namespace nvgs {

// The 32 inputs of one in-frustum Gaussian, in the asset's local frame (Sec. 3.3: means are
// translated and scaled back, view direction rotated back, distance corrected by Eq. 2):
//   [0..2]   p = 2 (mu - box centre) / box extent, in [-1, 1]
//   [3..14]  sin(2^k pi p), k = 0..3, axis fastest
//   [15..26] cos(2^k pi p)
//   [27..29] unit direction from the camera to mu
//   [30]     min-max normalised log d_t, d_t = |mu - c_local| f_t / f_r (Eq. 2), clamped
//   [31]     0 (pads K to a multiple of 16 for the tensor cores)
// The base octave uses the hardware sin/cos (|arg| <= pi); the higher octaves follow from it by
// the double-angle identities.
// The asset constants the inputs need (loaded once per pass) and the per-row instance values.
struct MlpAsset {
    float bc0, bc1, bc2, bs0, bs1, bs2, log_dmin, inv_log_range;
};
__device__ __forceinline__ MlpAsset mlp_asset(const AssetDev& a) {
    return MlpAsset{a.bbox_c[0], a.bbox_c[1], a.bbox_c[2], a.bbox_scale[0], a.bbox_scale[1],
                    a.bbox_scale[2], a.log_dmin, a.inv_log_range};
}

__device__ __forceinline__ void mlp_features(const MlpAsset& a, float clx, float cly, float clz,
                                             float dist_scale, float4 m, float f[32]) {
    float p[3] = {(m.x - a.bc0) * a.bs0, (m.y - a.bc1) * a.bs1, (m.z - a.bc2) * a.bs2};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float s, c;
        __sincosf(3.14159265358979f * p[k], &s, &c);   // |arg| <= pi: absolute error ~4e-7
        f[k] = p[k];
#pragma unroll
        for (int o = 0; o < 4; o++) {
            f[3 + 3 * o + k] = s;
            f[15 + 3 * o + k] = c;
            float s2 = 2.0f * s * c;
            float c2 = fmaf(-2.0f * s, s, 1.0f);
            s = s2;
            c = c2;
        }
    }
    float dx = m.x - clx, dy = m.y - cly, dz = m.z - clz;
    float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrtf(d2);
    float dist = d2 * inv;
    f[27] = dx * inv;
    f[28] = dy * inv;
    f[29] = dz * inv;
    // the hardware log2 (about 1e-7 relative; the feature is rounded to BF16 or kept in FP32)
    float dn = fmaf(2.0f * (__logf(dist * dist_scale) - a.log_dmin), a.inv_log_range, -1.0f);
    f[30] = fminf(1.0f, fmaxf(-1.0f, dn));
    f[31] = 0.0f;
}

__device__ __forceinline__ void mlp_features(const AssetDev& a, const FrameInst& fi, float4 m,
                                             float f[32]) {
    mlp_features(mlp_asset(a), fi.cam_local[0], fi.cam_local[1], fi.cam_local[2], fi.dist_scale, m, f);
}

}  // namespace nvgs
