// S2, FP32 variant: the visibility MLP (32 -> 64 -> 64 -> 64 -> 1, ReLU; NVGS Sec. 3.2) on CUDA
// cores, one thread per in-frustum Gaussian.  This is the "plain FP32 method" of the small
// single-asset workload; the BF16 tensor-core kernel (k_mlp_tc.cu) serves large scenes.
//
// Weights are read through the read-only cache: all lanes of a warp usually share an asset and
// read the same address (a broadcast).  Layer 2 is folded into layer 3 so that only two
// 64-wide activation vectors are live at once.
#include "mlp_common.cuh"

namespace nvgs {

__global__ void __launch_bounds__(128) k_mlp_fp32(const uint2* __restrict__ list, uint32_t n,
                                                  const uint32_t* __restrict__ n_dev,
                                                  const FrameInst* __restrict__ fis,
                                                  const AssetDev* __restrict__ assets,
                                                  const float* __restrict__ logits_override,
                                                  const int64_t* __restrict__ inst_offset,
                                                  float threshold, uint32_t* __restrict__ keep_bits,
                                                  float* __restrict__ logits_out) {
    if (n_dev) n = min(n, *n_dev);   // device-side count (n is then the capacity)
    if (blockIdx.x * blockDim.x >= n) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    if (i < n) {
        const uint2 e = list[i];
        const FrameInst& fi = fis[e.x];
        float logit;
        bool bypass = fi.gated;
        if (logits_override) {          // injected decisions replace every asset's MLP
            logit = logits_override[inst_offset[e.x] + e.y];
        } else if (fi.no_mlp) {
            logit = __int_as_float(0x7f800000);
            bypass = true;
        } else {
            const AssetDev& a = assets[fi.asset];
            float f[32];
            mlp_features(a, fi, __ldg(&a.mean_op[e.y]), f);
            const float* __restrict__ W1 = a.w_fp32;
            const float* __restrict__ b1 = W1 + 64 * 32;
            const float* __restrict__ W2 = b1 + 64;
            const float* __restrict__ b2 = W2 + 64 * 64;
            const float* __restrict__ W3 = b2 + 64;
            const float* __restrict__ b3 = W3 + 64 * 64;
            const float* __restrict__ W4 = b3 + 64;
            const float* __restrict__ b4 = W4 + 64;
            float h1[64];
#pragma unroll
            for (int j = 0; j < 64; j++) {
                float acc = __ldg(&b1[j]);
#pragma unroll
                for (int k = 0; k < 32; k++) acc = fmaf(__ldg(&W1[j * 32 + k]), f[k], acc);
                h1[j] = fmaxf(acc, 0.0f);
            }
            float h3[64];
#pragma unroll
            for (int m = 0; m < 64; m++) h3[m] = __ldg(&b3[m]);
#pragma unroll 4
            for (int j = 0; j < 64; j++) {
                float acc = __ldg(&b2[j]);
#pragma unroll
                for (int k = 0; k < 64; k++) acc = fmaf(__ldg(&W2[j * 64 + k]), h1[k], acc);
                const float h2 = fmaxf(acc, 0.0f);
#pragma unroll
                for (int m = 0; m < 64; m++) h3[m] = fmaf(__ldg(&W3[m * 64 + j]), h2, h3[m]);
            }
            logit = __ldg(&b4[0]);
#pragma unroll
            for (int m = 0; m < 64; m++) logit = fmaf(__ldg(&W4[m]), fmaxf(h3[m], 0.0f), logit);
        }
        keep = bypass || (logit > threshold);
        if (logits_out) logits_out[i] = logit;
    }
    const uint32_t w = __ballot_sync(0xffffffffu, keep);
    if ((threadIdx.x & 31) == 0 && (i & ~31u) < n) keep_bits[i >> 5] = w;
}

cudaError_t launch_mlp_fp32(const uint2* list, uint32_t n, const uint32_t* n_dev, const FrameInst* fi,
                            const AssetDev* assets, const float* logits_override,
                            const int64_t* inst_offset, float threshold, uint32_t* keep_bits,
                            float* logits_out, cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_mlp_fp32", k_mlp_fp32<<<(n + 127) / 128, 128, 0, s>>>(list, n, n_dev, fi, assets, logits_override, inst_offset, threshold, keep_bits, logits_out));
    return cudaGetLastError();
}

}  // namespace nvgs
