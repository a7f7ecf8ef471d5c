// Visibility-MLP training (NVGS Sec. 3.2 and 4.1): class-balanced binary cross-entropy on
// (Gaussian, view) samples labelled by the GPU labeller, Adam on FP32 master weights.
//
// One step = three kernels (the forward/backward kernel in FP32 here, or in BF16 on the tensor cores
// in k_train_tc.cu):
//   k_train_sample    draws B (view, gaussian) samples with a counter-based hash (SplitMix64's
//                     finaliser of seed, step, sample index) unless explicit samples are given,
//                     and counts the positive labels of the batch;
//   k_train_fwd_bwd   64 samples per block: features, the 32-64-64-64-1 forward pass, the
//                     weighted BCE and its backward pass, all through shared memory; each block
//                     writes its partial gradient (same flat layout as the weights) -- no atomics
//                     on gradients, so a step is deterministic;
//   k_train_adam      sums the partial gradients per weight and applies one Adam update.
// The loss weighting of Sec. 4.1 (each sample weighted by the frequency of its class in the
// batch) is read as class balancing: a sample of class c weighs B / (2 N_c).
#include "mlp_common.cuh"

namespace nvgs {

namespace {

constexpr int kS = 64;          // samples per block
constexpr int kT = 256;         // threads per block
constexpr int kP = 65;          // padded row stride (floats) of activations and transposed weights
// shared floats: W1T[32][65] W2T[64][65] W3T[64][65] b1 b2 b3 w4 b4(4) F[64][33] H1 H2 H3 [64][65] dz[64] y[64]
constexpr int kOffW1T = 0;
constexpr int kOffW2T = kOffW1T + 32 * kP;
constexpr int kOffW3T = kOffW2T + 64 * kP;
constexpr int kOffB1 = kOffW3T + 64 * kP;
constexpr int kOffB2 = kOffB1 + 64;
constexpr int kOffB3 = kOffB2 + 64;
constexpr int kOffW4 = kOffB3 + 64;
constexpr int kOffB4 = kOffW4 + 64;
constexpr int kOffF = kOffB4 + 4;
constexpr int kOffH1 = kOffF + kS * 33;
constexpr int kOffH2 = kOffH1 + kS * kP;
constexpr int kOffH3 = kOffH2 + kS * kP;
constexpr int kOffDz = kOffH3 + kS * kP;
constexpr int kOffRed = kOffDz + kS;
constexpr int kSmemFloats = kOffRed + 64;
constexpr int kSmemBytes = kSmemFloats * 4;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

}  // namespace

__global__ void __launch_bounds__(256) k_train_sample(uint32_t B, uint64_t seed, uint32_t step,
                                                      uint32_t n_views, uint32_t n_gauss,
                                                      const uint8_t* __restrict__ labels,
                                                      int32_t* __restrict__ sv, int32_t* __restrict__ sg,
                                                      int explicit_samples, uint32_t* __restrict__ n_pos) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    bool pos = false;
    if (k < B) {
        uint32_t v, g;
        if (explicit_samples) {
            v = (uint32_t)sv[k];
            g = (uint32_t)sg[k];
        } else {
            const uint64_t h = splitmix64(seed ^ splitmix64(((uint64_t)step << 32) | k));
            v = (uint32_t)(((h >> 32) * (uint64_t)n_views) >> 32);
            g = (uint32_t)(((h & 0xffffffffull) * (uint64_t)n_gauss) >> 32);
            sv[k] = (int32_t)v;
            sg[k] = (int32_t)g;
        }
        pos = labels[(size_t)v * n_gauss + g] != 0;
    }
    const uint32_t c = __popc(__ballot_sync(0xffffffffu, pos));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_pos, c);
}

// views: per training view (camera centre in the asset frame, dist_scale = f_t / f_view).
__global__ void __launch_bounds__(kT, 2) k_train_fwd_bwd(const float* __restrict__ w,
                                                         const AssetDev* __restrict__ asset,
                                                         const float4* __restrict__ views,
                                                         const uint8_t* __restrict__ labels,
                                                         const int32_t* __restrict__ sv,
                                                         const int32_t* __restrict__ sg, uint32_t B,
                                                         uint32_t n_gauss, const uint32_t* __restrict__ n_pos,
                                                         float* __restrict__ partial,
                                                         float* __restrict__ loss_sum) {
    extern __shared__ float sm[];
    const int t = threadIdx.x;
    const float* W1 = w;
    const float* b1 = W1 + 64 * 32;
    const float* W2 = b1 + 64;
    const float* b2 = W2 + 64 * 64;
    const float* W3 = b2 + 64;
    const float* b3 = W3 + 64 * 64;
    const float* W4 = b3 + 64;
    const float* b4 = W4 + 64;
    float* W1T = sm + kOffW1T;
    float* W2T = sm + kOffW2T;
    float* W3T = sm + kOffW3T;
    float* sb1 = sm + kOffB1;
    float* sb2 = sm + kOffB2;
    float* sb3 = sm + kOffB3;
    float* sw4 = sm + kOffW4;
    float* F = sm + kOffF;
    float* H1 = sm + kOffH1;
    float* H2 = sm + kOffH2;
    float* H3 = sm + kOffH3;
    float* dz = sm + kOffDz;
    float* red = sm + kOffRed;
    // ---- weights, transposed: WT[k][j] = W[j][k]
    for (int e = t; e < 64 * 32; e += kT) W1T[(e & 31) * kP + (e >> 5)] = W1[e];
    for (int e = t; e < 64 * 64; e += kT) {
        W2T[(e & 63) * kP + (e >> 6)] = W2[e];
        W3T[(e & 63) * kP + (e >> 6)] = W3[e];
    }
    if (t < 64) {
        sb1[t] = b1[t]; sb2[t] = b2[t]; sb3[t] = b3[t]; sw4[t] = W4[t];
    }
    const uint32_t s0 = blockIdx.x * kS;
    const uint32_t np = *n_pos;
    const float wpos = (np > 0 && np < B) ? (float)B / (2.0f * (float)np) : 1.0f;
    const float wneg = (np > 0 && np < B) ? (float)B / (2.0f * (float)(B - np)) : 1.0f;
    // ---- features (one thread per sample)
    if (t < kS) {
        float f[32];
        const uint32_t k = s0 + t;
        if (k < B) {
            const uint32_t v = (uint32_t)sv[k], g = (uint32_t)sg[k];
            const float4 vw = views[v];
            FrameInst fi;
            fi.cam_local[0] = vw.x; fi.cam_local[1] = vw.y; fi.cam_local[2] = vw.z;
            fi.dist_scale = vw.w;
            mlp_features(*asset, fi, __ldg(&asset->mean_op[g]), f);
        } else {
#pragma unroll
            for (int q = 0; q < 32; q++) f[q] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 32; q++) F[t * 33 + q] = f[q];
    }
    __syncthreads();
    // ---- forward: H1, H2, H3 (thread -> 16 (sample, unit) outputs, unit fastest in a warp)
#pragma unroll 4
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, s = o >> 6, j = o & 63;
        float acc = sb1[j];
#pragma unroll
        for (int k = 0; k < 32; k++) acc = fmaf(W1T[k * kP + j], F[s * 33 + k], acc);
        H1[s * kP + j] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, s = o >> 6, j = o & 63;
        float acc = sb2[j];
#pragma unroll 16
        for (int k = 0; k < 64; k++) acc = fmaf(W2T[k * kP + j], H1[s * kP + k], acc);
        H2[s * kP + j] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, s = o >> 6, j = o & 63;
        float acc = sb3[j];
#pragma unroll 16
        for (int k = 0; k < 64; k++) acc = fmaf(W3T[k * kP + j], H2[s * kP + k], acc);
        H3[s * kP + j] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
    // ---- output, loss and dL/dz (mean over the batch)
    if (t < kS) {
        const uint32_t k = s0 + t;
        float z = __ldg(b4);
        for (int j = 0; j < 64; j++) z = fmaf(sw4[j], H3[t * kP + j], z);
        float d = 0.0f, l = 0.0f;
        if (k < B) {
            const bool y = labels[(size_t)sg[k] + (size_t)sv[k] * n_gauss] != 0;
            const float wy = y ? wpos : wneg;
            // BCE with logits: max(z, 0) - z y + log(1 + e^-|z|)
            l = wy * (fmaxf(z, 0.0f) - (y ? z : 0.0f) + log1pf(expf(-fabsf(z))));
            const float p = 1.0f / (1.0f + expf(-z));
            d = wy * (p - (y ? 1.0f : 0.0f)) / (float)B;
        }
        dz[t] = d;
        red[t] = l;
    }
    __syncthreads();
    float* P = partial + (size_t)blockIdx.x * kMlpWeights;
    float* gW1 = P;
    float* gb1 = gW1 + 64 * 32;
    float* gW2 = gb1 + 64;
    float* gb2 = gW2 + 64 * 64;
    float* gW3 = gb2 + 64;
    float* gb3 = gW3 + 64 * 64;
    float* gW4 = gb3 + 64;
    float* gb4 = gW4 + 64;
    if (t < 64) {   // gW4[j] = sum_s dz_s H3[s][j]
        float a = 0.0f;
        for (int s = 0; s < kS; s++) a = fmaf(dz[s], H3[s * kP + t], a);
        gW4[t] = a;
    } else if (t == 64) {
        float a = 0.0f, l = 0.0f;
        for (int s = 0; s < kS; s++) { a += dz[s]; l += red[s]; }
        gb4[0] = a;
        atomicAdd(loss_sum, l / (float)B);
    }
    __syncthreads();
    // D3 = dz w4 * [H3 > 0]  (in place of H3)
    for (int o = t; o < kS * 64; o += kT) {
        const int s = o >> 6, j = o & 63;
        const float h = H3[s * kP + j];
        H3[s * kP + j] = h > 0.0f ? dz[s] * sw4[j] : 0.0f;
    }
    __syncthreads();
    // gW3[j][k] = sum_s D3[s][j] H2[s][k]; gb3[j] = sum_s D3[s][j]
#pragma unroll 2
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, j = o >> 6, k = o & 63;
        float a = 0.0f;
#pragma unroll 16
        for (int s = 0; s < kS; s++) a = fmaf(H3[s * kP + j], H2[s * kP + k], a);
        gW3[j * 64 + k] = a;
    }
    if (t < 64) {
        float a = 0.0f;
        for (int s = 0; s < kS; s++) a += H3[s * kP + t];
        gb3[t] = a;
    }
    __syncthreads();
    // D2[s][k] = (sum_j D3[s][j] W3[j][k]) [H2 > 0]   (W3[j][k] = W3T[k][j])
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, s = o >> 6, k = o & 63;
        float a = 0.0f;
#pragma unroll 16
        for (int j = 0; j < 64; j++) a = fmaf(H3[s * kP + j], W3T[k * kP + j], a);
        H2[s * kP + k] = H2[s * kP + k] > 0.0f ? a : 0.0f;   // own element only
    }
    __syncthreads();
    // gW2 = D2^T H1, gb2
#pragma unroll 2
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, j = o >> 6, k = o & 63;
        float a = 0.0f;
#pragma unroll 16
        for (int s = 0; s < kS; s++) a = fmaf(H2[s * kP + j], H1[s * kP + k], a);
        gW2[j * 64 + k] = a;
    }
    if (t < 64) {
        float a = 0.0f;
        for (int s = 0; s < kS; s++) a += H2[s * kP + t];
        gb2[t] = a;
    }
    __syncthreads();
    // D1[s][k] = (sum_j D2[s][j] W2[j][k]) [H1 > 0]
    for (int q = 0; q < 16; q++) {
        const int o = q * kT + t, s = o >> 6, k = o & 63;
        float a = 0.0f;
#pragma unroll 16
        for (int j = 0; j < 64; j++) a = fmaf(H2[s * kP + j], W2T[k * kP + j], a);
        H1[s * kP + k] = H1[s * kP + k] > 0.0f ? a : 0.0f;   // own element only
    }
    __syncthreads();
    // gW1[j][k] = sum_s D1[s][j] F[s][k]  (64 x 32), gb1
    for (int q = 0; q < 8; q++) {
        const int o = q * kT + t, j = o >> 5, k = o & 31;
        float a = 0.0f;
#pragma unroll 16
        for (int s = 0; s < kS; s++) a = fmaf(H1[s * kP + j], F[s * 33 + k], a);
        gW1[j * 32 + k] = a;
    }
    if (t < 64) {
        float a = 0.0f;
        for (int s = 0; s < kS; s++) a += H1[s * kP + t];
        gb1[t] = a;
    }
}

// Partial gradients are summed in two stages so that every weight's reduction is spread over
// many threads: k_train_reduce folds groups of kGroup blocks (coalesced across weights), then
// k_train_adam folds the groups and applies one Adam update (bias-corrected moments).
constexpr int kGroup = 16;

__global__ void __launch_bounds__(256) k_train_reduce(const float* __restrict__ partial, int n_blocks,
                                                      float* __restrict__ folded) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpWeights) return;
    const int b0 = blockIdx.y * kGroup, b1 = min(n_blocks, b0 + kGroup);
    float g = 0.0f;
    for (int b = b0; b < b1; b++) g += partial[(size_t)b * kMlpWeights + i];
    folded[(size_t)blockIdx.y * kMlpWeights + i] = g;
}

__global__ void __launch_bounds__(256) k_train_adam(const float* __restrict__ folded, int n_groups,
                                                    float* __restrict__ w, float* __restrict__ m,
                                                    float* __restrict__ v, float lr, float beta1,
                                                    float beta2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpWeights) return;
    float g = 0.0f;
    for (int b = 0; b < n_groups; b++) g += folded[(size_t)b * kMlpWeights + i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

size_t train_partial_bytes(uint32_t B) {
    const size_t nb = (B + kS - 1) / kS, ng = (nb + kGroup - 1) / kGroup;
    return (nb + ng) * kMlpWeights * 4;
}

cudaError_t launch_train_step(const AssetDev* asset_dev, uint32_t n_gauss, const float4* views,
                              uint32_t n_views, const uint8_t* labels, uint32_t B, uint64_t seed,
                              uint32_t step, int32_t* sv, int32_t* sg, int explicit_samples,
                              uint32_t* n_pos, float* loss_sum, float* partial, float* w, float* m,
                              float* v, float lr, float beta1, float beta2, float eps, int bf16,
                              uint32_t* err_flag, cudaStream_t s, LaunchLog* log) {
    static std::atomic<uint64_t> attr_done{0};
    {
        cudaError_t e = once_per_device(attr_done, [] {
            return cudaFuncSetAttribute(k_train_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        });
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(n_pos, 0, 4, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(loss_sum, 0, 4, s);
    if (e != cudaSuccess) return e;
    NVGS_LAUNCH(log, s, "k_train_sample", k_train_sample<<<(B + 255) / 256, 256, 0, s>>>(B, seed, step, n_views, n_gauss, labels, sv, sg, explicit_samples, n_pos));
    // partial gradients: one per block of 64 samples (FP32) or 128 samples (BF16 tensor cores)
    int nb;
    if (bf16) {
        nb = (int)((B + 127) / 128);
        e = launch_train_fwd_bwd_tc(w, asset_dev, views, labels, sv, sg, B, n_gauss, n_pos, partial, loss_sum,
                                    err_flag, s, log);
        if (e != cudaSuccess) return e;
    } else {
        nb = (int)((B + kS - 1) / kS);
        NVGS_LAUNCH(log, s, "k_train_fwd_bwd", k_train_fwd_bwd<<<nb, kT, kSmemBytes, s>>>(w, asset_dev, views, labels, sv, sg, B, n_gauss, n_pos, partial, loss_sum));
    }
    const double bc1 = 1.0 - pow((double)beta1, (double)step + 1.0);
    const double bc2 = 1.0 - pow((double)beta2, (double)step + 1.0);
    const int ng = (nb + kGroup - 1) / kGroup;
    float* folded = partial + (size_t)nb * kMlpWeights;
    const dim3 rgrid((kMlpWeights + 255) / 256, ng);
    NVGS_LAUNCH(log, s, "k_train_reduce", k_train_reduce<<<rgrid, 256, 0, s>>>(partial, nb, folded));
    NVGS_LAUNCH(log, s, "k_train_adam", k_train_adam<<<(kMlpWeights + 255) / 256, 256, 0, s>>>(folded, ng, w, m, v, lr, beta1, beta2, eps, (float)bc1, (float)bc2));
    return cudaGetLastError();
}

}  // namespace nvgs
