// Visibility-MLP training step in BF16 on the tcgen05 tensor cores (NVGS Sec. 3.2 and 4.1): the
// 32-64-64-64-1 forward pass, the class-balanced BCE and the backward pass of one block of 128
// (view, Gaussian) samples, with BF16 operands, FP32 accumulation in tensor memory, and FP32 master
// weights (the partial gradients feed the same reduction and Adam update as the FP32 step).
//
// Thread s owns sample s of the block (TMEM lane s).  Every GEMM is an M = 128 tcgen05.mma issued
// by thread 0:
//   forward   Z_l (s x 64) = A_{l-1} (s x K) W_l^T            A = activations, B = W_l (64 x K)
//   backward  dH_{l-1} (s x 64) = G_l (s x 64) W_l            B = W_l^T (the transposed tile)
//             gW_l (j x k) = G_l^T (j x s) H_{l-1} (s x k)     A = G_l^T padded to 128 rows,
//                                                              B = H_{l-1}^T with a row of ones, so
//                                                              that column 64 (32 for W1) of the
//                                                              accumulator is the bias gradient
// where G_l = dL/dZ_l.  Biases are added in FP32 in the forward epilogues; the 64 -> 1 output
// layer, the loss and dL/dz, and the gradient of w4 and b4 are FP32 on the CUDA cores.  Operand
// tiles are K-major without swizzle (8 x 16-byte core matrices, element (r, k) of a K-column tile
// at (r / 8) 16 K + (k / 8) 128 + (r % 8) 16 + (k % 8) 2 bytes); the transposed tiles are written
// element by element.  The hidden activations are rounded to BF16 where they feed a GEMM; the
// ReLU masks are taken from the FP32 pre-activations.
//
// Every mbarrier wait is bounded; on a timeout the block sets the error flag, waits (bounded) for
// its MMAs, frees its TMEM and returns (its partial gradient is then garbage and the step must be
// discarded: the call reports NVGS_ERR_TIMEOUT).
#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace nvgs {

namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kTmemCols = 256;
constexpr uint32_t kColG = 0;      // weight-gradient accumulator (up to 80 columns)
constexpr uint32_t kColZ = 128;    // forward / activation-gradient accumulator (64 columns)
// shared memory (bytes)
constexpr int kOffW1 = 0;          // B: W1 (64 x 32)
constexpr int kOffW2 = 4096;       // B: W2 (64 x 64)
constexpr int kOffW3 = 12288;      // B: W3
constexpr int kOffW2T = 20480;     // B: W2^T (64 x 64)
constexpr int kOffW3T = 28672;     // B: W3^T
constexpr int kOffF = 36864;       // A: features (128 x 32)
constexpr int kOffFT = 45056;      // B: features^T + ones row (48 x 128)
constexpr int kOffH1 = 57344;      // A: H1 (128 x 64)
constexpr int kOffH2 = 73728;      // A: H2
constexpr int kOffH1T = 90112;     // B: H1^T + ones row (80 x 128)
constexpr int kOffH2T = 110592;    // B: H2^T + ones row
constexpr int kOffG = 131072;      // A: G (128 x 64)
constexpr int kOffGT = 147456;     // A: G^T padded (128 x 128, rows >= 64 zero)
constexpr int kOffVec = 180224;    // FP32 b1 b2 b3 w4 (64 each), b4
constexpr int kOffRed = kOffVec + 1040;   // FP32 [4 warps][66]: gw4, gb4, loss partials
constexpr int kOffMisc = kOffRed + 4 * 66 * 4;
constexpr int kSmemBytes = kOffMisc + 64;
constexpr uint32_t kLbo = 128;

// kind::f16 instruction descriptor, D = F32, A = B = BF16, K-major, M = 128.
constexpr uint32_t idesc(uint32_t n) { return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24); }

__device__ __forceinline__ uint16_t bf16(float x) {
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Byte offset of element (r, k) in a K-major core-matrix tile with K columns.
__device__ __forceinline__ uint32_t tile_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * 16 * K + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void put_bf16(uint8_t* tile, int r, int k, int K, float x) {
    *reinterpret_cast<uint16_t*>(tile + tile_off(r, k, K)) = bf16(x);
}

// This thread's row r of a K-major A tile from 8 consecutive BF16 pairs per 16-byte chunk.
__device__ __forceinline__ void put_row(uint8_t* tile, int r, int K, const uint32_t* p) {
#pragma unroll
    for (int c = 0; c < 8; c++)
        if (c * 8 < K)
            *reinterpret_cast<uint4*>(tile + (r >> 3) * 16 * K + c * 128 + (r & 7) * 16) =
                make_uint4(p[4 * c], p[4 * c + 1], p[4 * c + 2], p[4 * c + 3]);
}

__device__ __forceinline__ void load64(uint32_t taddr, float* v) {
    uint32_t r[32];
    tmem_ld32(taddr, r);
#pragma unroll
    for (int q = 0; q < 32; q++) v[q] = __uint_as_float(r[q]);
    tmem_ld32(taddr + 32, r);
#pragma unroll
    for (int q = 0; q < 32; q++) v[32 + q] = __uint_as_float(r[q]);
}

// Issue K / 16 MMA steps (both operands from shared memory) into d and commit.
__device__ __forceinline__ void gemm(uint32_t d, const uint8_t* a, int ka, const uint8_t* b, int kb,
                                     int k_steps, uint32_t n, uint64_t* mbar) {
    const uint64_t da = sdesc(a, kLbo, 16u * ka);
    const uint64_t db = sdesc(b, kLbo, 16u * kb);
    for (int k = 0; k < k_steps; k++) mma_f16(d, da + 16u * k, db + 16u * k, idesc(n), k > 0);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_train_fwd_bwd_tc(
    const float* __restrict__ w, const AssetDev* __restrict__ asset, const float4* __restrict__ views,
    const uint8_t* __restrict__ labels, const int32_t* __restrict__ sv, const int32_t* __restrict__ sg,
    uint32_t B, uint32_t n_gauss, const uint32_t* __restrict__ n_pos, float* __restrict__ partial,
    float* __restrict__ loss_sum, uint32_t* __restrict__ err_flag) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
    float* vec = reinterpret_cast<float*>(sm + kOffVec);
    float* sb1 = vec;
    float* sb2 = vec + 64;
    float* sb3 = vec + 128;
    float* sw4 = vec + 192;
    float* red = reinterpret_cast<float*>(sm + kOffRed);
    const float* W1 = w;
    const float* b1 = W1 + 64 * 32;
    const float* W2 = b1 + 64;
    const float* b2 = W2 + 64 * 64;
    const float* W3 = b2 + 64;
    const float* b3 = W3 + 64 * 64;
    const float* W4 = b3 + 64;
    const float* b4 = W4 + 64;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"((uint32_t)kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // ---- weights from the FP32 master copy: W_l as B tiles, W2^T and W3^T as B tiles
    for (int e = tid; e < 64 * 32; e += kThreads) put_bf16(sm + kOffW1, e >> 5, e & 31, 32, W1[e]);
    for (int e = tid; e < 64 * 64; e += kThreads) {
        const int j = e >> 6, k = e & 63;
        const float a = W2[e], c = W3[e];
        put_bf16(sm + kOffW2, j, k, 64, a);
        put_bf16(sm + kOffW3, j, k, 64, c);
        put_bf16(sm + kOffW2T, k, j, 64, a);   // W2^T[k][j] = W2[j][k]
        put_bf16(sm + kOffW3T, k, j, 64, c);
    }
    if (tid < 64) { sb1[tid] = b1[tid]; sb2[tid] = b2[tid]; sb3[tid] = b3[tid]; sw4[tid] = W4[tid]; }
    if (tid == 0) vec[256] = b4[0];
    // ---- the constant parts: ones rows of the transposed B tiles, zero rows of G^T
    for (int e = tid; e < 16 * 128; e += kThreads) {
        const int r = e >> 7, s = e & 127;
        const float one = r == 0 ? 1.0f : 0.0f;
        put_bf16(sm + kOffFT, 32 + r, s, 128, one);
        put_bf16(sm + kOffH1T, 64 + r, s, 128, one);
        put_bf16(sm + kOffH2T, 64 + r, s, 128, one);
    }
    // rows 64..127 of G^T (row groups 8..15, 2048 bytes each): 16 KB of zeros
    static_assert(kOffGT + 16 * 2048 <= kOffVec, "G^T tile");
    for (int e = tid; e < 8 * 2048 / 16; e += kThreads)
        reinterpret_cast<uint4*>(sm + kOffGT + 8 * 2048)[e] = make_uint4(0u, 0u, 0u, 0u);

    // ---- features of this thread's sample
    const uint32_t s0 = blockIdx.x * kThreads;
    const uint32_t k_s = s0 + tid;
    const bool valid = k_s < B;
    bool y = false;
    {
        float f[32];
        if (valid) {
            const uint32_t v = (uint32_t)sv[k_s], g = (uint32_t)sg[k_s];
            const float4 vw = views[v];
            FrameInst fi;
            fi.cam_local[0] = vw.x; fi.cam_local[1] = vw.y; fi.cam_local[2] = vw.z;
            fi.dist_scale = vw.w;
            mlp_features(*asset, fi, __ldg(&asset->mean_op[g]), f);
            y = labels[(size_t)v * n_gauss + g] != 0;
        } else {
#pragma unroll
            for (int q = 0; q < 32; q++) f[q] = 0.0f;
        }
        uint32_t p[16];
#pragma unroll
        for (int q = 0; q < 16; q++) p[q] = bf16x2(f[2 * q], f[2 * q + 1]);
        put_row(sm + kOffF, tid, 32, p);
#pragma unroll
        for (int q = 0; q < 16; q++) {
            *reinterpret_cast<uint16_t*>(sm + kOffFT + tile_off(2 * q, tid, 128)) = (uint16_t)(p[q] & 0xffffu);
            *reinterpret_cast<uint16_t*>(sm + kOffFT + tile_off(2 * q + 1, tid, 128)) = (uint16_t)(p[q] >> 16);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    // one MMA group: issue (thread 0), commit, wait; false if the wait gave up anywhere
    auto run = [&](auto&& issue) -> bool {
        if (tid == 0) {
            tc_fence_after();
            issue();
            mma_commit(mbar);
        }
        const bool done = mbar_wait(mbar, phase);
        phase ^= 1u;
        tc_fence_after();
        return !__syncthreads_or(!done);
    };
    auto sync_operands = [&]() {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };

    float z[64];
    uint32_t m1[2] = {0u, 0u}, m2[2] = {0u, 0u}, m3[2] = {0u, 0u};
    // ---- forward: Z1 = F W1^T (+ b1), H1 = ReLU
    ok = run([&] { gemm(tmem + kColZ, sm + kOffF, 32, sm + kOffW1, 32, 2, 64, mbar); });
    if (ok) {
        load64(tmem + kColZ + lane_off, z);
        uint32_t p[32];
#pragma unroll
        for (int q = 0; q < 64; q++) {
            z[q] += sb1[q];
            if (z[q] > 0.0f) m1[q >> 5] |= 1u << (q & 31);
            z[q] = fmaxf(z[q], 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 32; q++) p[q] = bf16x2(z[2 * q], z[2 * q + 1]);
        put_row(sm + kOffH1, tid, 64, p);
#pragma unroll
        for (int q = 0; q < 32; q++) {
            *reinterpret_cast<uint16_t*>(sm + kOffH1T + tile_off(2 * q, tid, 128)) = (uint16_t)(p[q] & 0xffffu);
            *reinterpret_cast<uint16_t*>(sm + kOffH1T + tile_off(2 * q + 1, tid, 128)) = (uint16_t)(p[q] >> 16);
        }
        tc_fence_before();
        sync_operands();
        ok = run([&] { gemm(tmem + kColZ, sm + kOffH1, 64, sm + kOffW2, 64, 4, 64, mbar); });
    }
    // ---- Z2, H2
    if (ok) {
        load64(tmem + kColZ + lane_off, z);
        uint32_t p[32];
#pragma unroll
        for (int q = 0; q < 64; q++) {
            z[q] += sb2[q];
            if (z[q] > 0.0f) m2[q >> 5] |= 1u << (q & 31);
            z[q] = fmaxf(z[q], 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 32; q++) p[q] = bf16x2(z[2 * q], z[2 * q + 1]);
        put_row(sm + kOffH2, tid, 64, p);
#pragma unroll
        for (int q = 0; q < 32; q++) {
            *reinterpret_cast<uint16_t*>(sm + kOffH2T + tile_off(2 * q, tid, 128)) = (uint16_t)(p[q] & 0xffffu);
            *reinterpret_cast<uint16_t*>(sm + kOffH2T + tile_off(2 * q + 1, tid, 128)) = (uint16_t)(p[q] >> 16);
        }
        tc_fence_before();
        sync_operands();
        ok = run([&] { gemm(tmem + kColZ, sm + kOffH2, 64, sm + kOffW3, 64, 4, 64, mbar); });
    }
    // ---- Z3, H3 (FP32, as the inference's output layer takes it), logit, loss, dL/dz, G3 = dz w4 [Z3 > 0]
    float dz = 0.0f, loss = 0.0f;
    if (ok) {
        load64(tmem + kColZ + lane_off, z);
        float lg = vec[256];
#pragma unroll
        for (int q = 0; q < 64; q++) {
            z[q] += sb3[q];
            if (z[q] > 0.0f) m3[q >> 5] |= 1u << (q & 31);
            z[q] = fmaxf(z[q], 0.0f);
            lg = fmaf(sw4[q], z[q], lg);
        }
        const uint32_t np = *n_pos;
        const float wpos = (np > 0 && np < B) ? (float)B / (2.0f * (float)np) : 1.0f;
        const float wneg = (np > 0 && np < B) ? (float)B / (2.0f * (float)(B - np)) : 1.0f;
        if (valid) {
            const float wy = y ? wpos : wneg;
            // BCE with logits: max(z, 0) - z y + log(1 + e^-|z|)
            loss = wy * (fmaxf(lg, 0.0f) - (y ? lg : 0.0f) + log1pf(expf(-fabsf(lg))));
            const float pr = 1.0f / (1.0f + expf(-lg));
            dz = wy * (pr - (y ? 1.0f : 0.0f)) / (float)B;
        }
        // gW4, gb4 and the loss: sums over the block's samples (warp shuffles, then 4 warp partials)
#pragma unroll
        for (int q = 0; q < 64; q++) {
            float t = dz * z[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[warp * 66 + q] = t;
        }
        float t0 = dz, t1 = loss;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        }
        if (lane == 0) { red[warp * 66 + 64] = t0; red[warp * 66 + 65] = t1; }
        // G3 (row and transposed tiles)
        uint32_t p[32];
#pragma unroll
        for (int q = 0; q < 32; q++) {
            const float g0 = ((m3[(2 * q) >> 5] >> ((2 * q) & 31)) & 1u) ? dz * sw4[2 * q] : 0.0f;
            const float g1 = ((m3[(2 * q + 1) >> 5] >> ((2 * q + 1) & 31)) & 1u) ? dz * sw4[2 * q + 1] : 0.0f;
            p[q] = bf16x2(g0, g1);
        }
        put_row(sm + kOffG, tid, 64, p);
#pragma unroll
        for (int q = 0; q < 32; q++) {
            *reinterpret_cast<uint16_t*>(sm + kOffGT + tile_off(2 * q, tid, 128)) = (uint16_t)(p[q] & 0xffffu);
            *reinterpret_cast<uint16_t*>(sm + kOffGT + tile_off(2 * q + 1, tid, 128)) = (uint16_t)(p[q] >> 16);
        }
        tc_fence_before();
        sync_operands();
    }
    float* P = partial + (size_t)blockIdx.x * kMlpWeights;
    float* gW1 = P;
    float* gb1 = gW1 + 64 * 32;
    float* gW2 = gb1 + 64;
    float* gb2 = gW2 + 64 * 64;
    float* gW3 = gb2 + 64;
    float* gb3 = gW3 + 64 * 64;
    float* gW4 = gb3 + 64;
    float* gb4 = gW4 + 64;
    if (ok && tid < 64) {
        gW4[tid] = red[tid] + red[66 + tid] + red[132 + tid] + red[198 + tid];
        if (tid == 0) {
            gb4[0] = red[64] + red[66 + 64] + red[132 + 64] + red[198 + 64];
            atomicAdd(loss_sum, (red[65] + red[66 + 65] + red[132 + 65] + red[198 + 65]) / (float)B);
        }
    }
    // ---- layer 3 backward: gW3 | gb3 = G3^T [H2 | 1], dH2 = G3 W3
    if (ok)
        ok = run([&] {
            gemm(tmem + kColG, sm + kOffGT, 128, sm + kOffH2T, 128, 8, 80, mbar);
            gemm(tmem + kColZ, sm + kOffG, 64, sm + kOffW3T, 64, 4, 64, mbar);
        });
    if (ok) {
        if (warp < 2) {   // lanes 0..63 hold rows j of gW3 and, in column 64, gb3[j]
            float v[64];
            load64(tmem + kColG + lane_off, v);
            uint32_t r[2];
            tmem_ld2(tmem + kColG + 64 + lane_off, r);
            // scalar stores: a block's partial starts at blockIdx * 10497 floats (4-byte aligned)
#pragma unroll
            for (int q = 0; q < 64; q++) gW3[tid * 64 + q] = v[q];
            gb3[tid] = __uint_as_float(r[0]);
        }
        load64(tmem + kColZ + lane_off, z);   // dH2
        uint32_t p[32];
#pragma unroll
        for (int q = 0; q < 32; q++) {
            const float g0 = ((m2[(2 * q) >> 5] >> ((2 * q) & 31)) & 1u) ? z[2 * q] : 0.0f;
            const float g1 = ((m2[(2 * q + 1) >> 5] >> ((2 * q + 1) & 31)) & 1u) ? z[2 * q + 1] : 0.0f;
            p[q] = bf16x2(g0, g1);
        }
        put_row(sm + kOffG, tid, 64, p);
#pragma unroll
        for (int q = 0; q < 32; q++) {
            *reinterpret_cast<uint16_t*>(sm + kOffGT + tile_off(2 * q, tid, 128)) = (uint16_t)(p[q] & 0xffffu);
            *reinterpret_cast<uint16_t*>(sm + kOffGT + tile_off(2 * q + 1, tid, 128)) = (uint16_t)(p[q] >> 16);
        }
        tc_fence_before();
        sync_operands();
        // ---- layer 2 backward: gW2 | gb2 = G2^T [H1 | 1], dH1 = G2 W2
        ok = run([&] {
            gemm(tmem + kColG, sm + kOffGT, 128, sm + kOffH1T, 128, 8, 80, mbar);
            gemm(tmem + kColZ, sm + kOffG, 64, sm + kOffW2T, 64, 4, 64, mbar);
        });
    }
    if (ok) {
        if (warp < 2) {
            float v[64];
            load64(tmem + kColG + lane_off, v);
            uint32_t r[2];
            tmem_ld2(tmem + kColG + 64 + lane_off, r);
#pragma unroll
            for (int q = 0; q < 64; q++) gW2[tid * 64 + q] = v[q];
            gb2[tid] = __uint_as_float(r[0]);
        }
        load64(tmem + kColZ + lane_off, z);   // dH1
        uint32_t p[32];
#pragma unroll
        for (int q = 0; q < 32; q++) {
            const float g0 = ((m1[(2 * q) >> 5] >> ((2 * q) & 31)) & 1u) ? z[2 * q] : 0.0f;
            const float g1 = ((m1[(2 * q + 1) >> 5] >> ((2 * q + 1) & 31)) & 1u) ? z[2 * q + 1] : 0.0f;
            p[q] = bf16x2(g0, g1);
        }
#pragma unroll
        for (int q = 0; q < 32; q++) {
            *reinterpret_cast<uint16_t*>(sm + kOffGT + tile_off(2 * q, tid, 128)) = (uint16_t)(p[q] & 0xffffu);
            *reinterpret_cast<uint16_t*>(sm + kOffGT + tile_off(2 * q + 1, tid, 128)) = (uint16_t)(p[q] >> 16);
        }
        tc_fence_before();
        sync_operands();
        // ---- layer 1: gW1 | gb1 = G1^T [F | 1]
        ok = run([&] { gemm(tmem + kColG, sm + kOffGT, 128, sm + kOffFT, 128, 8, 48, mbar); });
    }
    if (ok && warp < 2) {
        float v[32];
        uint32_t r[32];
        tmem_ld32(tmem + kColG + lane_off, r);
#pragma unroll
        for (int q = 0; q < 32; q++) v[q] = __uint_as_float(r[q]);
        uint32_t b[2];
        tmem_ld2(tmem + kColG + 32 + lane_off, b);
#pragma unroll
        for (int q = 0; q < 32; q++) gW1[tid * 32 + q] = v[q];
        gb1[tid] = __uint_as_float(b[0]);
    }
    if (!ok) {
        if (tid == 0) atomicExch(err_flag, 1u);
        mbar_wait(mbar, phase ^ 1u);   // the group whose wait gave up may still run (bounded)
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"((uint32_t)kTmemCols) : "memory");
    }
}

size_t train_tc_smem_bytes() { return (size_t)kSmemBytes; }

cudaError_t launch_train_fwd_bwd_tc(const float* w, const AssetDev* asset, const float4* views,
                                    const uint8_t* labels, const int32_t* sv, const int32_t* sg, uint32_t B,
                                    uint32_t n_gauss, const uint32_t* n_pos, float* partial, float* loss_sum,
                                    uint32_t* err_flag, cudaStream_t s, LaunchLog* log) {
    static std::atomic<uint64_t> attr_done{0};
    {
        cudaError_t e = once_per_device(attr_done, [] {
            return cudaFuncSetAttribute(k_train_fwd_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        });
        if (e != cudaSuccess) return e;
    }
    const uint32_t nb = (B + kThreads - 1) / kThreads;
    NVGS_LAUNCH(log, s, "k_train_fwd_bwd_tc", k_train_fwd_bwd_tc<<<nb, kThreads, kSmemBytes, s>>>(w, asset, views, labels, sv, sg, B, n_gauss, n_pos, partial, loss_sum, err_flag));
    return cudaGetLastError();
}

}  // namespace nvgs
