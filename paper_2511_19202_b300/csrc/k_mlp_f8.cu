// S2, FP8 tensor-core variant: the visibility MLP (32 -> 64 -> 64 -> 64 -> 1, ReLU; NVGS Sec. 3.2,
// queried as in Sec. 3.3) with E4M3 operands and FP32 accumulation on the tcgen05 tensor cores
// (kind::f8f6f4, K = 32 per instruction).
//
// Quantisation, one scale per tensor ("amax / 448", 448 being the largest finite E4M3):
//   inputs   q_x = E4M3(256 x)            (|x| <= 1, so 256 |x| <= 448; small features stay normal)
//   weights  q_W = E4M3(W / s_W),          s_W = max |W| / 448 per layer
//   hidden   q_h = E4M3(h / s_h),          s_h = (bound of |h| when |x| <= 1) / 448, the bound
//            propagated layer by layer as max_j (sum_k |W_jk| bound_in + |b_j|)
// so that the accumulator of layer l holds sum_k q_in q_W and the epilogue is one FMA per value:
//   q_h = E4M3_sat(max(0, acc alpha_l + beta_j))  with alpha_l = s_in s_W / s_h, beta = b / s_h,
// and the third layer's h3 = max(0, acc alpha_3 + b3) stays FP32 for the 64 -> 1 output on the
// CUDA cores.  Conversions saturate (cvt .satfinite), so a value past its bound clamps to 448.
//
// Structure as in the BF16 kernel (k_mlp_tc.cu): four single-tile CTAs per SM, each walking a
// contiguous range of 128-row steps with 128 TMEM columns --
//   [0, 64)   D   FP32 accumulator
//   [64, 80)  H   the hidden activations as E4M3 (4 per 32-bit column, the lower k in the low byte):
//                 the next layer's A operand
//   [80, 96)  IN  two 8-column buffers of E4M3 inputs (this step's and the next step's)
// -- so an MMA reads only its weight tile from shared memory; a step is 1 + 2 + 2 MMAs in three round
// trips; the next step's list rows are staged in shared memory by cp.async and its inputs built
// during the first layer's round trip; rows of several assets run one pass per asset; every wait
// is bounded.  Weight tiles are K-major without swizzle; an 8-bit core matrix is 8 rows x 16
// elements, element (row, k) of a K-column tile at (row / 8) * SBO + (k / 16) * 128 + (row % 8) * 16
// + (k % 16), SBO = 8 K bytes.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace nvgs {

namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kCtasPerSm = 4;
constexpr int kRows = 128;
constexpr int kTmemCols = 128;
constexpr uint32_t kColD = 0;
constexpr uint32_t kColH = 64;
constexpr uint32_t kColIn = 80;       // + 8 * buffer
// blob (packed on the host): E4M3 weight tiles, then FP32 vectors
constexpr int kOffW1 = 0;        // 64 x 32 E4M3 (SBO 256)
constexpr int kOffW2 = 2048;     // 64 x 64 E4M3 (SBO 512)
constexpr int kOffW3 = 6144;
constexpr int kOffVec = 10240;   // FP32: beta1[64] beta2[64] b3[64] w4[64] b4 alpha1 alpha2 alpha3
constexpr int kVecFloats = 260;
constexpr int kBlobBytes = kOffVec + kVecFloats * 4;   // 11280
constexpr int kOffRowM = 11264 + 1024;                 // next step's mean per row (16 B)
constexpr int kOffRowE = kOffRowM + kRows * 16;        // next step's list entry per row (8 B)
constexpr int kOffMisc = kOffRowE + kRows * 8;
constexpr int kSmemBytes = kOffMisc + 128;
constexpr uint32_t kSboK32 = 256;
constexpr uint32_t kSboK64 = 512;
constexpr uint32_t kLbo = 128;
constexpr float kInScale = 256.0f;

// kind::f8f6f4 descriptor: D = F32 (bit 4), A = B = E4M3 (format 0 at bits 7 and 10), K-major,
// N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// (lo, hi) -> two saturated E4M3 codes, lo in the low byte (the lower k); the _relu form clamps
// negative values to 0 in the same conversion.
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi) {
    uint16_t d;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return (uint32_t)d;
}
__device__ __forceinline__ uint32_t e4m3x2_relu(float lo, float hi) {
    uint16_t d;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return (uint32_t)d;
}
__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
    return e4m3x2(a, b) | (e4m3x2(c, d) << 16);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                   "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void mma_f8_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %3, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %4, p;\n\t}\n"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b), "r"(accumulate), "r"(kIdesc)
        : "memory");
}

// hidden epilogue: q_h = E4M3_sat(max(0, acc alpha + beta)) into H, in two 32-column halves (the
// ReLU inside the saturating conversion, beta read four at a time)
__device__ __forceinline__ void epilogue_hidden(uint32_t t_lane, float alpha, const float* beta) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
        uint32_t r[32];
        tmem_ld32(t_lane + kColD + 32 * half, r);
        uint32_t p[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 b = *reinterpret_cast<const float4*>(beta + 32 * half + 4 * q);
            // the same FMAs lane by lane as packed FP32x2 instructions
            const float2 v01 = __ffma2_rn(make_float2(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1])),
                                          make_float2(alpha, alpha), make_float2(b.x, b.y));
            const float2 v23 = __ffma2_rn(make_float2(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3])),
                                          make_float2(alpha, alpha), make_float2(b.z, b.w));
            p[q] = e4m3x2_relu(v01.x, v01.y) | (e4m3x2_relu(v23.x, v23.y) << 16);
        }
        tmem_st8(t_lane + kColH + 8 * half, p);
    }
}

__device__ __forceinline__ float epilogue_logit(uint32_t t_lane, float alpha, const float* b3, const float* w4,
                                                float b4) {
    // four partial sums, (0, 1) and (2, 3) packed: the same FMAs lane by lane as FP32x2 instructions
    float2 l01 = make_float2(b4, 0.0f), l23 = make_float2(0.0f, 0.0f);
    const float2 al = make_float2(alpha, alpha);
#pragma unroll
    for (int half = 0; half < 2; half++) {
        uint32_t r[32];
        tmem_ld32(t_lane + kColD + 32 * half, r);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 b = *reinterpret_cast<const float4*>(b3 + 32 * half + 4 * q);
            const float4 w = *reinterpret_cast<const float4*>(w4 + 32 * half + 4 * q);
            const float2 v01 = __ffma2_rn(make_float2(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1])), al,
                                          make_float2(b.x, b.y));
            const float2 v23 = __ffma2_rn(make_float2(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3])), al,
                                          make_float2(b.z, b.w));
            l01 = __ffma2_rn(make_float2(w.x, w.y), make_float2(fmaxf(v01.x, 0.0f), fmaxf(v01.y, 0.0f)), l01);
            l23 = __ffma2_rn(make_float2(w.z, w.w), make_float2(fmaxf(v23.x, 0.0f), fmaxf(v23.y, 0.0f)), l23);
        }
    }
    return (l01.x + l01.y) + (l23.x + l23.y);
}

__device__ __forceinline__ void prefetch_mean(float4* s_m, const float4* m) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s_m)), "l"(m) : "memory");
}
__device__ __forceinline__ void prefetch_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void prefetch_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// This thread's row of E4M3 inputs into its lane of an input buffer (zeros past the list); returns
// the row's instance gate.
__device__ __forceinline__ bool build_inputs(uint32_t t_in, bool valid, uint2 e, float4 m, int asset,
                                             const FrameInst* __restrict__ fis,
                                             const AssetDev* __restrict__ assets) {
    uint32_t p[8];
    bool gated = false;
    if (valid) {
        const FrameInst& fr = fis[e.x];
        gated = fr.gated != 0;
        const MlpAsset ma = mlp_asset(assets[asset]);
        float f[32];
        mlp_features(ma, fr.cam_local[0], fr.cam_local[1], fr.cam_local[2], fr.dist_scale, m, f);
#pragma unroll
        for (int q = 0; q < 8; q++)
            p[q] = e4m3x4(f[4 * q] * kInScale, f[4 * q + 1] * kInScale, f[4 * q + 2] * kInScale, f[4 * q + 3] * kInScale);
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++) p[q] = 0u;
    }
    tmem_st8(t_in, p);
    return gated;
}

__device__ __forceinline__ bool build_next(uint32_t t_in, bool valid, const uint2* s_e, const float4* s_m,
                                           const FrameInst* __restrict__ fis,
                                           const AssetDev* __restrict__ assets, int& asset) {
    prefetch_wait();
    uint2 e = make_uint2(0, 0);
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    asset = INT_MAX;
    if (valid) {
        e = *s_e;
        m = *s_m;
        asset = fis[e.x].asset;
    }
    return build_inputs(t_in, valid, e, m, asset, fis, assets);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
k_mlp_f8(const uint2* __restrict__ list, uint32_t n,
         const uint32_t* __restrict__ n_dev, const FrameInst* __restrict__ fis,
         const AssetDev* __restrict__ assets, float threshold, uint32_t* __restrict__ keep_bits,
         float* __restrict__ logits_out, uint32_t* __restrict__ err_flag) {
    extern __shared__ __align__(1024) uint8_t sm[];
    if (n_dev) n = min(n, *n_dev);
    const float* sVec = reinterpret_cast<const float*>(sm + kOffVec);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
    // reduction slots: per step parity [0,4) min and [4,8) max, then [16,20) pass min
    int* s_red = reinterpret_cast<int*>(sm + kOffMisc + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"((uint32_t)kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint64_t dW1 = sdesc(sm + kOffW1, kLbo, kSboK32);
    const uint64_t dW2 = sdesc(sm + kOffW2, kLbo, kSboK64);
    const uint64_t dW3 = sdesc(sm + kOffW3, kLbo, kSboK64);

    uint32_t phase = 0;
    int loaded = -1, known = -1;
    bool has_mlp = false;
    bool abort = false;
    uint32_t buf = 0;
    const uint32_t n_steps = (n + kRows - 1) / kRows;
    const uint32_t per_cta = (n_steps + gridDim.x - 1) / gridDim.x;
    const uint32_t s_begin = min(n_steps, blockIdx.x * per_cta);
    const uint32_t s_end = min(n_steps, s_begin + per_cta);
    uint2* s_e = reinterpret_cast<uint2*>(sm + kOffRowE) + tid;
    float4* s_m = reinterpret_cast<float4*>(sm + kOffRowM) + tid;
    int my_asset_next = INT_MAX;
    bool gated = false;
    if (s_begin < s_end) {
        const uint32_t i0 = s_begin * kRows + tid;
        uint2 e = make_uint2(0, 0);
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        int a0 = INT_MAX;
        if (i0 < n) {
            e = __ldg(&list[i0]);
            a0 = fis[e.x].asset;
            m = __ldg(&assets[a0].mean_op[e.y]);
        }
        gated = build_inputs(t_lane + kColIn, i0 < n, e, m, a0, fis, assets);
        my_asset_next = a0;
    }
    // this thread's entry of the step after the current one: entries are loaded two steps ahead,
    // means one step ahead (addressed through the entry's instance and asset)
    uint2 e_ahead = make_uint2(0u, 0u);
    if (s_begin + 1 < s_end && (s_begin + 1) * kRows + tid < n) e_ahead = __ldg(&list[(s_begin + 1) * kRows + tid]);

    for (uint32_t step = s_begin; step < s_end && !abort; step++) {
        const uint32_t i = step * kRows + tid;
        const bool valid = i < n;
        const uint32_t nstep = step + 1;
        const uint32_t i_next = nstep * kRows + tid;
        const bool has_next = nstep < s_end;
        const bool next_valid = has_next && i_next < n;
        if (next_valid) {
            *s_e = e_ahead;
            prefetch_mean(s_m, assets[fis[e_ahead.x].asset].mean_op + e_ahead.y);
        }
        prefetch_commit();
        {
            const uint32_t i_next2 = (nstep + 1) * kRows + tid;
            e_ahead = (nstep + 1 < s_end && i_next2 < n) ? __ldg(&list[i_next2]) : make_uint2(0u, 0u);
        }
        const int my_asset = my_asset_next;
        bool gated_next = false;
        {
            const int amin = __reduce_min_sync(0xffffffffu, my_asset);
            const int amax = __reduce_max_sync(0xffffffffu, valid ? my_asset : INT_MIN);
            if (lane == 0) { s_red[8 * buf + warp] = amin; s_red[8 * buf + 4 + warp] = amax; }
        }
        tmem_wait_st();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const int* sr = s_red + 8 * buf;
        const int step_min = min(min(sr[0], sr[1]), min(sr[2], sr[3]));
        const int step_max = max(max(sr[4], sr[5]), max(sr[6], sr[7]));
        bool pending = valid, keep = false, built_next = false;
        float logit = 0.0f;
        const uint32_t a_in = tmem + kColIn + 8u * buf;
        int cur = step_min;
        while (cur != INT_MAX) {
            const bool mine = pending && my_asset == cur;
            if (cur != known) { has_mlp = assets[cur].w_f8 != nullptr; known = cur; }
            if (!has_mlp) {   // asset without an MLP: rendered unculled
                if (mine) { keep = true; logit = __int_as_float(0x7f800000); }
            } else {
                if (cur != loaded) {   // every MMA of earlier passes has completed (waited on)
                    const uint4* src = reinterpret_cast<const uint4*>(assets[cur].w_f8);
                    uint4* dst = reinterpret_cast<uint4*>(sm);
                    for (int k = tid; k < kBlobBytes / 16; k += kThreads) dst[k] = __ldg(&src[k]);
                    fence_async_smem();
                    __syncthreads();
                    loaded = cur;
                }
                bool ok = true;
#pragma unroll 1
                for (int layer = 0; layer < 3; layer++) {
                    if (tid == 0) {
                        tc_fence_after();
                        if (layer == 0) {
                            mma_f8_ts(tmem + kColD, a_in, dW1, 0);
                        } else {
                            const uint64_t dW = layer == 1 ? dW2 : dW3;
#pragma unroll
                            for (int k = 0; k < 2; k++)   // K = 64 in two K = 32 steps
                                mma_f8_ts(tmem + kColD, tmem + kColH + 8u * k, dW + 16u * k, k > 0);
                        }
                        mma_commit(mbar);
                    }
                    if (layer == 0 && !built_next) {   // overlaps the first layer's round trip
                        if (has_next)
                            gated_next = build_next(t_lane + kColIn + 8u * (buf ^ 1u), next_valid, s_e, s_m, fis,
                                                    assets, my_asset_next);
                        built_next = true;
                    }
                    ok = mbar_wait(mbar, phase);
                    phase ^= 1u;
                    tc_fence_after();
                    if (layer < 2) {
                        if (ok) epilogue_hidden(t_lane, sVec[257 + layer], sVec + 64 * layer);
                        tmem_wait_st();
                    } else if (ok) {
                        const float lg = epilogue_logit(t_lane, sVec[259], sVec + 128, sVec + 192, sVec[256]);
                        if (mine) { logit = lg; keep = gated || (lg > threshold); }
                    }
                    tc_fence_before();
                    if (__syncthreads_or(!ok)) { abort = true; break; }
                }
                if (abort) break;
            }
            if (mine) pending = false;
            if (step_min == step_max) break;
            {
                const int cand = __reduce_min_sync(0xffffffffu, pending ? my_asset : INT_MAX);
                if (lane == 0) s_red[16 + warp] = cand;
            }
            __syncthreads();
            cur = min(min(s_red[16], s_red[17]), min(s_red[18], s_red[19]));
            __syncthreads();
        }
        if (abort) break;
        if (!built_next && has_next)
            gated_next = build_next(t_lane + kColIn + 8u * (buf ^ 1u), next_valid, s_e, s_m, fis, assets,
                                    my_asset_next);
        if (!has_next) my_asset_next = INT_MAX;
        const uint32_t row0 = step * kRows;
        const uint32_t w = __ballot_sync(0xffffffffu, keep);
        if (lane == 0 && row0 + warp * 32 < n) keep_bits[(row0 >> 5) + warp] = w;
        if (logits_out && valid) logits_out[i] = logit;
        gated = gated_next;
        buf ^= 1u;
    }
    if (abort) {
        if (tid == 0) atomicExch(err_flag, 1u);
        mbar_wait(mbar, phase ^ 1u);   // the layer whose wait gave up may still run (bounded)
    }
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"((uint32_t)kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------------ host side
size_t mlp_f8_weight_bytes() { return (size_t)kBlobBytes; }

// E4M3 code of x (round to nearest even, saturating at +-448): 1 sign, 4 exponent (bias 7) and 3
// mantissa bits, subnormals below 2^-6 with quantum 2^-9.
static uint8_t f32_to_e4m3(float xf) {
    const double x = xf;
    const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
    double a = std::fabs(x);
    if (!(a == a)) return 0x7F;   // NaN (never produced from finite weights)
    if (a >= 448.0) return sign | 0x7E;
    if (a < std::ldexp(1.0, -6)) {                       // subnormal: m x 2^-9, m = 0..7
        const double m = std::nearbyint(a / std::ldexp(1.0, -9));
        if (m >= 8.0) return sign | 0x08;                // rounds up to the smallest normal
        return sign | (uint8_t)m;
    }
    int e = (int)std::floor(std::log2(a));
    double q = std::ldexp(1.0, e - 3);
    double m = std::nearbyint(a / q);                     // 8 .. 16
    if (m >= 16.0) { e += 1; m = 8.0; }
    if (e > 8 || (e == 8 && m > 14.0)) return sign | 0x7E;
    return sign | (uint8_t)(((e + 7) << 3) | ((int)m - 8));
}

// Packs the weights with the per-tensor scales described at the top of this file.  scales_out
// (nullable): s_W1, s_W2, s_W3, s_h1, s_h2.
void mlp_f8_pack_weights(const float* w, uint8_t* out, float* scales_out) {
    memset(out, 0, kBlobBytes);
    const float* W1 = w;
    const float* b1 = W1 + 64 * 32;
    const float* W2 = b1 + 64;
    const float* b2 = W2 + 64 * 64;
    const float* W3 = b2 + 64;
    const float* b3 = W3 + 64 * 64;
    const float* W4 = b3 + 64;
    const float* b4 = W4 + 64;
    auto amax = [](const float* p, int n) {
        double m = 0.0;
        for (int k = 0; k < n; k++) m = std::max(m, (double)std::fabs(p[k]));
        return m > 0.0 ? m : 1.0;
    };
    // |h| bounds for |x| <= 1, layer by layer
    auto bound = [](const float* W, const float* b, int K, double in) {
        double m = 0.0;
        for (int j = 0; j < 64; j++) {
            double s = std::fabs((double)b[j]);
            for (int k = 0; k < K; k++) s += std::fabs((double)W[j * K + k]) * in;
            m = std::max(m, s);
        }
        return m > 0.0 ? m : 1.0;
    };
    const double sW1 = amax(W1, 64 * 32) / 448.0, sW2 = amax(W2, 64 * 64) / 448.0, sW3 = amax(W3, 64 * 64) / 448.0;
    const double B1 = bound(W1, b1, 32, 1.0), B2 = bound(W2, b2, 64, B1);
    const double sh1 = B1 / 448.0, sh2 = B2 / 448.0;
    auto put = [&](int off, int K, const float* Wm, double sW) {
        const int sbo = 8 * K;
        for (int nrow = 0; nrow < 64; nrow++)
            for (int k = 0; k < K; k++)
                out[off + (nrow / 8) * sbo + (k / 16) * 128 + (nrow % 8) * 16 + (k % 16)] =
                    f32_to_e4m3((float)(Wm[nrow * K + k] / sW));
    };
    put(kOffW1, 32, W1, sW1);
    put(kOffW2, 64, W2, sW2);
    put(kOffW3, 64, W3, sW3);
    float* vec = reinterpret_cast<float*>(out + kOffVec);
    for (int k = 0; k < 64; k++) {
        vec[k] = (float)(b1[k] / sh1);
        vec[64 + k] = (float)(b2[k] / sh2);
        vec[128 + k] = b3[k];
        vec[192 + k] = W4[k];
    }
    vec[256] = b4[0];
    vec[257] = (float)((1.0 / kInScale) * sW1 / sh1);
    vec[258] = (float)(sh1 * sW2 / sh2);
    vec[259] = (float)(sh2 * sW3);
    if (scales_out) {
        scales_out[0] = (float)sW1; scales_out[1] = (float)sW2; scales_out[2] = (float)sW3;
        scales_out[3] = (float)sh1; scales_out[4] = (float)sh2;
    }
}

cudaError_t launch_mlp_f8(const uint2* list, uint32_t n, const uint32_t* n_dev,
                          const FrameInst* fi, const AssetDev* assets, float threshold, uint32_t* keep_bits,
                          float* logits_out, uint32_t* err_flag, int num_sms, cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    static std::atomic<uint64_t> attr_done{0};
    {
        cudaError_t e = once_per_device(attr_done, [] {
            return cudaFuncSetAttribute(k_mlp_f8, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        });
        if (e != cudaSuccess) return e;
    }
    const uint32_t steps = (n + kRows - 1) / kRows;
    const uint32_t grid = std::min<uint32_t>(steps, (uint32_t)num_sms * kCtasPerSm);
    NVGS_LAUNCH(log, s, "k_mlp_f8", k_mlp_f8<<<grid, kThreads, kSmemBytes, s>>>(list, n, n_dev, fi, assets, threshold, keep_bits, logits_out, err_flag));
    return cudaGetLastError();
}

}  // namespace nvgs
