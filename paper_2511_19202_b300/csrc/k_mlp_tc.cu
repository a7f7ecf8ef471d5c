// S2, BF16 tensor-core variant: the per-asset visibility MLP (32 -> 64 -> 64 -> 64 -> 1, ReLU;
// NVGS Sec. 3.2, queried per in-frustum Gaussian as in Sec. 3.3) on the 5th-generation tensor
// cores (tcgen05), BF16 operands with FP32 accumulation in tensor memory (TMEM).
//
// One CTA = one warpgroup (128 threads) walking 256-Gaussian steps of the in-frustum list, as
// two 128-row tiles that share every MMA round trip (thread r owns rows r and 128 + r):
//   1. thread r builds the 32 inputs of row r (Eq. 2 distance, frequency encoding) and writes
//      them as BF16 into the A tile in shared memory;
//   2. lane 0 of warp h issues tcgen05.mma (M = 128, K = 16 per instruction) for tile h's layer
//      with the accumulator in TMEM and commits to the layer's mbarrier (two arrivals);
//   3. after the mbarrier completes, each warp reads its 32 TMEM lanes (tcgen05.ld 32x32b),
//      applies ReLU while converting to BF16 and writes the activations back to shared memory as
//      the next layer's A operand.
// All four layers run on the tensor cores, the output layer as an N = 16 MMA whose first two
// columns hold w4 split into BF16 high and low parts (the logit is their sum).  Biases cost no
// CUDA-core work: every layer ends with one more K = 16 MMA step of a constant A tile whose
// first two columns are 1 against a B tile holding the bias split into BF16 high and low parts,
// so the accumulator already contains W h + b (to about 2^-16 of b).  The epilogue of a hidden
// layer is thus tcgen05.ld -> cvt.rn.relu.bf16x2 -> st.shared.
// Three CTAs share an SM (128 TMEM columns and 65 KB of shared memory each), so the epilogues of
// some overlap the MMAs of others.  Within a CTA, each thread builds the inputs of its rows of the
// next step while the first layer's MMAs of the current step run (kept in registers as BF16
// pairs; a row of another asset is built in its own pass as usual).
//
// Operand layout (both operands K-major, no swizzle): 8 x 16-byte "core matrices"; element
// (row, k) of a tile with K columns sits at (row / 8) * SBO + (k / 8) * 128 + (row % 8) * 16
// + (k % 8) * 2 with SBO = 16 * K bytes.  The weights are packed on the host into exactly this
// byte layout (mlp_tc_pack_weights) and copied to shared memory with 16-byte loads.
//
// Every mbarrier wait is bounded; on a timeout the CTA sets the error flag, frees its TMEM and
// returns.
#include <climits>
#include <cstring>

#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace nvgs {

namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kCtasPerSm = 3;
constexpr int kHalves = 2;                 // each CTA carries two 128-row tiles through a layer
constexpr int kRows = 128 * kHalves;       // rows per CTA step
constexpr int kTmemCols = 64 * kHalves;
// shared-memory map (bytes); the weight blob [0, kBlobBytes) is packed on the host
constexpr int kOffW1 = 0;            // 64 x 32 BF16
constexpr int kOffW2 = 4096;         // 64 x 64 BF16
constexpr int kOffW3 = 12288;        // 64 x 64 BF16
constexpr int kOffW4 = 20480;        // 16 x 64 BF16: row 0 = w4 high part, row 1 = low part
constexpr int kOffB1 = 22528;        // bias tiles, N x 16 BF16: column 0 = high, 1 = low part
constexpr int kOffB2 = 24576;
constexpr int kOffB3 = 26624;
constexpr int kOffB4 = 28672;        // 16 x 16: row 0 = b4
constexpr int kBlobBytes = 29184;
constexpr int kOffOnes = kBlobBytes; // 128 x 16 BF16, columns 0 and 1 = 1 (written in the kernel)
// Per half, the input tile A (128 x 32) overlays the first half of the hidden tile H (128 x 64):
// layer 1's MMA has finished reading A before its epilogue writes H, and the next step's inputs
// are written only after the output layer's MMA has finished reading H.
constexpr int kOffH = kOffOnes + 4096;
constexpr int kHBytes = 16384;
constexpr int kOffMisc = kOffH + kHalves * kHBytes;
constexpr int kSmemBytes = kOffMisc + 64;
constexpr uint32_t kSboK16 = 256;    // 16 * 16
constexpr uint32_t kSboK32 = 512;    // 16 * 32
constexpr uint32_t kSboK64 = 1024;   // 16 * 64
constexpr uint32_t kLbo = 128;

// kind::f16 instruction descriptors: D = F32 (bit 4), A = B = BF16 (bits 7, 10), both K-major,
// N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t idesc(uint32_t n) { return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24); }
constexpr uint32_t kIdescN64 = idesc(64);
constexpr uint32_t kIdescN16 = idesc(16);

// (lo, hi) -> BF16x2 with ReLU, lo in the low half (the lower address).
__device__ __forceinline__ uint32_t bf16x2_relu(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void st_chunk(uint8_t* tile, uint32_t sbo, int row, int chunk, uint4 v) {
    *reinterpret_cast<uint4*>(tile + (row >> 3) * sbo + chunk * kLbo + (row & 7) * 16) = v;
}

// TMEM accumulator (this lane, 64 columns, bias included) -> ReLU -> BF16 row of the next A
// operand.
__device__ __forceinline__ void epilogue_hidden(uint32_t t_lane, uint8_t* sH, int row) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
        uint32_t r[32];
        tmem_ld32(t_lane + half * 32, r);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            uint32_t p[4];
#pragma unroll
            for (int q = 0; q < 4; q++)
                p[q] = bf16x2_relu(__uint_as_float(r[c * 8 + 2 * q]), __uint_as_float(r[c * 8 + 2 * q + 1]));
            st_chunk(sH, kSboK64, row, half * 4 + c, make_uint4(p[0], p[1], p[2], p[3]));
        }
    }
}

// Issue one layer for one 128-row tile: K / 16 steps of A x B plus the bias step.  Descriptors
// are precomputed; consecutive K = 16 slices of a K-major tile are 256 bytes (16 in the
// descriptor's address field) apart.
__device__ __forceinline__ void issue_layer(uint32_t d, uint64_t da, int k_steps, uint64_t dw,
                                            uint64_t dbias, uint64_t dones, uint32_t idesc_) {
#pragma unroll 4
    for (int k = 0; k < k_steps; k++) mma_f16(d, da + 16u * k, dw + 16u * k, idesc_, k > 0);
    mma_f16(d, dones, dbias, idesc_, 1);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
k_mlp_tc(const uint2* __restrict__ list, const float4* __restrict__ list_mean, uint32_t n,
         const uint32_t* __restrict__ n_dev, const FrameInst* __restrict__ fis,
         const AssetDev* __restrict__ assets, float threshold, uint32_t* __restrict__ keep_bits,
         float* __restrict__ logits_out, uint32_t* __restrict__ err_flag) {
    extern __shared__ __align__(1024) uint8_t sm[];
    if (n_dev) n = min(n, *n_dev);   // device-side count (n is then the capacity)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
    int* s_red = reinterpret_cast<int*>(sm + kOffMisc + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"((uint32_t)kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar, kHalves);   // one commit per half per layer
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // constant A tile of the bias steps: row r = (1, 1, 0, ..., 0); core-matrix chunk 0 of row r
    // holds k = 0..7, chunk 1 k = 8..15
    {
        uint8_t* sOnes = sm + kOffOnes;
        st_chunk(sOnes, kSboK16, tid, 0, make_uint4(0x3F803F80u, 0u, 0u, 0u));
        st_chunk(sOnes, kSboK16, tid, 1, make_uint4(0u, 0u, 0u, 0u));
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    const int issue_h = warp & 1;   // lane 0 of warp h issues tile h's MMAs

    uint32_t phase = 0;
    int loaded = -1;
    bool abort = false;
    uint32_t pnext[kHalves][16];               // inputs of this thread's next-step rows, as BF16x2
    int pnext_asset[kHalves] = {-1, -1};       // the asset they were built for (-1: none)
    const uint32_t n_steps = (n + kRows - 1) / kRows;
    // row inputs of the next step are loaded one step ahead, so their latency overlaps the
    // current step's tensor-core chain
    uint2 e_next[kHalves];
    float4 m_next[kHalves];
#pragma unroll
    for (int h = 0; h < kHalves; h++) {
        const uint32_t i = blockIdx.x * kRows + h * 128 + tid;
        e_next[h] = make_uint2(0, 0);
        m_next[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (blockIdx.x < n_steps && i < n) {
            e_next[h] = __ldg(&list[i]);
            m_next[h] = __ldg(&list_mean[i]);
        }
    }
    for (uint32_t step = blockIdx.x; step < n_steps && !abort; step += gridDim.x) {
        uint2 e[kHalves];
        float4 m[kHalves], ci[kHalves];
        int my_asset[kHalves];
        bool pending[kHalves], keep[kHalves], gated[kHalves];
        float logit[kHalves];
#pragma unroll
        for (int h = 0; h < kHalves; h++) {
            const uint32_t i = step * kRows + h * 128 + tid;
            e[h] = e_next[h];
            m[h] = m_next[h];
            const uint32_t i_next = (step + gridDim.x) * kRows + h * 128 + tid;
            if (step + gridDim.x < n_steps && i_next < n) {
                e_next[h] = __ldg(&list[i_next]);
                m_next[h] = __ldg(&list_mean[i_next]);
            }
            // the list's mean carries the row's asset id in w; the instance values the inputs
            // need are loaded here, well ahead of their use after the asset pass
            my_asset[h] = i < n ? __float_as_int(m[h].w) : INT_MAX;
            ci[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            gated[h] = false;
            if (i < n) {
                const FrameInst& fr = fis[e[h].x];
                ci[h] = make_float4(fr.cam_local[0], fr.cam_local[1], fr.cam_local[2], fr.dist_scale);
                gated[h] = fr.gated != 0;
            }
            pending[h] = i < n;
            keep[h] = false;
            logit[h] = 0.0f;
        }
        bool pre_done = false;
        // rows of different assets (at instance boundaries) are evaluated in separate passes,
        // each with that asset's weights
        for (;;) {
            int cand = INT_MAX;
#pragma unroll
            for (int h = 0; h < kHalves; h++) cand = min(cand, pending[h] ? my_asset[h] : INT_MAX);
            cand = __reduce_min_sync(0xffffffffu, cand);
            if (lane == 0) s_red[warp] = cand;
            __syncthreads();
            const int cur = min(min(s_red[0], s_red[1]), min(s_red[2], s_red[3]));
            __syncthreads();
            if (cur == INT_MAX) break;
            const AssetDev& a = assets[cur];
            bool mine[kHalves];
#pragma unroll
            for (int h = 0; h < kHalves; h++) mine[h] = pending[h] && my_asset[h] == cur;
            if (a.w_tc == nullptr) {   // asset without an MLP: rendered unculled
#pragma unroll
                for (int h = 0; h < kHalves; h++)
                    if (mine[h]) { keep[h] = true; logit[h] = __int_as_float(0x7f800000); pending[h] = false; }
                continue;
            }
            if (cur != loaded) {
                const uint4* src = reinterpret_cast<const uint4*>(a.w_tc);
                uint4* dst = reinterpret_cast<uint4*>(sm);
                for (int k = tid; k < kBlobBytes / 16; k += kThreads) dst[k] = __ldg(&src[k]);
                loaded = cur;
            }
            // ---- inputs -> A (BF16), one row per half
#pragma unroll
            for (int h = 0; h < kHalves; h++) {
                uint32_t p[16];
                if (mine[h] && pnext_asset[h] == cur) {
#pragma unroll
                    for (int k = 0; k < 16; k++) p[k] = pnext[h][k];
                } else if (mine[h]) {
                    float f[32];
                    mlp_features(mlp_asset(a), ci[h].x, ci[h].y, ci[h].z, ci[h].w, m[h], f);
#pragma unroll
                    for (int k = 0; k < 16; k++) p[k] = bf16x2(f[2 * k], f[2 * k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; k++) p[k] = 0u;
                }
                uint8_t* sA = sm + kOffH + h * kHBytes;
#pragma unroll
                for (int c = 0; c < 4; c++)
                    st_chunk(sA, kSboK32, tid, c, make_uint4(p[4 * c], p[4 * c + 1], p[4 * c + 2], p[4 * c + 3]));
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();

            // ---- four tensor-core layers, both halves per round trip
            bool ok = true;
#pragma unroll 1
            for (int layer = 0; layer < 4 && ok; layer++) {
                // the two halves are issued by lane 0 of warps 0 and 1 concurrently (a single
                // thread issues an MMA only every ~50 cycles), each committing its own MMAs
                if (lane == 0 && warp < kHalves) {
                    tc_fence_after();
                    const uint32_t d = tmem + 64 * issue_h;
                    const uint8_t* sH = sm + kOffH + issue_h * kHBytes;
                    const uint64_t dOnes = sdesc(sm + kOffOnes, kLbo, kSboK16);
                    if (layer == 0)
                        issue_layer(d, sdesc(sH, kLbo, kSboK32), 2, sdesc(sm + kOffW1, kLbo, kSboK32),
                                    sdesc(sm + kOffB1, kLbo, kSboK16), dOnes, kIdescN64);
                    else if (layer == 1)
                        issue_layer(d, sdesc(sH, kLbo, kSboK64), 4, sdesc(sm + kOffW2, kLbo, kSboK64),
                                    sdesc(sm + kOffB2, kLbo, kSboK16), dOnes, kIdescN64);
                    else if (layer == 2)
                        issue_layer(d, sdesc(sH, kLbo, kSboK64), 4, sdesc(sm + kOffW3, kLbo, kSboK64),
                                    sdesc(sm + kOffB3, kLbo, kSboK16), dOnes, kIdescN64);
                    else
                        issue_layer(d, sdesc(sH, kLbo, kSboK64), 4, sdesc(sm + kOffW4, kLbo, kSboK64),
                                    sdesc(sm + kOffB4, kLbo, kSboK16), dOnes, kIdescN16);
                    mma_commit(mbar);
                }
                // the inputs of this thread's rows of the CTA's next step are built during the first
                // layer's round trip (when they belong to the asset of this pass), once every row of
                // this thread in the current step has had its inputs written (this pass or earlier)
                if (layer == 0 && !pre_done && (mine[0] || !pending[0]) && (mine[1] || !pending[1])) {
                    pre_done = true;
                    const MlpAsset ma = mlp_asset(a);
#pragma unroll
                    for (int h = 0; h < kHalves; h++) {
                        const uint32_t i_next = (step + gridDim.x) * kRows + h * 128 + tid;
                        pnext_asset[h] = -1;
                        if (step + gridDim.x < n_steps && i_next < n && __float_as_int(m_next[h].w) == cur) {
                            const FrameInst& fr = fis[e_next[h].x];
                            float f[32];
                            mlp_features(ma, fr.cam_local[0], fr.cam_local[1], fr.cam_local[2], fr.dist_scale,
                                         m_next[h], f);
#pragma unroll
                            for (int k = 0; k < 16; k++) pnext[h][k] = bf16x2(f[2 * k], f[2 * k + 1]);
                            pnext_asset[h] = cur;
                        }
                    }
                }
                const bool done = mbar_wait(mbar, phase);
                if (__syncthreads_or(!done)) { ok = false; break; }
                phase ^= 1u;
                tc_fence_after();
                if (layer < 3) {
#pragma unroll
                    for (int h = 0; h < kHalves; h++)
                        epilogue_hidden(t_lane + 64 * h, sm + kOffH + h * kHBytes, tid);
                    fence_async_smem();
                    tc_fence_before();
                    __syncthreads();
                } else {
#pragma unroll
                    for (int h = 0; h < kHalves; h++) {
                        uint32_t r[2];
                        tmem_ld2(t_lane + 64 * h, r);
                        const float lg = __uint_as_float(r[0]) + __uint_as_float(r[1]);
                        if (mine[h]) {
                            logit[h] = lg;
                            keep[h] = gated[h] || (lg > threshold);
                            pending[h] = false;
                        }
                    }
                    tc_fence_before();
                }
            }
            if (!ok) {
                if (tid == 0) atomicExch(err_flag, 1u);
                abort = true;
                break;
            }
        }
        if (abort) break;
#pragma unroll
        for (int h = 0; h < kHalves; h++) {
            const uint32_t row0 = step * kRows + h * 128;
            const uint32_t w = __ballot_sync(0xffffffffu, keep[h]);
            if (lane == 0 && row0 + warp * 32 < n) keep_bits[(row0 >> 5) + warp] = w;
            if (logits_out && row0 + tid < n) logits_out[row0 + tid] = logit[h];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"((uint32_t)kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------------ host side
size_t mlp_tc_weight_bytes() { return (size_t)kBlobBytes; }

static uint16_t f32_to_bf16_rne(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);   // inf / nan kept
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static float bf16_to_f32(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Packs W1 (64x32), W2, W3 (64x64) as BF16 core-matrix tiles (row = output neuron, K-major), w4
// as rows 0 (high part) and 1 (low part) of a 16 x 64 tile, and every bias as an N x 16 tile
// with the high part in column 0 and the low part (bias - high, rounded) in column 1, in the
// shared-memory byte layout k_mlp_tc reads.
void mlp_tc_pack_weights(const float* w, uint8_t* out) {
    memset(out, 0, kBlobBytes);
    const float* W1 = w;
    const float* b1 = W1 + 64 * 32;
    const float* W2 = b1 + 64;
    const float* b2 = W2 + 64 * 64;
    const float* W3 = b2 + 64;
    const float* b3 = W3 + 64 * 64;
    const float* W4 = b3 + 64;
    const float* b4 = W4 + 64;
    auto put1 = [&](int off, int K, int nrow, int k, uint16_t v) {
        const int b = off + (nrow / 8) * 16 * K + (k / 8) * 128 + (nrow % 8) * 16 + (k % 8) * 2;
        memcpy(out + b, &v, 2);
    };
    auto put = [&](int off, int K, int rows, const float* Wm) {
        for (int nrow = 0; nrow < rows; nrow++)
            for (int k = 0; k < K; k++) put1(off, K, nrow, k, f32_to_bf16_rne(Wm[nrow * K + k]));
    };
    auto split = [&](int off, int K, int nrow, int k0, float x) {   // x = high + low
        const uint16_t hi = f32_to_bf16_rne(x);
        put1(off, K, nrow, k0, hi);
        put1(off, K, nrow, k0 + 1, f32_to_bf16_rne(x - bf16_to_f32(hi)));
    };
    put(kOffW1, 32, 64, W1);
    put(kOffW2, 64, 64, W2);
    put(kOffW3, 64, 64, W3);
    for (int k = 0; k < 64; k++) {   // w4: rows 0 and 1 of the 16 x 64 tile
        const uint16_t hi = f32_to_bf16_rne(W4[k]);
        put1(kOffW4, 64, 0, k, hi);
        put1(kOffW4, 64, 1, k, f32_to_bf16_rne(W4[k] - bf16_to_f32(hi)));
    }
    for (int nrow = 0; nrow < 64; nrow++) {
        split(kOffB1, 16, nrow, 0, b1[nrow]);
        split(kOffB2, 16, nrow, 0, b2[nrow]);
        split(kOffB3, 16, nrow, 0, b3[nrow]);
    }
    split(kOffB4, 16, 0, 0, b4[0]);
}

cudaError_t launch_mlp_tc(const uint2* list, const float4* list_mean, uint32_t n, const uint32_t* n_dev,
                          const FrameInst* fi,
                          const AssetDev* assets,
                          float threshold, uint32_t* keep_bits, float* logits_out, uint32_t* err_flag,
                          int num_sms, int ctas_per_sm, cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    static std::atomic<uint64_t> attr_done{0};
    {
        cudaError_t e = once_per_device(attr_done, [] {
            return cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        });
        if (e != cudaSuccess) return e;
    }
    const uint32_t steps = (n + kRows - 1) / kRows;
    const uint32_t per_sm = ctas_per_sm >= 1 && ctas_per_sm <= kCtasPerSm ? (uint32_t)ctas_per_sm
                                                                           : (uint32_t)kCtasPerSm;
    const uint32_t grid = std::min<uint32_t>(steps, (uint32_t)num_sms * per_sm);
    NVGS_LAUNCH(log, s, "k_mlp_tc", k_mlp_tc<<<grid, kThreads, kSmemBytes, s>>>(list, list_mean, n, n_dev, fi, assets, threshold, keep_bits, logits_out, err_flag));
    return cudaGetLastError();
}

}  // namespace nvgs
