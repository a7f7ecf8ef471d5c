// S2, BF16 tensor-core variant: the per-asset visibility MLP (32 -> 64 -> 64 -> 64 -> 1, ReLU;
// NVGS Sec. 3.2, queried per in-frustum Gaussian as in Sec. 3.3) on the 5th-generation tensor
// cores (tcgen05), BF16 operands with FP32 accumulation in tensor memory (TMEM).
//
// One CTA = one warpgroup (128 threads) walking a contiguous range of 128-Gaussian steps of the
// in-frustum list (instance-major, so the asset -- and the weights in shared memory -- rarely
// changes within a range); thread r owns row r (TMEM lane r).  Four CTAs share an SM, each with 128 TMEM columns:
//   [0, 64)    D   FP32 accumulator of the current layer (N = 64)
//   [64, 96)   H   the layer's ReLU'd activations as BF16 pairs: the next layer's A operand
//   [96, 128)  IN  two 16-column buffers of BF16 inputs (this step's and the next step's)
// Every activation operand lives in tensor memory (tcgen05.mma with A from TMEM), so an MMA reads
// only its weight tile from shared memory, and a hidden epilogue is tcgen05.ld -> cvt.rn.relu.bf16x2
// -> tcgen05.st, with no shared-memory store or proxy fence.  Per step:
//   1. lane 0 of warp 0 issues the first layer (A = IN[b], K = 32) and commits to the mbarrier;
//      meanwhile every thread builds its row of the NEXT step's inputs (Eq. 2 distance, frequency
//      encoding) into IN[b ^ 1];
//   2. per hidden layer: wait for the commit, epilogue into H, barrier, issue the next layer;
//   3. the third layer's epilogue also evaluates the 64 -> 1 output layer on the CUDA cores
//      (FP32 w4 and b4 on the FP32 ReLU activations), so a step costs three MMA round
//      trips: each round trip (issue, commit, mbarrier) has a fixed latency of several hundred
//      cycles, which bounds the kernel more than the tensor work of its 64-wide layers.
// The hidden biases cost no CUDA-core work: every layer ends with one more K = 16 MMA step of a constant A
// tile (shared memory) whose first two columns are 1 against a B tile holding the bias split into
// BF16 high and low parts, so the accumulator already contains W h + b (to about 2^-16 of b).
// Rows of several assets in one step (at instance boundaries) run one pass per asset over the same
// inputs, each with that asset's weights.
//
// Weight layout (B operands, K-major, no swizzle): 8 x 16-byte core matrices; element (n, k) of a
// tile with K columns sits at (n / 8) * SBO + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2 with
// SBO = 16 * K bytes.  The host packs the weights into exactly this byte layout
// (mlp_tc_pack_weights); they are copied to shared memory with 16-byte loads.
//
// Every mbarrier wait is bounded; on a timeout the CTA sets the error flag, waits (bounded) for its
// MMAs in flight, frees its TMEM and returns.
#include <climits>
#include <cstring>

#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace nvgs {

namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kCtasPerSm = 4;
constexpr int kRows = 128;                 // rows per CTA step (one per thread)
constexpr int kTmemCols = 128;
constexpr uint32_t kColD = 0;
constexpr uint32_t kColH = 64;
constexpr uint32_t kColIn = 96;            // + 16 * buffer
// shared-memory map (bytes); the weight blob [0, kBlobBytes) is packed on the host
constexpr int kOffW1 = 0;            // 64 x 32 BF16
constexpr int kOffW2 = 4096;         // 64 x 64 BF16
constexpr int kOffW3 = 12288;        // 64 x 64 BF16
constexpr int kOffB1 = 20480;        // bias tiles, N x 16 BF16: column 0 = high, 1 = low part
constexpr int kOffB2 = 22528;
constexpr int kOffB3 = 24576;
constexpr int kOffW4 = 26624;        // FP32 w4[64], then b4
constexpr int kBlobBytes = 26896;
constexpr int kOffOnes = (kBlobBytes + 1023) / 1024 * 1024;   // 128 x 16 BF16, columns 0 and 1 = 1
                                                              // (written in the kernel)
constexpr int kOffRowM = kOffOnes + 4096;       // next step's mean per row (16 B)
constexpr int kOffRowE = kOffRowM + kRows * 16;  // next step's list entry per row (8 B)
constexpr int kOffMisc = kOffRowE + kRows * 8;
constexpr int kSmemBytes = kOffMisc + 128;
constexpr uint32_t kSboK16 = 256;    // 16 * 16
constexpr uint32_t kSboK32 = 512;    // 16 * 32
constexpr uint32_t kSboK64 = 1024;   // 16 * 64
constexpr uint32_t kLbo = 128;

// kind::f16 instruction descriptors: D = F32 (bit 4), A = B = BF16 (bits 7, 10), both K-major,
// N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t idesc(uint32_t n) { return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24); }
constexpr uint32_t kIdescN64 = idesc(64);

// (lo, hi) -> BF16x2 with ReLU, lo in the low half (the lower k).
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

// TMEM accumulator (this lane, 64 columns, bias included) -> ReLU -> BF16 pairs in H, in two
// 32-column halves (fewer live registers).
__device__ __forceinline__ void epilogue_hidden(uint32_t t_lane) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
        uint32_t r[32];
        tmem_ld32(t_lane + kColD + 32 * h, r);
        uint32_t p[16];
#pragma unroll
        for (int q = 0; q < 16; q++) p[q] = bf16x2_relu(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
        tmem_st16(t_lane + kColH + 16 * h, p);
    }
}

// Output layer on the CUDA cores: acc (64 FP32 columns, b3 included) -> ReLU -> dot with the FP32
// w4 (packed FP32x2 FMAs over neighbouring columns) -> + b4.  The third layer's activations stay
// in FP32 here: only the hidden activations that feed a tensor-core layer are rounded to BF16.
__device__ __forceinline__ float epilogue_output(uint32_t t_lane, const float* __restrict__ w4) {
    float2 a01 = make_float2(w4[64], 0.0f), a23 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int h = 0; h < 2; h++) {
        uint32_t r[32];
        tmem_ld32(t_lane + kColD + 32 * h, r);
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
            const float4 w = *reinterpret_cast<const float4*>(w4 + 32 * h + q);
            a01 = __ffma2_rn(make_float2(fmaxf(__uint_as_float(r[q]), 0.0f), fmaxf(__uint_as_float(r[q + 1]), 0.0f)),
                             make_float2(w.x, w.y), a01);
            a23 = __ffma2_rn(make_float2(fmaxf(__uint_as_float(r[q + 2]), 0.0f), fmaxf(__uint_as_float(r[q + 3]), 0.0f)),
                             make_float2(w.z, w.w), a23);
        }
    }
    return (a01.x + a01.y) + (a23.x + a23.y);
}

// Asynchronous copy of the mean of this thread's next row into shared memory (read only when the
// next step's inputs are built, so no register holds it meanwhile; the row's list entry is stored
// beside it with a plain store).
__device__ __forceinline__ void prefetch_mean(float4* s_m, const float4* m) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s_m)), "l"(m) : "memory");
}
__device__ __forceinline__ void prefetch_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void prefetch_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// This thread's row of inputs (32 features as 16 BF16 pairs) into its lane of an input buffer;
// rows past the list get zeros (their outputs are never used).  Returns the row's instance gate
// (Sec. 3.3: an instance nearer than d_min bypasses the MLP).
__device__ __forceinline__ bool build_inputs(uint32_t t_in, bool valid, uint2 e, float4 m, int asset,
                                             const FrameInst* __restrict__ fis,
                                             const AssetDev* __restrict__ assets) {
    uint32_t p[16];
    bool gated = false;
    if (valid) {
        const FrameInst& fr = fis[e.x];
        gated = fr.gated != 0;
        const MlpAsset ma = mlp_asset(assets[asset]);
        float f[32];
        mlp_features(ma, fr.cam_local[0], fr.cam_local[1], fr.cam_local[2], fr.dist_scale, m, f);
#pragma unroll
        for (int k = 0; k < 16; k++) p[k] = bf16x2(f[2 * k], f[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < 16; k++) p[k] = 0u;
    }
    tmem_st16(t_in, p);
    return gated;
}

// The next step's inputs from the row staged in shared memory; also returns that row's asset.
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

// One layer for the CTA's 128 rows (issued by one thread): K / 16 steps of A (TMEM) x W, then the
// bias step (A = the ones tile in shared memory), committed to the mbarrier.
__device__ __forceinline__ void issue_layer(uint32_t d, uint32_t a_tmem, int k_steps, uint64_t dw,
                                            uint64_t dbias, uint64_t dones, uint32_t idesc_, uint64_t* mbar) {
#pragma unroll 4
    for (int k = 0; k < k_steps; k++) mma_f16_ts(d, a_tmem + 8u * k, dw + 16u * k, idesc_, k > 0);
    mma_f16(d, dones, dbias, idesc_, 1);
    mma_commit(mbar);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
k_mlp_tc(const uint2* __restrict__ list, uint32_t n,
         const uint32_t* __restrict__ n_dev, const FrameInst* __restrict__ fis,
         const AssetDev* __restrict__ assets, float threshold, uint32_t* __restrict__ keep_bits,
         float* __restrict__ logits_out, uint32_t* __restrict__ err_flag) {
    extern __shared__ __align__(1024) uint8_t sm[];
    if (n_dev) n = min(n, *n_dev);   // device-side count (n is then the capacity)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
    // reduction slots: per step parity [0,4) min and [4,8) max (so that a warp that runs ahead into
    // the next step never overwrites a slot another warp has still to read), then [16,20) pass min
    int* s_red = reinterpret_cast<int*>(sm + kOffMisc + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"((uint32_t)kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar, 1);   // one commit per layer
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

    uint32_t phase = 0;
    int loaded = -1;              // asset whose weights are in shared memory
    int known = -1;               // asset whose MLP presence is in has_mlp
    bool has_mlp = false;
    bool abort = false;
    uint32_t buf = 0;
    const uint32_t n_steps = (n + kRows - 1) / kRows;
    // this CTA's contiguous range of steps [s_begin, s_end)
    const uint32_t per_cta = (n_steps + gridDim.x - 1) / gridDim.x;
    const uint32_t s_begin = min(n_steps, blockIdx.x * per_cta);
    const uint32_t s_end = min(n_steps, s_begin + per_cta);
    // the first step's inputs are built here, every later step's during the previous step's
    // first-layer round trip (from the list entry and mean staged in shared memory)
    uint2* s_e = reinterpret_cast<uint2*>(sm + kOffRowE) + tid;
    float4* s_m = reinterpret_cast<float4*>(sm + kOffRowM) + tid;
    int my_asset_next = INT_MAX;   // asset of this thread's row of the next step
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
    const uint64_t dOnes = sdesc(sm + kOffOnes, kLbo, kSboK16);
    const uint64_t dW1 = sdesc(sm + kOffW1, kLbo, kSboK32), dB1 = sdesc(sm + kOffB1, kLbo, kSboK16);
    const uint64_t dW2 = sdesc(sm + kOffW2, kLbo, kSboK64), dB2 = sdesc(sm + kOffB2, kLbo, kSboK16);
    const uint64_t dW3 = sdesc(sm + kOffW3, kLbo, kSboK64), dB3 = sdesc(sm + kOffB3, kLbo, kSboK16);

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
        // the CTA's smallest and largest asset of this step; the barrier also orders this step's
        // input stores and the previous step's accumulator reads before the first MMA
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
        const uint32_t a_in = tmem + kColIn + 16u * buf;
        int cur = step_min;
        while (cur != INT_MAX) {
            const bool mine = pending && my_asset == cur;
            if (cur != known) { has_mlp = assets[cur].w_tc != nullptr; known = cur; }
            if (!has_mlp) {   // asset without an MLP: rendered unculled
                if (mine) { keep = true; logit = __int_as_float(0x7f800000); }
            } else {
                if (cur != loaded) {   // every MMA of earlier passes has completed (waited on)
                    const uint4* src = reinterpret_cast<const uint4*>(assets[cur].w_tc);
                    uint4* dst = reinterpret_cast<uint4*>(sm);
                    // four loads in flight per thread before their stores
                    for (int k0 = tid; k0 < kBlobBytes / 16; k0 += 4 * kThreads) {
                        uint4 v[4];
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (k0 + j * kThreads < kBlobBytes / 16) v[j] = __ldg(&src[k0 + j * kThreads]);
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (k0 + j * kThreads < kBlobBytes / 16) dst[k0 + j * kThreads] = v[j];
                    }
                    fence_async_smem();
                    __syncthreads();
                    loaded = cur;
                }
                // ---- three layers, one round trip each; the output layer in the last epilogue
                bool ok = true;
#pragma unroll 1
                for (int layer = 0; layer < 3; layer++) {
                    if (tid == 0) {
                        tc_fence_after();
                        if (layer == 0) issue_layer(tmem + kColD, a_in, 2, dW1, dB1, dOnes, kIdescN64, mbar);
                        else if (layer == 1) issue_layer(tmem + kColD, tmem + kColH, 4, dW2, dB2, dOnes, kIdescN64, mbar);
                        else issue_layer(tmem + kColD, tmem + kColH, 4, dW3, dB3, dOnes, kIdescN64, mbar);
                    }
                    if (layer == 0 && !built_next) {   // overlaps the first layer's round trip
                        if (has_next) gated_next = build_next(t_lane + kColIn + 16u * (buf ^ 1u), next_valid, s_e, s_m,
                                                              fis, assets, my_asset_next);
                        built_next = true;
                    }
                    ok = mbar_wait(mbar, phase);
                    phase ^= 1u;
                    tc_fence_after();
                    if (layer < 2) {
                        if (ok) epilogue_hidden(t_lane);
                        tmem_wait_st();
                    } else if (ok) {
                        const float lg = epilogue_output(t_lane, reinterpret_cast<const float*>(sm + kOffW4));
                        if (mine) { logit = lg; keep = gated || (lg > threshold); }
                    }
                    tc_fence_before();
                    if (__syncthreads_or(!ok)) { abort = true; break; }
                }
                if (abort) break;
            }
            if (mine) pending = false;
            if (step_min == step_max) break;   // one asset in this step (the common case)
            // next asset of this step: the smallest one still pending
            {
                const int cand = __reduce_min_sync(0xffffffffu, pending ? my_asset : INT_MAX);
                if (lane == 0) s_red[16 + warp] = cand;
            }
            __syncthreads();
            cur = min(min(s_red[16], s_red[17]), min(s_red[18], s_red[19]));
            __syncthreads();
        }
        if (abort) break;
        if (!built_next && has_next) gated_next = build_next(t_lane + kColIn + 16u * (buf ^ 1u), next_valid, s_e, s_m,
                                                             fis, assets, my_asset_next);
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
        // the MMAs of the layer whose wait gave up may still be running: wait for them (bounded)
        // before the tensor memory is released
        mbar_wait(mbar, phase ^ 1u);
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

// Packs W1 (64x32), W2, W3 (64x64) as BF16 core-matrix tiles (row = output neuron, K-major), every
// hidden bias as a 64 x 16 tile with the high part in column 0 and the low part (bias - high,
// rounded) in column 1, and w4, b4 as FP32, in the shared-memory byte layout k_mlp_tc reads.
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
    for (int nrow = 0; nrow < 64; nrow++) {
        split(kOffB1, 16, nrow, 0, b1[nrow]);
        split(kOffB2, 16, nrow, 0, b2[nrow]);
        split(kOffB3, 16, nrow, 0, b3[nrow]);
    }
    memcpy(out + kOffW4, W4, 64 * sizeof(float));
    memcpy(out + kOffW4 + 256, b4, sizeof(float));
}

cudaError_t launch_mlp_tc(const uint2* list, uint32_t n, const uint32_t* n_dev,
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
    NVGS_LAUNCH(log, s, "k_mlp_tc", k_mlp_tc<<<grid, kThreads, kSmemBytes, s>>>(list, n, n_dev, fi, assets, threshold, keep_bits, logits_out, err_flag));
    return cudaGetLastError();
}

}  // namespace nvgs
