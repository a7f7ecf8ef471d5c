// S1 frustum culling on the Gaussian mean and S3 stream compaction (NVGS Sec. 3.3).
//
// Work layout: every instance is cut into chunks of kChunk consecutive Gaussians.  One CTA
// handles one chunk: 256 threads x 8 loads of a 16-byte (x, y, z, opacity-logit) vector, the
// in-frustum predicate becomes one ballot word per warp and load step, so the chunk's 2048
// decisions are 64 consecutive bitmask words.  Compaction is then popcount -> exclusive scan of
// per-chunk counts -> an order-preserving expansion of the set bits into (instance, gaussian)
// entries.  The survivor order is therefore instance-major, Gaussian-minor (the order the
// oracle uses to break depth ties).
#include "nvgs_internal.cuh"

namespace nvgs {

// ------------------------------------------------------------------ per-frame instance setup
// FP64 composition of camera and instance transforms (one thread per instance), rounded once to
// FP32 so that the per-Gaussian camera-space position is three FMAs per coordinate.
__global__ void k_instance_setup(const InstanceRaw* __restrict__ inst, int n_inst,
                                 const AssetDev* __restrict__ assets, const CamParams* __restrict__ camp,
                                 FrameInst* __restrict__ out, const int2* __restrict__ fi_map) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_inst) return;
    // frame instance k: (view, instance) of a multi-view batch, or instance k of view 0
    const int2 vi = fi_map ? fi_map[k] : make_int2(0, k);
    const CamParams cam = camp[vi.x];
    InstanceRaw r = inst[vi.y];
    const AssetDev& a = assets[r.asset];
    double Rc[9], Ri[9], W[9];
    for (int k = 0; k < 9; k++) { Rc[k] = cam.R[k]; Ri[k] = r.R[k]; }
    for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++)
            W[3 * p + q] = Rc[3 * p] * Ri[q] + Rc[3 * p + 1] * Ri[3 + q] + Rc[3 * p + 2] * Ri[6 + q];
    double s = r.s;
    double b[3], c[3], cl[3];
    for (int p = 0; p < 3; p++)
        b[p] = Rc[3 * p] * r.t[0] + Rc[3 * p + 1] * r.t[1] + Rc[3 * p + 2] * r.t[2] + cam.t[p];
    for (int q = 0; q < 3; q++)   // camera centre -R^T t
        c[q] = -(Rc[q] * cam.t[0] + Rc[3 + q] * cam.t[1] + Rc[6 + q] * cam.t[2]);
    for (int q = 0; q < 3; q++) {  // R_i^T (c - t_i) / s
        double d0 = c[0] - r.t[0], d1 = c[1] - r.t[1], d2 = c[2] - r.t[2];
        cl[q] = (Ri[q] * d0 + Ri[3 + q] * d1 + Ri[6 + q] * d2) / s;
    }
    FrameInst f;
    for (int k = 0; k < 9; k++) { f.W[k] = (float)W[k]; f.M[k] = (float)(s * W[k]); }
    for (int p = 0; p < 3; p++) { f.b[p] = (float)b[p]; f.cam_local[p] = (float)cl[p]; }
    f.s = r.s;
    f.asset = r.asset;
    double dist_scale = (double)a.train_focal / (double)cam.f_r;
    f.dist_scale = (double)dist_scale;

    // bounding sphere of the means (centre of the box, half its diagonal) against the planes
    // of the guard-band frustum; a small relative margin keeps the test conservative.
    double cx = 0, cy = 0, cz = 0;
    for (int q = 0; q < 3; q++) {
        cx += s * W[q] * a.bbox_c[q];
        cy += s * W[3 + q] * a.bbox_c[q];
        cz += s * W[6 + q] * a.bbox_c[q];
    }
    cx += b[0]; cy += b[1]; cz += b[2];
    double rad = s * (double)a.bbox_r * (1.0 + 1e-4) + 1e-6;
    double lx = cam.lim_x, ly = cam.lim_y;
    int outside = (cz < (double)cam.z_near - rad) ||
                  (lx * cz - fabs(cx) < -rad * sqrt(1.0 + lx * lx)) ||
                  (ly * cz - fabs(cy) < -rad * sqrt(1.0 + ly * ly));
    f.visible = !outside;

    // MLP gate: corrected distance of the box centre below d_min -> keep everything (Sec. 3.3)
    double dd = 0;
    for (int q = 0; q < 3; q++) dd += ((double)a.bbox_c[q] - cl[q]) * ((double)a.bbox_c[q] - cl[q]);
    f.gated = cam.mlp_gate && (sqrt(dd) * dist_scale) < (double)a.d_min;
    // assets without an MLP are rendered unculled (Fig. 4: mixed neural / plain assets)
    f.no_mlp = a.w_fp32 == nullptr;
    f.view = vi.x;
    out[k] = f;
}

cudaError_t launch_instance_setup(const InstanceRaw* inst, int n_inst, const AssetDev* assets,
                                  const CamParams* cam_dev, FrameInst* out, cudaStream_t s, LaunchLog* log,
                                  const int2* fi_map, int n_fi) {
    const int n = fi_map ? n_fi : n_inst;
    if (n <= 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_instance_setup", k_instance_setup<<<(n + 127) / 128, 128, 0, s>>>(inst, n, assets, cam_dev, out, fi_map));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ S1
__device__ __forceinline__ bool in_frustum(const FrameInst& f, const CamParams& cam, float4 m) {
    const float3 p = cam_point(f, m.x, m.y, m.z);
    return (p.z > cam.z_near) && (fabsf(p.x) <= cam.lim_x * p.z) && (fabsf(p.y) <= cam.lim_y * p.z);
}

__global__ void __launch_bounds__(256) k_frustum(const Chunk* __restrict__ chunks,
                                                 const FrameInst* __restrict__ fi,
                                                 const AssetDev* __restrict__ assets, const CamParams* __restrict__ camp,
                                                 uint32_t* __restrict__ bits,
                                                 uint32_t* __restrict__ chunk_counts) {
    __shared__ uint32_t warp_tot[8];
    const int c = blockIdx.x;
    const Chunk ch = chunks[c];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* out = bits + (size_t)c * kChunkWords;
    const FrameInst& f = fi[ch.inst];
    const CamParams cam = camp[f.view];
    uint32_t tot = 0;
    if (!f.visible) {
        if (threadIdx.x < kChunkWords) out[threadIdx.x] = 0u;
        if (threadIdx.x == 0) chunk_counts[c] = 0u;
        return;
    }
    const float4* __restrict__ mean = assets[f.asset].mean_op + ch.g0;
    float4 m[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {  // issue all loads first
        int k = j * 256 + threadIdx.x;
        m[j] = k < ch.count ? __ldg(&mean[k]) : make_float4(0.f, 0.f, -1.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
        int k = j * 256 + threadIdx.x;
        bool p = (k < ch.count) && in_frustum(f, cam, m[j]);
        uint32_t w = __ballot_sync(0xffffffffu, p);
        if (lane == 0) out[j * 8 + warp] = w;
        tot += __popc(w);
    }
    if (lane == 0) warp_tot[warp] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < 8; w++) s += warp_tot[w];
        chunk_counts[c] = s;
    }
}

cudaError_t launch_frustum(const Chunk* chunks, int n_chunks, const FrameInst* fi,
                           const AssetDev* assets, const CamParams* cam_dev, uint32_t* bits,
                           uint32_t* chunk_counts, cudaStream_t s, LaunchLog* log) {
    if (n_chunks <= 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_frustum", k_frustum<<<n_chunks, 256, 0, s>>>(chunks, fi, assets, cam_dev, bits, chunk_counts));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ bitmask expansion
// Exclusive prefix of the 64 word popcounts of one chunk, in shared memory.
__device__ __forceinline__ void chunk_word_prefix(const uint32_t* __restrict__ words, int n_words,
                                                  uint32_t* s_word, uint32_t* s_pref) {
    if (threadIdx.x < 64) {
        uint32_t w = threadIdx.x < n_words ? words[threadIdx.x] : 0u;
        s_word[threadIdx.x] = w;
        uint32_t c = __popc(w);
        // two-warp inclusive scan of 64 values
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) c += t;
        }
        s_pref[threadIdx.x] = c;  // inclusive within each warp
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        uint32_t incl = s_pref[threadIdx.x] + (threadIdx.x >= 32 ? s_pref[31] : 0u);
        __syncwarp();
        s_pref[64 + threadIdx.x] = incl - __popc(s_word[threadIdx.x]);  // exclusive
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_expand_chunks(const Chunk* __restrict__ chunks,
                                                       const uint32_t* __restrict__ bits,
                                                       const uint32_t* __restrict__ chunk_offsets,
                                                       uint2* __restrict__ out) {
    __shared__ uint32_t s_word[64];
    __shared__ uint32_t s_pref[128];
    const int c = blockIdx.x;
    const Chunk ch = chunks[c];
    chunk_word_prefix(bits + (size_t)c * kChunkWords, kChunkWords, s_word, s_pref);
    const uint32_t base = chunk_offsets[c];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        int w = warp * 8 + k;
        uint32_t word = s_word[w];
        if ((word >> lane) & 1u) {
            uint32_t pos = base + s_pref[64 + w] + __popc(word & lt);
            const uint32_t g = (uint32_t)(ch.g0 + w * 32 + lane);
            out[pos] = make_uint2((uint32_t)ch.inst, g);
        }
    }
}

cudaError_t launch_expand_chunks(const Chunk* chunks, int n_chunks, const uint32_t* bits,
                                 const uint32_t* chunk_offsets, uint2* out, cudaStream_t s,
                                 LaunchLog* log) {
    if (n_chunks <= 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_expand_chunks", k_expand_chunks<<<n_chunks, 256, 0, s>>>(chunks, bits, chunk_offsets, out));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ S3 on a list
__global__ void __launch_bounds__(64) k_bit_counts(const uint32_t* __restrict__ bits, uint32_t n,
                                                   const uint32_t* __restrict__ n_dev,
                                                   uint32_t* __restrict__ block_counts) {
    if (n_dev) n = min(n, *n_dev);   // blocks past the device count write 0
    const uint32_t n_words = (n + 31) / 32;
    const uint32_t w = blockIdx.x * kChunkWords + threadIdx.x;
    uint32_t c = w < n_words ? __popc(bits[w]) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ uint32_t s[2];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) block_counts[blockIdx.x] = s[0] + s[1];
}

cudaError_t launch_bit_counts(const uint32_t* bits, uint32_t n, const uint32_t* n_dev,
                              uint32_t* block_counts, cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    uint32_t nb = (n + kChunk - 1) / kChunk;
    NVGS_LAUNCH(log, s, "k_bit_counts", k_bit_counts<<<nb, 64, 0, s>>>(bits, n, n_dev, block_counts));
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_compact_list(const uint2* __restrict__ list, uint32_t n,
                                                      const uint32_t* __restrict__ n_dev,
                                                      const uint32_t* __restrict__ bits,
                                                      const uint32_t* __restrict__ block_offsets,
                                                      uint2* __restrict__ out) {
    __shared__ uint32_t s_word[64];
    __shared__ uint32_t s_pref[128];
    if (n_dev) n = min(n, *n_dev);
    const uint32_t n_words = (n + 31) / 32;
    const uint32_t w0 = blockIdx.x * kChunkWords;
    if (w0 >= n_words) return;
    int nw = (int)min((uint32_t)kChunkWords, n_words - w0);
    chunk_word_prefix(bits + w0, nw, s_word, s_pref);
    const uint32_t base = block_offsets[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        int w = warp * 8 + k;
        uint32_t word = s_word[w];
        if ((word >> lane) & 1u) {
            uint32_t pos = base + s_pref[64 + w] + __popc(word & lt);
            out[pos] = list[(size_t)(w0 + w) * 32 + lane];
        }
    }
}

cudaError_t launch_compact_list(const uint2* list, uint32_t n, const uint32_t* n_dev, const uint32_t* bits,
                                const uint32_t* block_offsets, uint2* out, cudaStream_t s,
                                LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    uint32_t nb = (n + kChunk - 1) / kChunk;
    NVGS_LAUNCH(log, s, "k_compact_list", k_compact_list<<<nb, 256, 0, s>>>(list, n, n_dev, bits, block_offsets, out));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ nvgs_query_visibility
__global__ void k_scatter_visibility(const uint2* __restrict__ list, uint32_t n,
                                     const uint32_t* __restrict__ keep_bits,
                                     const float* __restrict__ logits,
                                     const int64_t* __restrict__ inst_offset,
                                     const FrameInst* __restrict__ fi, float* __restrict__ out_logits,
                                     uint8_t* __restrict__ out_keep) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint2 e = list[i];
    int64_t idx = inst_offset[e.x] + e.y;
    if (out_keep) out_keep[idx] = (uint8_t)((keep_bits[i >> 5] >> (i & 31)) & 1u);
    if (out_logits)
        out_logits[idx] = (fi[e.x].gated || fi[e.x].no_mlp) ? __int_as_float(0x7f800000) : logits[i];
}

cudaError_t launch_scatter_visibility(const uint2* list, uint32_t n, const uint32_t* keep_bits,
                                      const float* logits, const int64_t* inst_offset,
                                      const FrameInst* fi, float* out_logits, uint8_t* out_keep,
                                      cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_scatter_visibility", k_scatter_visibility<<<(n + 255) / 256, 256, 0, s>>>(list, n, keep_bits, logits, inst_offset, fi, out_logits, out_keep));
    return cudaGetLastError();
}

}  // namespace nvgs
