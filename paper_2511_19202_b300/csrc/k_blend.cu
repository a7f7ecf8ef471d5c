// S6: front-to-back alpha compositing per tile (NVGS Sec. 4.1 blending rules on the 3DGS tiled
// rasteriser).
//
// One CTA per TS x TS tile, one thread per pixel.  The tile's Gaussians (a contiguous range of
// the sorted pairs) are staged through shared memory in batches of TS*TS records, gathered by
// survivor index; every thread then walks the batch for its pixel:
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy      (conic [[A, B], [B, C]], pixel centre - mean)
//   skip if power > 0;  alpha = min(alpha_max, opacity e^power);  skip if alpha < alpha_min;
//   stop (without blending) if T (1 - alpha) < t_stop;  C += alpha T rgb;  T *= 1 - alpha.
// The CTA leaves the range as soon as every pixel has stopped (a block-wide vote per batch).
// With `mark` set, every blended fragment also flags its survivor (the visibility labeller).
#include "nvgs_internal.cuh"

namespace nvgs {

template <int TS>
__global__ void __launch_bounds__(TS* TS) k_blend(const uint32_t* __restrict__ ranges,
                                                  const uint32_t* __restrict__ values,
                                                  const float4* __restrict__ rec, CamParams cam,
                                                  float* __restrict__ image, float* __restrict__ final_T,
                                                  int32_t* __restrict__ n_contrib,
                                                  uint8_t* __restrict__ mark) {
    constexpr int B = TS * TS;
    __shared__ float4 s_a[B];
    __shared__ float4 s_b[B];
    __shared__ float4 s_c[B];
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int px = tx * TS + (threadIdx.x % TS), py = ty * TS + (threadIdx.x / TS);
    const bool inside = px < cam.W && py < cam.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    int count = 0;
    bool done = !inside;
    for (uint32_t base = start; base < end; base += B) {
        if (__syncthreads_count(done) == B) break;   // also: previous batch fully consumed
        const uint32_t k = base + threadIdx.x;
        if (k < end) {
            const size_t idx = 3 * (size_t)values[k];
            s_a[threadIdx.x] = __ldg(&rec[idx]);
            s_b[threadIdx.x] = __ldg(&rec[idx + 1]);
            s_c[threadIdx.x] = __ldg(&rec[idx + 2]);
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)B, end - base);
        for (int j = 0; j < nb && !done; j++) {
            const float4 a = s_a[j];
            const float dx = fx - a.x, dy = fy - a.y;
            const float4 b = s_b[j];
            const float power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
            if (power > 0.0f) continue;
            const float alpha = fminf(cam.alpha_max, b.y * __expf(power));
            if (alpha < cam.alpha_min) continue;
            const float nt = T * (1.0f - alpha);
            if (nt < cam.t_stop) { done = true; break; }
            const float4 c = s_c[j];
            const float w = alpha * T;
            if (mark) mark[values[base + j]] = 1;   // contribution alpha * T > 0 (Sec. 3.1)
            C0 = fmaf(w, c.x, C0);
            C1 = fmaf(w, c.y, C1);
            C2 = fmaf(w, c.z, C2);
            T = nt;
            count++;
        }
    }
    if (inside) {
        const size_t p = (size_t)py * cam.W + px;
        image[3 * p] = fmaf(T, cam.bg[0], C0);
        image[3 * p + 1] = fmaf(T, cam.bg[1], C1);
        image[3 * p + 2] = fmaf(T, cam.bg[2], C2);
        if (final_T) final_T[p] = T;
        if (n_contrib) n_contrib[p] = count;
    }
}

cudaError_t launch_blend(const uint32_t* ranges, const uint32_t* values, const float4* rec,
                         CamParams cam, float* image, float* final_T, int32_t* n_contrib,
                         uint8_t* mark, cudaStream_t s, LaunchLog* log) {
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    if (n_tiles <= 0) return cudaSuccess;
    switch (cam.tile_size) {
        case 8: NVGS_LAUNCH(log, s, "k_blend<8>", k_blend<8><<<n_tiles, 64, 0, s>>>(ranges, values, rec, cam, image, final_T, n_contrib, mark)); break;
        case 16: NVGS_LAUNCH(log, s, "k_blend<16>", k_blend<16><<<n_tiles, 256, 0, s>>>(ranges, values, rec, cam, image, final_T, n_contrib, mark)); break;
        case 32: NVGS_LAUNCH(log, s, "k_blend<32>", k_blend<32><<<n_tiles, 1024, 0, s>>>(ranges, values, rec, cam, image, final_T, n_contrib, mark)); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_mark_labels(const uint2* __restrict__ surv, uint32_t n,
                                                     const uint8_t* __restrict__ mark,
                                                     uint8_t* __restrict__ labels_row) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && mark[i]) labels_row[surv[i].y] = 1;
}

cudaError_t launch_mark_labels(const uint2* surv, uint32_t n_surv, const uint8_t* mark,
                               uint8_t* labels_row, cudaStream_t s, LaunchLog* log) {
    if (n_surv == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_mark_labels", k_mark_labels<<<(n_surv + 255) / 256, 256, 0, s>>>(surv, n_surv, mark, labels_row));
    return cudaGetLastError();
}

}  // namespace nvgs
