// S5 (first and last parts): tile binning and tile ranges (NVGS Sec. 3.3 -> 3DGS tiled pipeline).
//
// Binning writes one (key, value) pair per (survivor, covered tile) at the survivor's exclusive
// prefix of tile counts, so pairs appear in survivor order (instance-major) before the sort.
// key = tile << depth_bits | (depth bits - minimum depth bits): camera-space depth is positive,
// so its IEEE bit pattern orders like the value and only the span of this frame's depths needs
// key bits.  A stable sort of these keys gives every tile its Gaussians front to back, ties in
// instance-then-Gaussian order.
#include "nvgs_internal.cuh"

namespace nvgs {

__global__ void __launch_bounds__(256) k_duplicate(const int4* __restrict__ rects,
                                                   const float4* __restrict__ rec,
                                                   const uint32_t* __restrict__ offsets, uint32_t n,
                                                   int tiles_x, int depth_bits,
                                                   const uint32_t* __restrict__ depth_minmax,
                                                   unsigned long long* __restrict__ keys,
                                                   uint32_t* __restrict__ values) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 r = rects[i];
    if (r.x > r.z || r.y > r.w) return;
    const uint32_t dk = __float_as_uint(rec[3 * (size_t)i + 1].z) - depth_minmax[0];
    uint32_t o = offsets[i];
    for (int ty = r.y; ty <= r.w; ty++)
        for (int tx = r.x; tx <= r.z; tx++) {
            keys[o] = ((unsigned long long)(ty * tiles_x + tx) << depth_bits) | dk;
            values[o] = i;
            o++;
        }
}

cudaError_t launch_duplicate(const int4* rects, const float4* rec, const uint32_t* offsets,
                             uint32_t n, int tiles_x, int depth_bits, const uint32_t* depth_minmax,
                             unsigned long long* keys, uint32_t* values, cudaStream_t s,
                             LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_duplicate", k_duplicate<<<(n + 255) / 256, 256, 0, s>>>(rects, rec, offsets, n, tiles_x, depth_bits, depth_minmax, keys, values));
    return cudaGetLastError();
}

// ranges[2t] / ranges[2t+1] = first / one-past-last index of tile t in the sorted keys.
// Tiles without pairs keep the zeros the caller wrote.
__global__ void __launch_bounds__(256) k_tile_ranges(const unsigned long long* __restrict__ keys,
                                                     uint32_t n, int depth_bits,
                                                     uint32_t* __restrict__ ranges) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = (uint32_t)(keys[i] >> depth_bits);
    if (i == 0 || (uint32_t)(keys[i - 1] >> depth_bits) != t) ranges[2 * t] = i;
    if (i == n - 1 || (uint32_t)(keys[i + 1] >> depth_bits) != t) ranges[2 * t + 1] = i + 1;
}

cudaError_t launch_tile_ranges(const unsigned long long* keys, uint32_t n, int depth_bits,
                               uint32_t* ranges, cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_tile_ranges", k_tile_ranges<<<(n + 255) / 256, 256, 0, s>>>(keys, n, depth_bits, ranges));
    return cudaGetLastError();
}

}  // namespace nvgs
