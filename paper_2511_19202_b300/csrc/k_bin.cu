// S5 around the sorts: binning and tile ranges (NVGS Sec. 3.3 -> 3DGS tiled pipeline).
//
// The (tile, depth) order of the pairs is produced by two stable radix sorts instead of one
// sort of 64-bit (tile << depth | depth) keys:
//   1. the survivors are sorted by depth (32-bit IEEE pattern of the positive camera-space z),
//      stably, so equal depths keep the survivor order (instance-major, Gaussian-minor);
//   2. k_duplicate walks the survivors in that order and writes one (tile id, survivor) pair per
//      covered tile at the survivor's prefix of tile counts (also taken in depth order);
//   3. the pairs are sorted stably by tile id alone.
// Inside every tile the pairs then come front to back with ties in survivor order, exactly the
// order of a stable sort on (tile, depth) -- at 32-bit keys and two tile passes instead of five
// 64-bit passes over the pairs.
#include "nvgs_internal.cuh"

namespace nvgs {

__global__ void __launch_bounds__(256) k_gather_counts(const uint32_t* __restrict__ order,
                                                       const uint32_t* __restrict__ counts, uint32_t n,
                                                       uint32_t* __restrict__ counts_sorted) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) counts_sorted[k] = counts[order[k]];
}

cudaError_t launch_gather_counts(const uint32_t* order, const uint32_t* counts, uint32_t n,
                                 uint32_t* counts_sorted, cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_gather_counts", k_gather_counts<<<(n + 255) / 256, 256, 0, s>>>(order, counts, n, counts_sorted));
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_duplicate(const uint32_t* __restrict__ order,
                                                   const int4* __restrict__ rects,
                                                   const uint32_t* __restrict__ offsets, uint32_t n,
                                                   int tiles_x, uint32_t* __restrict__ keys,
                                                   uint32_t* __restrict__ values) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t i = order[k];
    const int4 r = rects[i];
    if (r.x > r.z || r.y > r.w) return;
    uint32_t o = offsets[k];
    for (int ty = r.y; ty <= r.w; ty++)
        for (int tx = r.x; tx <= r.z; tx++) {
            keys[o] = (uint32_t)(ty * tiles_x + tx);
            values[o] = i;
            o++;
        }
}

cudaError_t launch_duplicate(const uint32_t* order, const int4* rects, const uint32_t* offsets,
                             uint32_t n, int tiles_x, uint32_t* keys, uint32_t* values,
                             cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_duplicate", k_duplicate<<<(n + 255) / 256, 256, 0, s>>>(order, rects, offsets, n, tiles_x, keys, values));
    return cudaGetLastError();
}

// ranges[2t] / ranges[2t+1] = first / one-past-last index of tile t in the sorted keys: one
// thread per tile, two binary searches (lower bounds of t and t + 1) instead of a pass over the
// pairs.
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&a[mid]) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ keys, uint32_t n,
                                                     uint32_t n_tiles, uint32_t* __restrict__ ranges) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    ranges[2 * t] = lower_bound_u32(keys, n, t);
    ranges[2 * t + 1] = lower_bound_u32(keys, n, t + 1);
}

cudaError_t launch_tile_ranges(const uint32_t* keys, uint32_t n, uint32_t n_tiles, uint32_t* ranges,
                               cudaStream_t s, LaunchLog* log) {
    if (n_tiles == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_tile_ranges", k_tile_ranges<<<(n_tiles + 255) / 256, 256, 0, s>>>(keys, n, n_tiles, ranges));
    return cudaGetLastError();
}

}  // namespace nvgs
