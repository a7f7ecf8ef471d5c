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
#include <algorithm>

#include "nvgs_internal.cuh"

namespace nvgs {

__global__ void __launch_bounds__(256) k_gather_counts(const uint32_t* __restrict__ order,
                                                       const uint32_t* __restrict__ counts, uint32_t n,
                                                       const uint32_t* __restrict__ n_dev,
                                                       uint32_t* __restrict__ counts_sorted) {
    if (n_dev) n = min(n, *n_dev);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        counts_sorted[k] = counts[order[k]];
}

cudaError_t launch_gather_counts(const uint32_t* order, const uint32_t* counts, uint32_t n,
                                 const uint32_t* n_dev, uint32_t* counts_sorted, int num_sms,
                                 cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    const uint32_t grid = std::min<uint32_t>((n + 255) / 256, (uint32_t)num_sms * 8);
    NVGS_LAUNCH(log, s, "k_gather_counts", k_gather_counts<<<grid, 256, 0, s>>>(order, counts, n, n_dev, counts_sorted));
    return cudaGetLastError();
}

// One warp per 32 consecutive survivors (depth order).  Their pairs form one contiguous run of
// the output starting at the first survivor's offset, so the warp walks the concatenation of the
// 32 tile rectangles 32 candidates at a time: each lane finds its candidate's survivor by a
// binary search over the lanes' rectangle prefix sums, tests the tile (as the projection counted
// it), and the passing candidates are written at the running offset plus their rank in the
// ballot -- balanced over the warp whatever the rectangle sizes, and coalesced.
__global__ void __launch_bounds__(256) k_duplicate(const uint32_t* __restrict__ order,
                                                   const int4* __restrict__ rects,
                                                   const float4* __restrict__ rec,
                                                   const uint32_t* __restrict__ offsets, uint32_t n,
                                                   const uint32_t* __restrict__ n_dev,
                                                   const CamParams* __restrict__ camp, const uint32_t* __restrict__ n_pairs,
                                                   uint32_t pair_cap, uint32_t* __restrict__ overflow,
                                                   uint32_t* __restrict__ keys,
                                                   uint32_t* __restrict__ values) {
    const CamParams cam = *camp;
    if (n_dev) n = min(n, *n_dev);
    const int lane = threadIdx.x & 31;
    const uint32_t n_pairs_all = *n_pairs;
    const uint32_t limit = min(n_pairs_all, pair_cap);
    if (n_pairs_all > pair_cap && blockIdx.x == 0 && threadIdx.x == 0 && overflow) *overflow = 1u;
    const uint32_t n_warps = (blockDim.x * gridDim.x) >> 5;
    for (uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; warp * 32u < n; warp += n_warps) {
        const uint32_t base = warp * 32u;
        const uint32_t k = base + lane;
        uint32_t i = 0;
        SplatTiles st{};
        st.w = 1;
        if (k < n) {
            i = order[k];
            const int4 r = rects[i];
            if (r.x <= r.z && r.y <= r.w) {
                st.w = (uint32_t)(r.z - r.x + 1);
                st.area = st.w * (uint32_t)(r.w - r.y + 1);
                st.rx = r.x; st.ry = r.y;
                st.test = st.area > 1u;
                if (st.test) {
                    const float4 a = rec[3 * (size_t)i];
                    const float4 b = rec[3 * (size_t)i + 1];
                    st.u = a.x; st.v = a.y; st.A = a.z; st.B = a.w; st.C = b.x; st.kk = -2.0f * b.w;
                    st.det = rec[3 * (size_t)i + 2].w;
                }
            }
        }
        const uint32_t total = warp_prefix(st.area, st.pre);
        uint32_t out = __shfl_sync(0xffffffffu, k < n ? offsets[k] : 0u, 0);
        for (uint32_t c0 = 0; c0 < total; c0 += 32) {
            int j, tx = 0, ty = 0;
            const bool pass = warp_tile_candidate(st, c0 + lane, total, cam, j, tx, ty);
            const uint32_t ij = __shfl_sync(0xffffffffu, i, j);
            const uint32_t bal = __ballot_sync(0xffffffffu, pass);
            if (pass) {
                const uint32_t pos = out + __popc(bal & ((1u << lane) - 1u));
                if (pos < limit) {
                    keys[pos] = (uint32_t)(ty * cam.tiles_x + tx);
                    values[pos] = ij;
                }
            }
            out += __popc(bal);
        }
    }
}

cudaError_t launch_duplicate(const uint32_t* order, const int4* rects, const float4* rec,
                             const uint32_t* offsets, uint32_t n, const uint32_t* n_dev,
                             const CamParams* cam_dev, const uint32_t* n_pairs, uint32_t pair_cap,
                             uint32_t* overflow, uint32_t* keys, uint32_t* values, int num_sms,
                             cudaStream_t s, LaunchLog* log) {
    if (n == 0) return cudaSuccess;
    const uint32_t warps = (n + 31) / 32;
    const uint32_t grid = std::min<uint32_t>((warps + 7) / 8, (uint32_t)num_sms * 8);
    NVGS_LAUNCH(log, s, "k_duplicate", k_duplicate<<<grid, 256, 0, s>>>(order, rects, rec, offsets, n, n_dev, cam_dev, n_pairs, pair_cap, overflow, keys, values));
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
                                                     const uint32_t* __restrict__ n_dev,
                                                     uint32_t n_tiles, uint32_t* __restrict__ ranges) {
    if (n_dev) n = min(n, *n_dev);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    ranges[2 * t] = lower_bound_u32(keys, n, t);
    ranges[2 * t + 1] = lower_bound_u32(keys, n, t + 1);
}

cudaError_t launch_tile_ranges(const uint32_t* keys, uint32_t n, const uint32_t* n_dev, uint32_t n_tiles,
                               uint32_t* ranges, cudaStream_t s, LaunchLog* log) {
    if (n_tiles == 0) return cudaSuccess;
    NVGS_LAUNCH(log, s, "k_tile_ranges", k_tile_ranges<<<(n_tiles + 255) / 256, 256, 0, s>>>(keys, n, n_dev, n_tiles, ranges));
    return cudaGetLastError();
}

}  // namespace nvgs
