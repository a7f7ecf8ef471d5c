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
// the output starting at the first survivor's offset.  The warp walks (survivor, tile row) units
// 32 at a time: each lane finds its unit's survivor by a binary search over the lanes' row
// prefix sums and computes the row's kept tile span once (as the projection counted it); a
// second walk over the batch's pairs writes them, each lane finding its unit by a binary search
// over the span prefix -- balanced whatever the rectangle sizes, and coalesced.  The survivors'
// ellipse terms (computed once per survivor) and the batch's units are staged in shared memory
// rather than shuffled field by field.  (Letting each lane write a small rectangle's pairs itself,
// without the walk, measured slower: its divergent loops leave most lanes idle.)
constexpr int kDupWarps = 8;

__device__ __forceinline__ int warp_owner(uint32_t pre, uint32_t c) {
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint32_t pj = __shfl_sync(0xffffffffu, pre, j + step);
        if (pj <= c) j += step;
    }
    return j;
}

// kMV (multi-view batches): the rect's w carries the survivor's view in its high 16 bits, and the
// pair key is that view's tile_base plus its local tile id.  KT: the key type (16-bit tile ids
// when the frame or batch has at most 65536 tiles).
template <bool kMV, typename KT>
__global__ void __launch_bounds__(kDupWarps * 32) k_duplicate(const uint32_t* __restrict__ order,
                                                              const float4* __restrict__ rec,
                                                              const uint32_t* __restrict__ offsets, uint32_t n,
                                                              const uint32_t* __restrict__ n_dev,
                                                              const CamParams* __restrict__ camp,
                                                              const uint32_t* __restrict__ n_pairs,
                                                              uint32_t pair_cap, uint32_t* __restrict__ overflow,
                                                              KT* __restrict__ keys,
                                                              uint32_t* __restrict__ values) {
    // the warp's survivors: ellipse (u, v, cb, rcc), (det, ck, ymax or -1 for a whole rectangle
    // row, yr), rectangle (x0, x1, y0 - row prefix, index), its view's (tiles per row, first
    // tile); and a batch's units (first key - span prefix, index)
    __shared__ float4 s_e0[kDupWarps][32], s_e1[kDupWarps][32];
    __shared__ int4 s_r[kDupWarps][32];
    __shared__ int2 s_x[kMV ? kDupWarps : 1][32];
    __shared__ uint2 s_u[kDupWarps][32];
    const CamParams cam = *camp;
    const int ts = cam.tile_size;
    const float rts = 1.0f / (float)ts;
    if (n_dev) n = min(n, *n_dev);
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const uint32_t n_pairs_all = *n_pairs;
    const uint32_t limit = min(n_pairs_all, pair_cap);
    if (n_pairs_all > pair_cap && blockIdx.x == 0 && threadIdx.x == 0 && overflow) *overflow = 1u;
    const uint32_t n_warps = (blockDim.x * gridDim.x) >> 5;
    for (uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; warp * 32u < n; warp += n_warps) {
        const uint32_t k = warp * 32u + lane;
        // this lane's survivor
        uint32_t i = 0, rows = 0, off = 0;
        int4 r = make_int4(0, 0, -1, -1);
        int tiles_x = cam.tiles_x, tile_base = 0;
        bool test = false;
        SplatEllipse el{};
        if (k < n) {
            i = order[k];
            off = offsets[k];
            r = rec_rect(rec, i);
            if (kMV) {
                const CamParams& cv = camp[r.w >> 16];
                tiles_x = cv.tiles_x;
                tile_base = cv.tile_base;
                r.w &= 0xffff;
            }
            if (r.x <= r.z && r.y <= r.w) {
                rows = (uint32_t)(r.w - r.y + 1);
                test = (r.z - r.x + 1) * (int)rows > 1;
                if (test) {
                    const float4 a = __ldg(&rec[kRecF4 * (size_t)i]);
                    const float4 b = __ldg(&rec[kRecF4 * (size_t)i + 1]);
                    el = splat_ellipse(a.x, a.y, a.z, a.w, b.x, b.z, -2.0f * b.w);
                }
            }
        }
        uint32_t row_pre;
        const uint32_t n_units = warp_prefix(rows, row_pre);
        __syncwarp();   // the previous iteration's walk has read the staging arrays
        s_e0[wi][lane] = make_float4(el.u, el.v, el.cb, el.rcc);
        s_e1[wi][lane] = make_float4(el.det, el.ck, test ? el.ymax : -1.0f, el.yr);
        s_r[wi][lane] = make_int4(r.x, r.z, r.y - (int)row_pre, (int)i);
        if (kMV) s_x[wi][lane] = make_int2(tiles_x, tile_base);
        __syncwarp();
        uint32_t out = __shfl_sync(0xffffffffu, off, 0);
        for (uint32_t c0 = 0; c0 < n_units; c0 += 32) {
            // ---- unit (survivor j, tile row ty): its kept span [t0, t1]
            const uint32_t c = c0 + lane;
            const int j = warp_owner(row_pre, c);
            const int4 sr = s_r[wi][j];
            int t0 = 1, t1 = 0, row0 = 0;
            if (c < n_units) {
                const int ty = sr.z + (int)c;
                if (kMV) {
                    const int2 sx = s_x[kMV ? wi : 0][j];
                    row0 = sx.y + ty * sx.x;
                } else {
                    row0 = ty * cam.tiles_x;
                }
                const float4 e1 = s_e1[wi][j];
                if (e1.z >= 0.0f) {
                    const float4 e0 = s_e0[wi][j];
                    SplatEllipse ej;
                    ej.u = e0.x; ej.v = e0.y; ej.cb = e0.z; ej.rcc = e0.w;
                    ej.det = e1.x; ej.ck = e1.y; ej.ymax = e1.z; ej.yr = e1.w;
                    row_tile_span(ej, ty, ts, rts, t0, t1);
                    t0 = max(t0, sr.x);
                    t1 = min(t1, sr.y);
                } else {
                    t0 = sr.x; t1 = sr.y;
                }
            }
            const uint32_t cnt = t0 <= t1 ? (uint32_t)(t1 - t0 + 1) : 0u;
            uint32_t cnt_pre;
            const uint32_t batch = warp_prefix(cnt, cnt_pre);
            __syncwarp();   // the previous batch's pairs have read s_u
            s_u[wi][lane] = make_uint2((uint32_t)(row0 + t0) - cnt_pre, (uint32_t)sr.w);
            __syncwarp();
            // ---- the batch's pairs, 32 at a time
            for (uint32_t p0 = 0; p0 < batch; p0 += 32) {
                const uint32_t p = p0 + lane;
                const int q = warp_owner(cnt_pre, p);
                const uint2 uq = s_u[wi][q];
                const uint32_t pos = out + p;
                if (p < batch && pos < limit) {
                    keys[pos] = (KT)(uq.x + p);
                    values[pos] = uq.y;
                }
            }
            out += batch;
        }
    }
}

cudaError_t launch_duplicate(const uint32_t* order, const float4* rec,
                             const uint32_t* offsets, uint32_t n, const uint32_t* n_dev,
                             const CamParams* cam_dev, const uint32_t* n_pairs, uint32_t pair_cap,
                             uint32_t* overflow, void* keys, int key_bytes, uint32_t* values, int num_sms,
                             cudaStream_t s, LaunchLog* log, int multi_view) {
    if (key_bytes != 2 && key_bytes != 4) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    // a grid-stride kernel with equal shares per CTA: exactly the CTAs that are resident at once
    // (a fraction of a second wave would run alone at the end)
    int dev = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<int> per_sm_cache[64];   // per device ordinal; 0 = not measured yet
    if (dev >= 0 && dev < 64) per_sm = per_sm_cache[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_duplicate<false, uint32_t>, kDupWarps * 32, 0);
        if (e != cudaSuccess) return e;
        per_sm = std::max(per_sm, 1);
        if (dev >= 0 && dev < 64) per_sm_cache[dev].store(per_sm, std::memory_order_relaxed);
    }
    const uint32_t warps = (n + 31) / 32;
    const uint32_t grid = std::min<uint32_t>((warps + kDupWarps - 1) / kDupWarps, (uint32_t)(num_sms * per_sm));
    uint16_t* k16 = static_cast<uint16_t*>(keys);
    uint32_t* k32 = static_cast<uint32_t*>(keys);
    if (multi_view && key_bytes == 2)
        NVGS_LAUNCH(log, s, "k_duplicate_views", k_duplicate<true, uint16_t><<<grid, kDupWarps * 32, 0, s>>>(order, rec, offsets, n, n_dev, cam_dev, n_pairs, pair_cap, overflow, k16, values));
    else if (multi_view)
        NVGS_LAUNCH(log, s, "k_duplicate_views", k_duplicate<true, uint32_t><<<grid, kDupWarps * 32, 0, s>>>(order, rec, offsets, n, n_dev, cam_dev, n_pairs, pair_cap, overflow, k32, values));
    else if (key_bytes == 2)
        NVGS_LAUNCH(log, s, "k_duplicate", k_duplicate<false, uint16_t><<<grid, kDupWarps * 32, 0, s>>>(order, rec, offsets, n, n_dev, cam_dev, n_pairs, pair_cap, overflow, k16, values));
    else
        NVGS_LAUNCH(log, s, "k_duplicate", k_duplicate<false, uint32_t><<<grid, kDupWarps * 32, 0, s>>>(order, rec, offsets, n, n_dev, cam_dev, n_pairs, pair_cap, overflow, k32, values));
    return cudaGetLastError();
}

// ranges[2t] / ranges[2t+1] = first / one-past-last index of tile t in the sorted keys: one
// thread per tile, two binary searches (lower bounds of t and t + 1) instead of a pass over the
// pairs.
template <typename KT>
__device__ __forceinline__ uint32_t lower_bound_key(const KT* __restrict__ a, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if ((uint32_t)__ldg(&a[mid]) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <typename KT>
__global__ void __launch_bounds__(256) k_tile_ranges(const KT* __restrict__ keys, uint32_t n,
                                                     const uint32_t* __restrict__ n_dev,
                                                     uint32_t n_tiles, uint32_t* __restrict__ ranges) {
    if (n_dev) n = min(n, *n_dev);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    ranges[2 * t] = lower_bound_key(keys, n, t);
    ranges[2 * t + 1] = lower_bound_key(keys, n, t + 1);
}

cudaError_t launch_tile_ranges(const void* keys, int key_bytes, uint32_t n, const uint32_t* n_dev,
                               uint32_t n_tiles, uint32_t* ranges, cudaStream_t s, LaunchLog* log) {
    if (n_tiles == 0) return cudaSuccess;
    if (key_bytes == 2)
        NVGS_LAUNCH(log, s, "k_tile_ranges", k_tile_ranges<uint16_t><<<(n_tiles + 255) / 256, 256, 0, s>>>(static_cast<const uint16_t*>(keys), n, n_dev, n_tiles, ranges));
    else if (key_bytes == 4)
        NVGS_LAUNCH(log, s, "k_tile_ranges", k_tile_ranges<uint32_t><<<(n_tiles + 255) / 256, 256, 0, s>>>(static_cast<const uint32_t*>(keys), n, n_dev, n_tiles, ranges));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace nvgs
