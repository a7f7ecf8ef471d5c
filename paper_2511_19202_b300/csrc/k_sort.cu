// Device-wide exclusive scan and the stable LSD radix sort of S5 (NVGS Sec. 3.3 -> 3DGS sorts
// (tile, depth) keys).  Both are reduce-then-scan designs: no CTA ever waits on another, so
// there is no inter-CTA spin of any kind.
//
// Radix sort, per digit pass (8 bits by default, 1..8 selectable) over tiles of 4096 pairs
// (256 threads x 16):
//   1. k_rs_hist:        per-tile digit histogram, stored digit-major: hist[d * n_tiles + tile]
//   2. k_rs_digit_scan:  one CTA per digit scans its row in place (start of every (digit, tile)
//                        bucket among that digit's buckets) and writes the digit's total; the
//                        scatter adds the exclusive prefix of the 256 totals
//   3. k_rs_scatter: stable rank of every pair inside its tile (digit peers from eight warp
//      ballots + per-warp running digit counters, each warp owning a contiguous 512-pair slice),
//      a local counting sort in shared memory, then runs of equal digits written to consecutive
//      global addresses.
#include <algorithm>

#include "nvgs_internal.cuh"

namespace nvgs {

// ================================================================== exclusive scan (uint32)
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t* s_warp,
                                                             uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < 8 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < 8) s_warp[8 + lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t warp_excl = warp ? s_warp[8 + warp - 1] : 0u;
    if (total) *total = s_warp[15];
    return warp_excl + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              uint64_t n, const uint32_t* __restrict__ n_dev,
                                                              uint32_t* __restrict__ sums) {
    if (n_dev) n = min(n, (uint64_t)*n_dev);   // elements past the device count read as 0
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        uint64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t w[8];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < 8; k++) t += w[k];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const uint32_t* __restrict__ in,
                                                            uint32_t* __restrict__ out, uint64_t n,
                                                            const uint32_t* __restrict__ n_dev,
                                                            const uint32_t* __restrict__ offsets,
                                                            uint32_t* __restrict__ total) {
    __shared__ uint32_t s[kScanTile + kScanTile / 32];
    __shared__ uint32_t s_warp[16];
    const uint64_t n_out = n;   // outputs are written over the whole (capacity) range
    if (n_dev) n = min(n, (uint64_t)*n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    // striped, coalesced load; padded index p + p/32 avoids bank conflicts on the blocked read
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int p = j * kScanThreads + threadIdx.x;
        const uint64_t i = base + p;
        s[p + (p >> 5)] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int p = threadIdx.x * kScanItems + j;
        v[j] = s[p + (p >> 5)];
        sum += v[j];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan_256(sum, s_warp, &tot);
    if (offsets) run += offsets[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int p = threadIdx.x * kScanItems + j;
        s[p + (p >> 5)] = run;
        run += v[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int p = j * kScanThreads + threadIdx.x;
        const uint64_t i = base + p;
        if (i < n_out) out[i] = s[p + (p >> 5)];
    }
    if (total && threadIdx.x == 0) *total = tot;
}

static uint64_t scan_levels_bytes(uint64_t n) {
    uint64_t bytes = 0;
    while (n > (uint64_t)kScanTile) {
        uint64_t nb = (n + kScanTile - 1) / kScanTile;
        bytes += 2 * ((nb * 4 + 255) / 256 * 256);
        n = nb;
    }
    return bytes;
}

size_t scan_scratch_bytes(uint64_t n) { return (size_t)scan_levels_bytes(n) + 256; }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* total,
                               void* scratch, cudaStream_t s, LaunchLog* log, const uint32_t* n_dev) {
    if (n == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return cudaSuccess;
    }
    if (n <= (uint64_t)kScanTile) {
        NVGS_LAUNCH(log, s, "k_scan_tile", k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, n_dev, nullptr, total));
        return cudaGetLastError();
    }
    const uint64_t nb = (n + kScanTile - 1) / kScanTile;
    const uint64_t seg = (nb * 4 + 255) / 256 * 256;
    uint32_t* sums = (uint32_t*)scratch;
    uint32_t* sums_scan = (uint32_t*)((char*)scratch + seg);
    void* rest = (char*)scratch + 2 * seg;
    NVGS_LAUNCH(log, s, "k_scan_reduce", k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, n_dev, sums));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan_u32(sums, sums_scan, nb, total, rest, s, log);
    if (e != cudaSuccess) return e;
    NVGS_LAUNCH(log, s, "k_scan_tile", k_scan_tile<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, n_dev, sums_scan, nullptr));
    return cudaGetLastError();
}

// ================================================================== radix sort
constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096
constexpr int kRsWarps = kRsThreads / 32;       // 8

// Lanes of the warp whose 8-bit digit equals this lane's, from one ballot per bit (cheaper than
// a warp match instruction); lanes with ok = false match only themselves.  `vary` (the same in
// every thread) has a bit set for every digit bit that differs between some keys of the pass: a
// bit that every key shares cannot separate two of them, so its ballot is skipped (the ranking is
// bound by the integer ALU pipe, and e.g. 13-bit tile ids leave three bits of their second digit
// constant).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool ok, uint32_t vary) {
    uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < 8; b++) {
        if (vary & (1u << b)) {
            const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
    }
    return ok ? peers : 1u << (threadIdx.x & 31);
}

template <typename K>
constexpr int rs_smem_bytes() { return kRsWarps * 256 * 4 + kRsTile * (int)sizeof(K) + kRsTile * 4 + 2 * 256 * 4; }

// One CTA per tile; tiles at or past the (device-side) element count write zero counts, so the
// digit-major layout always spans n_tiles (the capacity's tile count).
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K* __restrict__ keys, uint64_t n,
                                                        const uint32_t* __restrict__ n_dev, int shift,
                                                        uint32_t mask, uint32_t n_tiles,
                                                        uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kRsWarps][256];
    if (n_dev) n = min(n, (uint64_t)*n_dev);
    const int warp = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x;
    const uint64_t base = (uint64_t)tile * kRsTile;
    if (base >= n) {
        if (threadIdx.x < 256) hist[(uint64_t)threadIdx.x * n_tiles + tile] = 0u;
        return;
    }
    for (int k = threadIdx.x; k < kRsWarps * 256; k += kRsThreads) (&h[0][0])[k] = 0u;
    __syncthreads();
    const bool vec = sizeof(K) <= 4 && base + kRsTile <= n && ((uintptr_t)(keys + base) & 15u) == 0;
    bool counted = false;
    if constexpr (sizeof(K) == 2) {
        if (vec) {
            // a full tile of 16-bit keys: two 16-byte loads (eight keys each) per thread
            const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
            uint4 v[kRsItems / 8];
#pragma unroll
            for (int j = 0; j < kRsItems / 8; j++) v[j] = k4[j * kRsThreads + threadIdx.x];
#pragma unroll
            for (int j = 0; j < kRsItems / 8; j++) {
                const uint32_t w[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    atomicAdd(&h[warp][((w[q] & 0xffffu) >> shift) & mask], 1u);
                    atomicAdd(&h[warp][((w[q] >> 16) >> shift) & mask], 1u);
                }
            }
            counted = true;
        }
    }
    if constexpr (sizeof(K) == 4) {
        if (vec) {
            // a full tile of 32-bit keys: four 16-byte loads per thread, all in flight at once
            const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
            uint4 v[kRsItems / 4];
#pragma unroll
            for (int j = 0; j < kRsItems / 4; j++) v[j] = k4[j * kRsThreads + threadIdx.x];
#pragma unroll
            for (int j = 0; j < kRsItems / 4; j++) {
                atomicAdd(&h[warp][(v[j].x >> shift) & mask], 1u);
                atomicAdd(&h[warp][(v[j].y >> shift) & mask], 1u);
                atomicAdd(&h[warp][(v[j].z >> shift) & mask], 1u);
                atomicAdd(&h[warp][(v[j].w >> shift) & mask], 1u);
            }
            counted = true;
        }
    }
    if (!counted) {
#pragma unroll 4
        for (int j = 0; j < kRsItems; j++) {
            const uint64_t i = base + (uint64_t)j * kRsThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[warp][(uint32_t)(keys[i] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; w++) sum += h[w][threadIdx.x];
        hist[(uint64_t)threadIdx.x * n_tiles + tile] = sum;
    }
}

// Row d of the digit-major histogram (n_tiles counts) -> its exclusive prefix, in place; the row's
// total to totals[d].  One CTA of 1024 threads per digit, 4096 counts per step (four per thread,
// consecutive) with a running carry: a 1080p frame's 17k tiles of pairs take five steps.
constexpr int kDigitScanThreads = 1024;
__global__ void __launch_bounds__(kDigitScanThreads) k_rs_digit_scan(uint32_t* __restrict__ hist, uint32_t n_tiles,
                                                                     uint32_t* __restrict__ totals) {
    __shared__ uint32_t s_warp[2][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* row = hist + (uint64_t)blockIdx.x * n_tiles;
    uint32_t carry = 0;
    int par = 0;
    for (uint32_t base = 0; base < n_tiles; base += 4 * kDigitScanThreads, par ^= 1) {
        const uint32_t i0 = base + 4 * threadIdx.x;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = i0 + k < n_tiles ? row[i0 + k] : 0u;
        const uint32_t sum = v[0] + v[1] + v[2] + v[3];
        // inclusive scan within the warp, then over the 32 warp totals (slots alternate between
        // steps so that one barrier a step suffices)
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_warp[par][warp] = x;
        __syncthreads();
        uint32_t wt = s_warp[par][lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wt, o);
            if (lane >= o) wt += t;
        }
        const uint32_t warp_excl = __shfl_sync(0xffffffffu, wt, (warp + 31) & 31) * (warp > 0);
        const uint32_t total = __shfl_sync(0xffffffffu, wt, 31);
        uint32_t run = carry + warp_excl + x - sum;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (i0 + k < n_tiles) row[i0 + k] = run;
            run += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Registers hold the tile's keys and one packed (digit << 16 | rank-in-warp) word per item;
// values are read only when they are placed in shared memory, so four CTAs fit on an SM
// (smaller, more numerous CTAs overlap their load, rank and write phases better).
template <typename K>
__global__ void __launch_bounds__(kRsThreads, sizeof(K) <= 4 ? 4 : 2) k_rs_scatter(
    const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, K* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, uint64_t n, const uint32_t* __restrict__ n_dev, int shift,
    uint32_t mask, uint32_t n_tiles, const uint32_t* __restrict__ hist_scan,
    const uint32_t* __restrict__ totals) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* cnt = (uint32_t*)smem;                                   // [8 warps][256]
    K* s_keys = (K*)(smem + kRsWarps * 256 * 4);
    uint32_t* s_vals = (uint32_t*)(smem + kRsWarps * 256 * 4 + kRsTile * sizeof(K));
    uint32_t* d_local = s_vals + kRsTile;                              // [256] tile-local start
    uint32_t* d_global = d_local + 256;                                // [256] global start
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    if (n_dev) n = min(n, (uint64_t)*n_dev);
    const uint32_t tile = blockIdx.x;   // one CTA per tile; CTAs past the device-side count exit
    if ((uint64_t)tile * kRsTile >= n) return;
    // this thread's digit: the pass's total and this tile's bucket start, loaded now so that
    // their latency hides behind the ranking
    const uint32_t my_total = totals[threadIdx.x];
    const uint32_t my_hs = hist_scan[(uint64_t)threadIdx.x * n_tiles + tile];
    // the digit bits that differ between keys of the pass: OR of the present digits (a pass total
    // above 0) and OR of their complements, per warp here and over the CTA after the barrier
    // (d_global is free until the bucket starts are written)
    {
        const uint32_t any1 = __reduce_or_sync(0xffffffffu, my_total ? threadIdx.x : 0u);
        const uint32_t any0 = __reduce_or_sync(0xffffffffu, my_total ? (~threadIdx.x & 255u) : 0u);
        if (lane == 0) { d_global[warp] = any1; d_global[kRsWarps + warp] = any0; }
    }
    for (int k = threadIdx.x; k < kRsWarps * 256; k += kRsThreads) cnt[k] = 0u;
    __syncthreads();
    uint32_t vm;
    {
        uint32_t any1 = 0u, any0 = 0u;
#pragma unroll
        for (int w = 0; w < kRsWarps; w++) { any1 |= d_global[w]; any0 |= d_global[kRsWarps + w]; }
        vm = any1 & any0;
    }

    const uint64_t base = (uint64_t)tile * kRsTile;
    const uint64_t tile_n64 = n - base < (uint64_t)kRsTile ? n - base : (uint64_t)kRsTile;
    const int tile_n = (int)tile_n64;
    K key[kRsItems];
    uint32_t pk[kRsItems];   // digit << 16 | rank among the warp's earlier items of that digit
    // each warp ranks its own contiguous slice [warp*512, warp*512 + 512) in order
#pragma unroll
    for (int r = 0; r < kRsItems; r++) {
        const int p = warp * (kRsItems * 32) + r * 32 + lane;
        key[r] = p < tile_n ? keys_in[base + p] : (K)0;
    }
    {   // the values are read only after the ranking: start their 128-byte lines towards L2 now
        const int p = warp * (kRsItems * 32) + lane * 32;
        if (lane < kRsItems && p < tile_n)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(vals_in + base + p));
    }
#pragma unroll
    for (int r = 0; r < kRsItems; r++) {
        const int p = warp * (kRsItems * 32) + r * 32 + lane;
        const bool ok = p < tile_n;
        const uint32_t d = ok ? ((uint32_t)(key[r] >> shift) & mask) : 256u + lane;  // unmatched
        // the lowest lane of each digit group reserves the group's slots with one shared-memory
        // atomic; a warp's atomics on a counter complete in program order, so the ranks keep the
        // input order (stable) without a load / store round trip between the items
        const uint32_t peers = digit_peers(d & 255u, ok, vm);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0u;
        if (ok && leader == lane) before = atomicAdd(&cnt[warp * 256 + d], (uint32_t)__popc(peers));
        before = __shfl_sync(0xffffffffu, before, leader);
        pk[r] = (d << 16) | (before + __popc(peers & lt));
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then over digits (tile-local bucket starts)
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; w++) {
            const uint32_t c = cnt[w * 256 + d];
            cnt[w * 256 + d] = run;
            run += c;
        }
        d_local[d] = run;        // this tile's digit total for now
        d_global[d] = my_total;   // the pass's digit total for now
    }
    __syncthreads();
    // warps 0 and 1: exclusive scans of the tile's and of the pass's 256 digit totals
    if (threadIdx.x < 64) {
        uint32_t* a = threadIdx.x < 32 ? d_local : d_global;
        uint32_t v[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) { v[k] = a[lane * 8 + k]; s += v[k]; }
        uint32_t x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        uint32_t run = x - s;
#pragma unroll
        for (int k = 0; k < 8; k++) { a[lane * 8 + k] = run; run += v[k]; }
    }
    __syncthreads();
    // global start of this tile's bucket of digit d: digit d's start + its count in earlier tiles
    if (threadIdx.x < 256) d_global[threadIdx.x] += my_hs;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsItems; r++) {
        const int p = warp * (kRsItems * 32) + r * 32 + lane;
        if (p < tile_n) {
            const uint32_t d = pk[r] >> 16;
            const uint32_t lp = d_local[d] + cnt[warp * 256 + d] + (pk[r] & 0xffffu);
            s_keys[lp] = key[r];
            s_vals[lp] = vals_in[base + p];
        }
    }
    __syncthreads();
    // the tile is now sorted by digit in shared memory; stream it out in order
#pragma unroll 4
    for (int j = 0; j < kRsItems; j++) {
        const int p = j * kRsThreads + threadIdx.x;
        if (p < tile_n) {
            const K k = s_keys[p];
            const uint32_t d = (uint32_t)(k >> shift) & mask;
            const uint64_t g = (uint64_t)d_global[d] + (uint32_t)(p - d_local[d]);
            keys_out[g] = k;
            vals_out[g] = s_vals[p];
        }
    }
}

size_t radix_scratch_bytes(uint64_t n) {
    const uint64_t tiles = (n + kRsTile - 1) / kRsTile;
    const uint64_t h = (256 * tiles * 4 + 255) / 256 * 256;
    return (size_t)(h + 256 * 4);
}

// n is the element count, or with n_dev the capacity (the count then lives on the device and
// every kernel reads it; nothing here waits for it).
// Digits are `digit_bits` wide (1..8); the last pass takes only the key bits that remain, so bits
// at or above key_bits never influence the order.
template <typename K>
static cudaError_t radix_sort_impl(K* keys, uint32_t* values, K* keys_alt, uint32_t* values_alt,
                                   uint64_t n, int key_bits, void* scratch, cudaStream_t s,
                                   LaunchLog* log, int* passes_out, int copy_back, int* result_in_alt,
                                   const uint32_t* n_dev, int digit_bits = 8) {
    if (digit_bits < 1 || digit_bits > 8) return cudaErrorInvalidValue;
    int passes = key_bits <= 0 ? 0 : (key_bits + digit_bits - 1) / digit_bits;
    if (n <= 1 && !n_dev) passes = 0;
    if (n == 0) passes = 0;
    if (passes_out) *passes_out = passes;
    if (result_in_alt) *result_in_alt = 0;
    if (passes == 0) return cudaSuccess;
    static std::atomic<uint64_t> attr_done{0};
    {
        cudaError_t e = once_per_device(attr_done, [] {
            return cudaFuncSetAttribute(k_rs_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             rs_smem_bytes<K>());
        });
        if (e != cudaSuccess) return e;
    }
    const uint64_t tiles = (n + kRsTile - 1) / kRsTile;
    const uint64_t h = (256 * tiles * 4 + 255) / 256 * 256;
    uint32_t* hist = (uint32_t*)scratch;
    uint32_t* totals = (uint32_t*)((char*)scratch + h);
    K* kin = keys;
    uint32_t* vin = values;
    K* kout = keys_alt;
    uint32_t* vout = values_alt;
    const char* hname = sizeof(K) == 8 ? "k_rs_hist<u64>" : sizeof(K) == 4 ? "k_rs_hist<u32>" : "k_rs_hist<u16>";
    const char* sname = sizeof(K) == 8 ? "k_rs_scatter<u64>" : sizeof(K) == 4 ? "k_rs_scatter<u32>" : "k_rs_scatter<u16>";
    // one CTA per tile; with a device-side count the CTAs past it exit at once (the histogram
    // ones after writing zero counts)
    const unsigned hgrid = (unsigned)tiles;
    const unsigned sgrid = (unsigned)tiles;
    for (int p = 0; p < passes; p++) {
        const int shift = digit_bits * p;
        const int width = std::min(digit_bits, key_bits - shift);
        const uint32_t mask = (1u << width) - 1u;
        NVGS_LAUNCH(log, s, hname, k_rs_hist<K><<<hgrid, kRsThreads, 0, s>>>(kin, n, n_dev, shift, mask, (uint32_t)tiles, hist));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        NVGS_LAUNCH(log, s, "k_rs_digit_scan", k_rs_digit_scan<<<256, kDigitScanThreads, 0, s>>>(hist, (uint32_t)tiles, totals));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        NVGS_LAUNCH(log, s, sname, k_rs_scatter<K><<<sgrid, kRsThreads, rs_smem_bytes<K>(), s>>>(kin, vin, kout, vout, n, n_dev, shift, mask, (uint32_t)tiles, hist, totals));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        K* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys) {  // odd number of passes: the result sits in the alternate buffers
        if (!copy_back) {
            if (result_in_alt) *result_in_alt = 1;
            return cudaSuccess;
        }
        cudaError_t e = cudaMemcpyAsync(keys, kin, n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(values, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t radix_sort_pairs(unsigned long long* keys, uint32_t* values,
                             unsigned long long* keys_alt, uint32_t* values_alt, uint64_t n,
                             int key_bits, void* scratch, cudaStream_t s, LaunchLog* log,
                             int* passes_out, int copy_back, int* result_in_alt) {
    return radix_sort_impl<unsigned long long>(keys, values, keys_alt, values_alt, n, key_bits, scratch,
                                               s, log, passes_out, copy_back, result_in_alt, nullptr);
}

cudaError_t radix_sort_pairs_u32(uint32_t* keys, uint32_t* values, uint32_t* keys_alt,
                                 uint32_t* values_alt, uint64_t n, int key_bits, void* scratch,
                                 cudaStream_t s, LaunchLog* log, int* passes_out, int copy_back,
                                 int* result_in_alt, const uint32_t* n_dev, int digit_bits) {
    return radix_sort_impl<uint32_t>(keys, values, keys_alt, values_alt, n, key_bits, scratch, s, log,
                                     passes_out, copy_back, result_in_alt, n_dev, digit_bits);
}

cudaError_t radix_sort_pairs_u16(uint16_t* keys, uint32_t* values, uint16_t* keys_alt,
                                 uint32_t* values_alt, uint64_t n, int key_bits, void* scratch,
                                 cudaStream_t s, LaunchLog* log, int* passes_out, int copy_back,
                                 int* result_in_alt, const uint32_t* n_dev, int digit_bits) {
    if (key_bits > 16) return cudaErrorInvalidValue;
    return radix_sort_impl<uint16_t>(keys, values, keys_alt, values_alt, n, key_bits, scratch, s, log,
                                     passes_out, copy_back, result_in_alt, n_dev, digit_bits);
}

}  // namespace nvgs
