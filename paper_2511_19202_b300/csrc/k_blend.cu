// S6: front-to-back alpha compositing per tile (NVGS Sec. 4.1 blending rules on the 3DGS tiled
// rasteriser).
//
// One CTA per TS x TS tile, one thread per pixel.  The tile's Gaussians (a contiguous range of
// the sorted pairs) are staged through shared memory in batches of up to 256 records, gathered by
// survivor index; every thread then walks the batch for its pixel:
//   power = -1/2 (A dx^2 + C dy^2) - B dx dy      (conic [[A, B], [B, C]], pixel centre - mean)
//   skip if power > 0;  alpha = min(alpha_max, opacity e^power);  skip if alpha < alpha_min;
//   stop (without blending) if T (1 - alpha) < t_stop;  C += alpha T rgb;  T *= 1 - alpha.
// The walk takes two fragments per step: the batch is staged as pairs of records side by side, so
// that the exponents, the opacity products and 1 - alpha of both come from packed FP32x2
// instructions (Blackwell's paired FP32 pipe), and the step has no branch per fragment (a
// rejected fragment gets alpha 0, which leaves C and T unchanged bit for bit).  Every rounding
// step is the scalar rule's, lane by lane, so the image is the same as a one-fragment walk's.
// The CTA leaves the range as soon as every pixel has stopped (a block-wide vote per batch).
// With `mark` set, every blended fragment also flags its survivor (the visibility labeller);
// the kernels that track the last blended pair and the marks (kAux) are separate instances, so
// that an ordinary frame does not carry that bookkeeping.
//
// Dense tiles (the supplement's section on Gaussian and asset density: many Gaussians on few pixels balance
// badly): k_blend walks at most `split_len` pairs of a tile.  If some pixel of a longer tile is
// still unsaturated after them, its state (colour, T, count) is saved and the rest of the range
// is cut into chunks of split_len that separate CTAs process in three steps --
//   k_blend_split_T  the product of (1 - alpha) over each chunk's blended fragments per pixel;
//   k_blend_split_C  each chunk again, entering with T = the saved T times the products of the
//                    earlier chunks (nothing to do once that is below t_stop), stop rule applied;
//   k_blend_split_D  per pixel, the saved colour plus the chunks' colours up to the one that
//                    stopped, and the transmittance left by it composing the background.
// Only the grouping of the T products differs from the one-CTA order (FP32 rounding).
#include <algorithm>

#include "nvgs_internal.cuh"

namespace nvgs {

namespace {

struct Frag {
    float T, C0, C1, C2;
    uint32_t last;       // global index + 1 of the last pair blended at the pixel (0: none)
    bool done;
    uint32_t walked;     // (pixel, fragment) evaluations up to the stop -- the compositing's unit
    uint32_t blended;    // of those, the fragments composited
    __device__ Frag(float T_, bool done_)
        : T(T_), C0(0.f), C1(0.f), C2(0.f), last(0), done(done_), walked(0), blended(0) {}
};

// View of global tile `tile` in a multi-view batch: the last view whose tile_base is <= tile (views
// are numbered in tile order).  One view: 0.
__device__ __forceinline__ int tile_view(const CamParams* __restrict__ camp, int n_views, int tile) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (camp[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Adds the block's evaluations and composited fragments to out[0], out[1] (profiling; nullable).
__device__ __forceinline__ void add_evals(unsigned long long* out, const Frag& f) {
    if (!out) return;
    unsigned long long v = f.walked, e = f.blended;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    if ((threadIdx.x & 31) == 0 && v) {
        atomicAdd(out, v);
        atomicAdd(out + 1, e);
    }
}

// A batch of up to 256 staged fragments, stored in pairs (fragments 2p and 2p + 1 side by side) so
// that every pixel evaluates two fragments per step with packed FP32x2 arithmetic.
template <int TS>
struct Smem {
    static constexpr int NB = TS * TS < 256 ? TS * TS : 256;   // fragments a batch (even)
    static constexpr int NP = NB / 2;
    float4 uv[NP];   // (-u, -u', -v, -v'): the mean, negated
    float4 ab[NP];   // (kA, kA', kB, kB')
    float4 co[NP];   // (kC, kC', opacity, opacity')
    float4 rg[NP];   // (r, r', g, g')
    float2 bl[NP];   // (b, b')
};

// The compositing kernels' shared memory: the staged batches while walking, then the tile's final
// colours for the image write.
template <int TS>
union BlendShared {
    Smem<TS> st;
    float rgb[3 * TS * TS];
};

// Writes a block of `rows` tile rows, whose colours are in rgb (3 floats per pixel, row-major,
// TS pixels a row), to the image rows y0.. at columns x0..: consecutive threads store consecutive
// floats of an image row, so each tile row leaves as one contiguous run (192 bytes at 16 x 16)
// rather than as three 12-byte-strided stores per pixel -- what keeps a page-locked host image
// written over the host link at full width.  Pixels outside the image are skipped.  Call after
// a barrier that follows the rgb stores.
template <int TS, int kThreads>
__device__ __forceinline__ void store_rows_rgb(const float* rgb, int rows, float* __restrict__ image,
                                               const CamParams& cam, int x0, int y0) {
    const int run = 3 * min(TS, cam.W - x0);
    for (int q = threadIdx.x; q < 3 * TS * rows; q += kThreads) {
        const int r = q / (3 * TS), c = q - r * (3 * TS);
        if (y0 + r < cam.H && c < run) image[((size_t)(y0 + r) * cam.W + x0) * 3 + c] = rgb[q];
    }
}

// Stages fragment k = base + t of a batch (gathered by its survivor index) into slot (t / 2, t % 2);
// past the range it stages a fragment of zero opacity, which no pixel composites (the padding of
// an odd last pair).
template <int TS>
__device__ __forceinline__ void stage(Smem<TS>& sm, const uint32_t* __restrict__ values,
                                      const float4* __restrict__ rec, int t, uint32_t k, uint32_t end) {
    const int p = t >> 1, h = t & 1;
    float* uv = reinterpret_cast<float*>(&sm.uv[p]);
    float* ab = reinterpret_cast<float*>(&sm.ab[p]);
    float* co = reinterpret_cast<float*>(&sm.co[p]);
    float* rg = reinterpret_cast<float*>(&sm.rg[p]);
    float* bl = reinterpret_cast<float*>(&sm.bl[p]);
    if (k < end) {
        const size_t idx = kRecF4 * (size_t)values[k];
        float4 sa, sb;
        stage_splat(__ldg(&rec[idx]), __ldg(&rec[idx + 1]), sa, sb);
        const float4 c = __ldg(&rec[idx + 2]);
        uv[h] = -sa.x; uv[2 + h] = -sa.y;
        ab[h] = sa.z;  ab[2 + h] = sa.w;
        co[h] = sb.x;  co[2 + h] = sb.y;
        rg[h] = c.x;   rg[2 + h] = c.y;
        bl[h] = c.z;
    } else {   // zero opacity: alpha 0 < alpha_min everywhere
        uv[h] = 0.f; uv[2 + h] = 0.f;
        ab[h] = 0.f; ab[2 + h] = 0.f;
        co[h] = 0.f; co[2 + h] = 0.f;
        rg[h] = 0.f; rg[2 + h] = 0.f;
        bl[h] = 0.f;
    }
}

// Blend staged fragments [base, base + nb) into one pixel, two per step, in straight-line code
// (no branch per fragment: a rejected fragment gets alpha 0).  Per fragment, in list order,
// exactly the scalar rules with the same FP32 operations lane by lane: the exponent p2, skip if
// p2 > 0; alpha = min(alpha_max, opacity 2^p2), skip if alpha < alpha_min (this also covers the
// ln(alpha_min / opacity) pre-test, whose 1e-4 margin lies far outside ex2's error); stop
// without blending if T (1 - alpha) < t_stop; else C += alpha T rgb, T *= 1 - alpha.  The second
// fragment of a pair sees the T the first one left.  transmittance_only: no stop rule before the
// update and no colour -- the product of (1 - alpha), ending once it is below t_stop.  kAux:
// also track the last blended pair and flag blended survivors in `mark`.
template <int TS, bool kTransmittanceOnly, bool kAux, bool kCount>
__device__ __forceinline__ void blend_batch(const Smem<TS>& sm, int nb, float fx, float fy,
                                            const CamParams& cam, Frag& f,
                                            const uint32_t* __restrict__ values, uint32_t base,
                                            uint8_t* __restrict__ mark) {
    const float2 FX = make_float2(fx, fx), FY = make_float2(fy, fy);
    const float2 ONE = make_float2(1.0f, 1.0f), MINUS = make_float2(-1.0f, -1.0f);
    const int np = (nb + 1) >> 1;
    for (int p = 0; p < np && !f.done; p++) {
        const float4 uv = sm.uv[p];
        const float4 ab = sm.ab[p];
        const float4 co = sm.co[p];
        const float2 dx = __fadd2_rn(FX, make_float2(uv.x, uv.y));
        const float2 dy = __fadd2_rn(FY, make_float2(uv.z, uv.w));
        const float2 t = __ffma2_rn(make_float2(ab.x, ab.y), dx, __fmul2_rn(make_float2(ab.z, ab.w), dy));
        const float2 p2 = __ffma2_rn(dx, t, __fmul2_rn(__fmul2_rn(make_float2(co.x, co.y), dy), dy));
        const float2 og = __fmul2_rn(make_float2(co.z, co.w), make_float2(ex2_approx(p2.x), ex2_approx(p2.y)));
        const float2 al = make_float2(fminf(cam.alpha_max, og.x), fminf(cam.alpha_max, og.y));
        // alpha of a fragment that passes the tests, else 0 (a passing alpha is >= alpha_min > 0)
        const float ax = (!(p2.x > 0.0f) && al.x >= cam.alpha_min) ? al.x : 0.0f;
        const float ay = (!(p2.y > 0.0f) && al.y >= cam.alpha_min) ? al.y : 0.0f;
        const float2 om = __ffma2_rn(MINUS, make_float2(ax, ay), ONE);   // 1 - alpha, as the scalar rule
        // T after each (T >= t_stop on entry, and a skipped fragment leaves it as it is): the
        // first stops iff T (1 - a1) < t_stop, the pair stops (at the first or the second) iff
        // T (1 - a1) (1 - a2) < t_stop
        const float ntx = f.T * om.x;
        const float nty = ntx * om.y;
        const bool sx = ntx < cam.t_stop, sy = nty < cam.t_stop;
        if (kTransmittanceOnly) {   // the stopping factor is applied, then the product ends
            if (kCount) {
                f.walked += sx ? 1 : min(2, nb - 2 * p);
                f.blended += (int)(ax > 0.0f) + (int)(!sx && ay > 0.0f);
            }
            f.T = sx ? ntx : nty;
            f.done = sy;
            continue;
        }
        const float4 rg = sm.rg[p];
        const float2 bl = sm.bl[p];
        const float2 w0 = __fmul2_rn(make_float2(ax, ay), make_float2(f.T, ntx));
        const float wx = sx ? 0.0f : w0.x, wy = sy ? 0.0f : w0.y;   // a stopping fragment is not blended
        // in list order, as the scalar rule (an unblended fragment adds 0 x rgb: C is unchanged)
        f.C0 = fmaf(wy, rg.y, fmaf(wx, rg.x, f.C0));
        f.C1 = fmaf(wy, rg.w, fmaf(wx, rg.z, f.C1));
        f.C2 = fmaf(wy, bl.y, fmaf(wx, bl.x, f.C2));
        const bool blx = !sx && ax > 0.0f, bly = !sy && ay > 0.0f;
        if (kAux) {
            if (mark) {   // contribution alpha * T > 0 (Sec. 3.1)
                if (blx) mark[values[base + 2 * p]] = 1;
                if (bly) mark[values[base + 2 * p + 1]] = 1;
            }
            f.last = bly ? base + 2 * p + 2 : (blx ? base + 2 * p + 1 : f.last);
        }
        if (kCount) {
            f.walked += sx ? 1 : min(2, nb - 2 * p);
            f.blended += (int)blx + (int)bly;
        }
        f.T = sy ? (sx ? f.T : ntx) : nty;
        f.done = sy;
    }
}

// Walk pairs [start, end) for this thread's pixel in staged batches (the CTA's kThreads threads
// stage them together), with a block-wide exit vote per batch.
template <int TS, int kThreads, bool kTransmittanceOnly, bool kAux, bool kCount>
__device__ __forceinline__ void walk(const uint32_t* __restrict__ values, const float4* __restrict__ rec,
                                     uint32_t start, uint32_t end, float fx, float fy,
                                     const CamParams& cam, Frag& f, uint8_t* __restrict__ mark, Smem<TS>& sm) {
    constexpr int NB = Smem<TS>::NB;
    for (uint32_t base = start; base < end; base += NB) {
        if (__syncthreads_count(f.done) == kThreads) break;   // also: the previous batch is consumed
#pragma unroll
        for (int t = threadIdx.x; t < NB; t += kThreads) stage<TS>(sm, values, rec, t, base + t, end);
        __syncthreads();
        const int nb = (int)min((uint32_t)NB, end - base);
        blend_batch<TS, kTransmittanceOnly, kAux, kCount>(sm, nb, fx, fy, cam, f, values, base, mark);
    }
}

}  // namespace

// CTAs per SM the compositing kernels are compiled for: 4 at 16 x 16 (up to 64 registers a
// thread), which holds the paired evaluation without spills (at 5, 48 registers spill and the
// kernel is slower).
template <int TS>
constexpr int blend_min_blocks() { return 1536 / (TS * TS) < 4 ? 1536 / (TS * TS) : 4; }

// CTAs that share one tile in k_blend, each compositing TS / parts full rows of it (all of them
// stage the tile's whole list): a CTA ends with the last of its own pixels, so that a tile whose
// rows saturate at different depths frees part of its SM early.
template <int TS>
constexpr int blend_parts() { return 1; }
constexpr int kMaxBlendParts = 4;

template <int TS, bool kAux, bool kCount>
__global__ void __launch_bounds__(TS * TS / blend_parts<TS>(), 4 * blend_parts<TS>()) k_blend(const uint32_t* __restrict__ ranges,
                                                  const uint32_t* __restrict__ values,
                                                  const float4* __restrict__ rec, const CamParams* __restrict__ camp,
                                                  float* __restrict__ image, float* __restrict__ final_T,
                                                  int32_t* __restrict__ n_contrib,
                                                  uint8_t* __restrict__ mark, uint32_t split_len,
                                                  const uint32_t* __restrict__ split_dev,
                                                  float4* __restrict__ state_tc,
                                                  int32_t* __restrict__ state_cnt,
                                                  uint32_t* __restrict__ alive,
                                                  unsigned long long* __restrict__ evals_out,
                                                  int n_views, float* const* __restrict__ images,
                                                  const uint32_t* __restrict__ tile_order) {
    constexpr int B = TS * TS, P = blend_parts<TS>(), kThreads = B / P;
    __shared__ BlendShared<TS> sh;
    Smem<TS>& sm = sh.st;
    if (split_dev) split_len = *split_dev;   // resolved on the device (sync-free batches)
    const int tile = tile_order ? (int)tile_order[blockIdx.x / P] : (int)(blockIdx.x / P), part = blockIdx.x % P;
    const int li = part * kThreads + threadIdx.x;   // the pixel within the tile
    const int view = n_views > 1 ? tile_view(camp, n_views, tile) : 0;
    const CamParams cam = camp[view];
    if (images) image = images[view];
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const bool longer = end - start > split_len;
    const int lt = tile - cam.tile_base;   // the tile within its view
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TS + (li % TS), py = ty * TS + (li / TS);
    const bool inside = px < cam.W && py < cam.H;
    Frag f(1.0f, !inside);
    walk<TS, kThreads, false, kAux, kCount>(values, rec, start, longer ? start + split_len : end, (float)px + 0.5f,
                            (float)py + 0.5f, cam, f, mark, sm);
    if (kCount) add_evals(evals_out, f);
    if (longer) {
        const bool all_done = __syncthreads_count(f.done) == kThreads;
        if (threadIdx.x == 0) alive[(size_t)tile * kMaxBlendParts + part] = all_done ? 0u : 1u;
        if (!all_done) {   // the chunked kernels finish this part of the tile
            state_tc[(size_t)tile * B + li] = make_float4(f.C0, f.C1, f.C2, f.done ? -f.T - 1.0f : f.T);
            state_cnt[(size_t)tile * B + li] = (int32_t)f.last;
            return;
        }
    }
    __syncthreads();   // every thread is past the last staged batch: sh.rgb may overwrite it
    sh.rgb[3 * threadIdx.x] = fmaf(f.T, cam.bg[0], f.C0);
    sh.rgb[3 * threadIdx.x + 1] = fmaf(f.T, cam.bg[1], f.C1);
    sh.rgb[3 * threadIdx.x + 2] = fmaf(f.T, cam.bg[2], f.C2);
    if (inside) {
        const size_t p = (size_t)py * cam.W + px;
        if (final_T) final_T[p] = f.T;
        if (n_contrib) n_contrib[p] = (int32_t)f.last;
    }
    __syncthreads();
    store_rows_rgb<TS, kThreads>(sh.rgb, kThreads / TS, image, cam, tx * TS, ty * TS + part * (kThreads / TS));
}

// ------------------------------------------------------------------ dense tiles
// The automatic split length from the frame's pair count on the device, with the integer rule the
// synchronous path applies on the host: max(4096, 4 (n_pairs / n_tiles + 1)), capped at 2^31 - 1.
__global__ void k_split_auto(const uint32_t* __restrict__ n_pairs, uint32_t n_tiles,
                             uint32_t* __restrict__ split_len) {
    const uint64_t a = max((uint64_t)4096, 4 * ((uint64_t)*n_pairs / n_tiles + 1));
    *split_len = (uint32_t)min(a, (uint64_t)0x7fffffffu);
}

__global__ void k_split_count(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ alive,
                              int parts, int n_tiles, uint32_t split_len, const uint32_t* __restrict__ split_dev,
                              uint32_t* __restrict__ n_chunks) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    if (split_dev) split_len = *split_dev;
    const uint32_t n = ranges[2 * t + 1] - ranges[2 * t];
    bool any = false;   // some part of the tile is still unsaturated
    for (int q = 0; q < parts; q++) any = any || alive[(size_t)t * kMaxBlendParts + q] != 0u;
    n_chunks[t] = (n > split_len && any) ? (n - split_len + split_len - 1) / split_len : 0u;
}

__global__ void k_split_fill(const uint32_t* __restrict__ n_chunks, const uint32_t* __restrict__ first,
                             int n_tiles, uint2* __restrict__ items) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    for (uint32_t c = 0; c < n_chunks[t]; c++) items[first[t] + c] = make_uint2((uint32_t)t, c);
}

// [start, end) of chunk c of a continued tile (the first split_len pairs were k_blend's)
__device__ __forceinline__ void chunk_range(const uint32_t* __restrict__ ranges, uint2 it,
                                            uint32_t split_len, uint32_t& start, uint32_t& end) {
    start = ranges[2 * it.x] + (it.y + 1) * split_len;
    end = min(ranges[2 * it.x + 1], start + split_len);
}

template <int TS, bool kCount>
__global__ void __launch_bounds__(TS * TS, blend_min_blocks<TS>()) k_blend_split_T(const uint32_t* __restrict__ ranges,
                                                          const uint32_t* __restrict__ values,
                                                          const float4* __restrict__ rec, const CamParams* __restrict__ camp,
                                                          const uint2* __restrict__ items,
                                                          const uint32_t* __restrict__ n_items,
                                                          uint32_t split_len,
                                                          const uint32_t* __restrict__ split_dev,
                                                          const float4* __restrict__ state_tc,
                                                          float* __restrict__ Tch,
                                                          unsigned long long* __restrict__ evals_out,
                                                          int n_views) {
    constexpr int B = TS * TS;
    __shared__ Smem<TS> sm;
    // persistent: the grid is sized for the GPU, not for the worst-case item count
    const uint32_t n_it = *n_items;
    if (split_dev) split_len = *split_dev;
    for (uint32_t item = blockIdx.x; item < n_it; item += gridDim.x) {
        const uint2 it = items[item];
        const int tile = (int)it.x;
        uint32_t start, end;
        chunk_range(ranges, it, split_len, start, end);
        const CamParams cam = camp[n_views > 1 ? tile_view(camp, n_views, tile) : 0];
        const int lt = tile - cam.tile_base;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const int px = tx * TS + (threadIdx.x % TS), py = ty * TS + (threadIdx.x / TS);
        const bool stopped = state_tc[(size_t)tile * B + threadIdx.x].w < 0.0f;
        Frag f(1.0f, stopped || !(px < cam.W && py < cam.H));
        __syncthreads();   // the previous item's last batch is fully consumed
        walk<TS, TS * TS, true, false, kCount>(values, rec, start, end, (float)px + 0.5f, (float)py + 0.5f, cam, f, nullptr,
                                      sm);
        Tch[(size_t)item * B + threadIdx.x] = f.T;
        if (kCount) add_evals(evals_out, f);
    }
}

template <int TS, bool kAux, bool kCount>
__global__ void __launch_bounds__(TS * TS, blend_min_blocks<TS>()) k_blend_split_C(const uint32_t* __restrict__ ranges,
                                                          const uint32_t* __restrict__ values,
                                                          const float4* __restrict__ rec, const CamParams* __restrict__ camp,
                                                          const uint2* __restrict__ items,
                                                          const uint32_t* __restrict__ n_items,
                                                          uint32_t split_len,
                                                          const uint32_t* __restrict__ split_dev,
                                                          const float4* __restrict__ state_tc,
                                                          const float* __restrict__ Tch,
                                                          float4* __restrict__ part, int32_t* __restrict__ pcount,
                                                          uint8_t* __restrict__ mark,
                                                          unsigned long long* __restrict__ evals_out,
                                                          int n_views) {
    constexpr int B = TS * TS;
    __shared__ Smem<TS> sm;
    const uint32_t n_it = *n_items;
    if (split_dev) split_len = *split_dev;
    for (uint32_t item = blockIdx.x; item < n_it; item += gridDim.x) {
        const uint2 it = items[item];
        const int tile = (int)it.x;
        uint32_t start, end;
        chunk_range(ranges, it, split_len, start, end);
        const CamParams cam = camp[n_views > 1 ? tile_view(camp, n_views, tile) : 0];
        const int lt = tile - cam.tile_base;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const int px = tx * TS + (threadIdx.x % TS), py = ty * TS + (threadIdx.x / TS);
        // transmittance entering this chunk: after k_blend's pairs, times the earlier chunks
        const float sw = state_tc[(size_t)tile * B + threadIdx.x].w;
        float T_in = sw < 0.0f ? 0.0f : sw;
        for (uint32_t c = 0; c < it.y; c++) T_in *= Tch[(size_t)(item - it.y + c) * B + threadIdx.x];
        const bool dead = sw < 0.0f || T_in < cam.t_stop;
        Frag f(T_in, dead || !(px < cam.W && py < cam.H));
        __syncthreads();   // the previous item's last batch is fully consumed
        walk<TS, TS * TS, false, kAux, kCount>(values, rec, start, end, (float)px + 0.5f, (float)py + 0.5f, cam, f, mark,
                                      sm);
        // w < 0 marks "stopped inside this chunk or before"
        part[(size_t)item * B + threadIdx.x] = make_float4(f.C0, f.C1, f.C2, (f.done || dead) ? -f.T - 1.0f : f.T);
        pcount[(size_t)item * B + threadIdx.x] = (int32_t)f.last;
        if (kCount) add_evals(evals_out, f);
    }
}

template <int TS>
__global__ void __launch_bounds__(TS* TS) k_blend_split_D(const uint32_t* __restrict__ n_chunks,
                                                          const uint32_t* __restrict__ first,
                                                          const CamParams* __restrict__ camp, const float4* __restrict__ state_tc,
                                                          const int32_t* __restrict__ state_cnt,
                                                          const float4* __restrict__ part,
                                                          const int32_t* __restrict__ pcount,
                                                          float* __restrict__ image, float* __restrict__ final_T,
                                                          int32_t* __restrict__ n_contrib,
                                                          int n_views, float* const* __restrict__ images) {
    constexpr int B = TS * TS;
    __shared__ float rgb[3 * B];
    const int tile = blockIdx.x;
    const uint32_t nc = n_chunks[tile];
    if (nc == 0) return;
    const int view = n_views > 1 ? tile_view(camp, n_views, tile) : 0;
    const CamParams cam = camp[view];
    if (images) image = images[view];
    const int lt = tile - cam.tile_base;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TS + (threadIdx.x % TS), py = ty * TS + (threadIdx.x / TS);
    const float4 st = state_tc[(size_t)tile * B + threadIdx.x];
    float C0 = st.x, C1 = st.y, C2 = st.z, T;
    int32_t last = state_cnt[(size_t)tile * B + threadIdx.x];
    if (st.w < 0.0f) {
        T = -st.w - 1.0f;   // stopped inside k_blend's pairs
    } else {
        T = st.w;
        for (uint32_t c = 0; c < nc; c++) {
            const size_t q = (size_t)(first[tile] + c) * B + threadIdx.x;
            const float4 v = part[q];
            C0 += v.x; C1 += v.y; C2 += v.z;
            if (pcount[q] > 0) last = pcount[q];
            if (v.w < 0.0f) { T = -v.w - 1.0f; break; }   // stopped: later chunks add nothing
            T = v.w;
        }
    }
    rgb[3 * threadIdx.x] = fmaf(T, cam.bg[0], C0);
    rgb[3 * threadIdx.x + 1] = fmaf(T, cam.bg[1], C1);
    rgb[3 * threadIdx.x + 2] = fmaf(T, cam.bg[2], C2);
    if (px < cam.W && py < cam.H) {
        const size_t p = (size_t)py * cam.W + px;
        if (final_T) final_T[p] = T;
        if (n_contrib) n_contrib[p] = last;
    }
    __syncthreads();
    store_rows_rgb<TS, B>(rgb, TS, image, cam, tx * TS, ty * TS);
}

static inline uint64_t round256(uint64_t b) { return (b + 255) / 256 * 256; }

size_t blend_split_scratch_bytes(int n_tiles, uint64_t n_pairs, int tile_size, uint32_t split_len) {
    const uint64_t items = n_pairs / split_len + 2;
    const uint64_t B = (uint64_t)tile_size * tile_size;
    return (size_t)(round256((uint64_t)n_tiles * (8 + 4 * kMaxBlendParts) + 64) + round256((uint64_t)n_tiles * B * 16) +
                    round256((uint64_t)n_tiles * B * 4) + round256(items * 8) + round256(items * B * 4) +
                    round256(items * B * 16) + round256(items * B * 4));
}

// The tiles in descending classes of their work, min(pair count, split length) rounded down to a
// power of two (the order inside a class is whatever the shared-memory atomics give: a tile's
// result does not depend on when its CTA runs).  One CTA.
__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t* __restrict__ ranges, int n_tiles,
                                                     uint32_t split_len, const uint32_t* __restrict__ split_dev,
                                                     uint32_t* __restrict__ order) {
    __shared__ uint32_t slot[33];
    if (split_dev) split_len = *split_dev;
    if (threadIdx.x < 33) slot[threadIdx.x] = 0u;
    __syncthreads();
    auto cls = [&](int t) {
        const uint32_t w = min(ranges[2 * t + 1] - ranges[2 * t], split_len);
        return w ? 32 - __clz(w) : 0;   // 0 (empty) .. 32
    };
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) atomicAdd(&slot[cls(t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {   // class starts, the heaviest class first
        uint32_t run = 0;
        for (int c = 32; c >= 0; c--) { const uint32_t k = slot[c]; slot[c] = run; run += k; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) order[atomicAdd(&slot[cls(t)], 1u)] = (uint32_t)t;
}

template <int TS>
static cudaError_t blend_ts(const uint32_t* ranges, const uint32_t* values, const float4* rec,
                            const CamParams& cam, const CamParams* cam_dev, float* image, float* final_T,
                            int32_t* n_contrib, uint8_t* mark, uint32_t split_len, uint64_t n_pairs,
                            const uint32_t* auto_split_pairs, void* scratch, void* scan_scratch,
                            int num_sms, unsigned long long* evals, cudaStream_t s, LaunchLog* log,
                            int n_views, float* const* images, int n_tiles, uint32_t* tile_order) {
    constexpr int B = TS * TS;
    const bool may_split = n_pairs > split_len;
    const bool aux = n_contrib || mark;   // the last blended pair per pixel, blended survivors
    // carve the scratch; every section starts on a 256-byte boundary
    char* p = static_cast<char*>(scratch);
    uint32_t *n_chunks = nullptr, *first = nullptr, *n_items = nullptr, *alive = nullptr;
    uint32_t* split_dev = nullptr;
    float4* state_tc = nullptr;
    int32_t* state_cnt = nullptr;
    uint2* items = nullptr;
    float* Tch = nullptr;
    float4* part = nullptr;
    int32_t* pcount = nullptr;
    const uint64_t max_items = n_pairs / split_len + 2;
    if (may_split) {
        n_chunks = reinterpret_cast<uint32_t*>(p);
        first = n_chunks + n_tiles;
        alive = first + n_tiles;   // per tile, one flag per part
        n_items = alive + (size_t)n_tiles * kMaxBlendParts;
        if (auto_split_pairs) split_dev = n_items + 1;   // inside the region's 64 spare bytes
        p += round256((uint64_t)n_tiles * (8 + 4 * kMaxBlendParts) + 64);
        state_tc = reinterpret_cast<float4*>(p);
        p += round256((uint64_t)n_tiles * B * 16);
        state_cnt = reinterpret_cast<int32_t*>(p);
        p += round256((uint64_t)n_tiles * B * 4);
        items = reinterpret_cast<uint2*>(p);
        p += round256(max_items * 8);
        Tch = reinterpret_cast<float*>(p);
        p += round256(max_items * B * 4);
        part = reinterpret_cast<float4*>(p);
        p += round256(max_items * B * 16);
        pcount = reinterpret_cast<int32_t*>(p);
    }
    if (split_dev) {
        NVGS_LAUNCH(log, s, "k_split_auto", k_split_auto<<<1, 1, 0, s>>>(auto_split_pairs, (uint32_t)n_tiles, split_dev));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (tile_order) {
        NVGS_LAUNCH(log, s, "k_tile_order", k_tile_order<<<1, 1024, 0, s>>>(ranges, n_tiles, split_len, split_dev, tile_order));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    NVGS_LAUNCH(log, s, TS == 8 ? "k_blend<8>" : TS == 16 ? "k_blend<16>" : "k_blend<32>",
                (evals ? k_blend<TS, true, true> : aux ? k_blend<TS, true, false> : k_blend<TS, false, false>)<<<n_tiles * blend_parts<TS>(), B / blend_parts<TS>(), 0, s>>>(ranges, values, rec, cam_dev, image, final_T, n_contrib, mark,
                                                  split_len, split_dev, state_tc, state_cnt, alive, evals, n_views, images,
                                                  tile_order));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !may_split) return e;
    NVGS_LAUNCH(log, s, "k_split_count", k_split_count<<<(n_tiles + 255) / 256, 256, 0, s>>>(ranges, alive, blend_parts<TS>(), n_tiles, split_len, split_dev, n_chunks));
    e = exclusive_scan_u32(n_chunks, first, n_tiles, n_items, scan_scratch, s, log);
    if (e != cudaSuccess) return e;
    NVGS_LAUNCH(log, s, "k_split_fill", k_split_fill<<<(n_tiles + 255) / 256, 256, 0, s>>>(n_chunks, first, n_tiles, items));
    // persistent grids: enough CTAs to fill the GPU (the item count lives on the device)
    const unsigned pgrid = (unsigned)std::min<uint64_t>(max_items, (uint64_t)num_sms * (2048 / B));
    NVGS_LAUNCH(log, s, "k_blend_split_T", (evals ? k_blend_split_T<TS, true> : k_blend_split_T<TS, false>)<<<pgrid, B, 0, s>>>(ranges, values, rec, cam_dev, items, n_items, split_len, split_dev, state_tc, Tch, evals, n_views));
    NVGS_LAUNCH(log, s, "k_blend_split_C", (evals ? k_blend_split_C<TS, true, true> : aux ? k_blend_split_C<TS, true, false> : k_blend_split_C<TS, false, false>)<<<pgrid, B, 0, s>>>(ranges, values, rec, cam_dev, items, n_items, split_len, split_dev, state_tc, Tch, part, pcount, mark, evals, n_views));
    NVGS_LAUNCH(log, s, "k_blend_split_D", k_blend_split_D<TS><<<n_tiles, B, 0, s>>>(n_chunks, first, cam_dev, state_tc, state_cnt, part, pcount, image, final_T, n_contrib, n_views, images));
    return cudaGetLastError();
}

cudaError_t launch_blend(const uint32_t* ranges, const uint32_t* values, const float4* rec,
                         const CamParams& cam, const CamParams* cam_dev, float* image, float* final_T,
                         int32_t* n_contrib, uint8_t* mark, uint32_t split_len, uint64_t n_pairs,
                         const uint32_t* auto_split_pairs, void* scratch, void* scan_scratch,
                         int num_sms, unsigned long long* evals, cudaStream_t s, LaunchLog* log,
                         int n_views, float* const* images, int n_tiles_total, uint32_t* tile_order) {
    const int n_tiles = n_tiles_total > 0 ? n_tiles_total : cam.tiles_x * cam.tiles_y;
    if (n_tiles <= 0) return cudaSuccess;
    switch (cam.tile_size) {
        case 8: return blend_ts<8>(ranges, values, rec, cam, cam_dev, image, final_T, n_contrib, mark, split_len, n_pairs, auto_split_pairs, scratch, scan_scratch, num_sms, evals, s, log, n_views, images, n_tiles, tile_order);
        case 16: return blend_ts<16>(ranges, values, rec, cam, cam_dev, image, final_T, n_contrib, mark, split_len, n_pairs, auto_split_pairs, scratch, scan_scratch, num_sms, evals, s, log, n_views, images, n_tiles, tile_order);
        case 32: return blend_ts<32>(ranges, values, rec, cam, cam_dev, image, final_T, n_contrib, mark, split_len, n_pairs, auto_split_pairs, scratch, scan_scratch, num_sms, evals, s, log, n_views, images, n_tiles, tile_order);
        default: return cudaErrorInvalidValue;
    }
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
