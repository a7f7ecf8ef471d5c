// Internal declarations shared by the CUDA translation units of libnvgs (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/nvgs.h"

namespace nvgs {

// Per-device once-only setup of a kernel (a function attribute belongs to the device it was set
// on): `done` holds one bit per device ordinal below 64; a device at or above 64 repeats the setup
// every time, which is correct, only slower.  Setting the same attribute twice is harmless, so
// two host threads that race here both succeed.
template <typename Setup>
cudaError_t once_per_device(std::atomic<uint64_t>& done, Setup setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = setup();
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

constexpr int kMlpIn = 32;
constexpr int kMlpHidden = 64;
constexpr int kMlpWeights = 64 * 32 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1;  // 10497
constexpr int kChunk = 2048;          // Gaussians per S1 work item (64 bitmask words)
constexpr int kChunkWords = kChunk / 32;

// One asset in device memory (structure of arrays of 16-byte vectors).
struct AssetDev {
    const float4* mean_op;    // (x, y, z, opacity logit)
    const float4* scale_quat; // per Gaussian (log sx, log sy, log sz, 0) then (w, x, y, z): the
                              // 32 bytes the projection reads together, one sector
    const float* sh;          // n * sh_stride floats, coefficient-major, RGB innermost
    const float* w_fp32;      // visibility MLP, kMlpWeights floats (nullptr: no MLP)
    const uint8_t* w_tc;      // BF16 operand tiles for the tcgen05 MLP (nullptr: none)
    const uint8_t* w_f8;      // E4M3 operand tiles + FP32 scales for the FP8 tcgen05 MLP (nullptr: none)
    int64_t n;
    int sh_degree;
    int sh_stride;            // floats per Gaussian, multiple of 4
    float bbox_c[3];          // centre of the means' bounding box
    float bbox_scale[3];      // 2 / extent: p = (mu - c) * scale lies in [-1, 1]
    float bbox_r;             // half the box diagonal
    float log_dmin;           // ln d_min
    float inv_log_range;      // 1 / (ln d_max - ln d_min)
    float d_min, d_max;
    float train_focal;        // f_t = 1 / tan(theta_t / 2)
};

// Per frame, per instance: transforms composed in FP64 on the device, rounded to FP32.
struct FrameInst {
    float M[9];               // s * Rc * Ri: local point -> camera frame (linear part)
    float b[3];               // Rc * t_i + t_c
    float W[9];               // Rc * Ri (rotation part; covariance uses s^2 W S W^T)
    float cam_local[3];       // camera centre in the instance's local frame
    float s;
    float dist_scale;         // f_t / f_r (Eq. 2; the 1/s is inside cam_local)
    int asset;
    int visible;              // bounding sphere meets the guard-band frustum
    int gated;                // instance closer than d_min: bypass the MLP (Sec. 3.3)
    int no_mlp;               // the asset has no visibility MLP: rendered unculled
    int view;                 // the view (camera) of this frame instance in a multi-view batch
};

// Camera-space position of a local mean: the small terms M mu first, the instance offset b last,
// so that points of one instance keep their relative depth to about one FP32 ulp.
__device__ __forceinline__ float3 cam_point(const FrameInst& f, float mx, float my, float mz) {
    float x = fmaf(f.M[0], mx, fmaf(f.M[1], my, f.M[2] * mz)) + f.b[0];
    float y = fmaf(f.M[3], mx, fmaf(f.M[4], my, f.M[5] * mz)) + f.b[1];
    float z = fmaf(f.M[6], mx, fmaf(f.M[7], my, f.M[8] * mz)) + f.b[2];
    return make_float3(x, y, z);
}

// Camera plus blending constants, passed by value to kernels.
struct CamParams {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int W, H;
    float z_near;
    float lim_x, lim_y;       // guard_band * W / (2 fx), guard_band * H / (2 fy)
    float f_r;                // 2 fx / W
    float alpha_min, alpha_max, t_stop, dilation;
    float bg[3];
    int tile_size, tiles_x, tiles_y;
    int mlp_gate;             // 1: instances closer than d_min bypass the MLP
    float clip_det;           // radius clipping: splats with det Sigma_2D below it are not binned (0: off)
    int tile_base;            // first global tile id of this view (multi-view batches; 0 otherwise)
};

// Real spherical harmonics up to degree 3 (the 3DGS sign convention), Y[(l+1)^2].
// Constants: 1/(2 sqrt pi); sqrt(3/(4 pi)); sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4;
// sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float* Y) {
    Y[0] = 0.28209479177387814f;
    if (deg < 1) return;
    Y[1] = -0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = -0.4886025119029199f * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    if (deg < 3) return;
    Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
    Y[10] = 2.890611442640554f * x * y * z;
    Y[11] = -0.4570457994644658f * y * (4.0f * zz - xx - yy);
    Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -0.4570457994644658f * x * (4.0f * zz - xx - yy);
    Y[14] = 1.445305721320277f * z * (xx - yy);
    Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
}

// Compositing form of a splat record a = (u, v, A, B), b = (C, opacity, depth, ln(alpha_min/o)):
// the exponent in base 2, p2 = log2(e) (-1/2 (A dx^2 + C dy^2) - B dx dy), costs five operations
// per pixel with the per-splat constants kA = -log2(e) A / 2, kB = -log2(e) B, kC = -log2(e) C / 2
// folded in once, and alpha = opacity 2^p2 needs no further multiply.  The pre-test bound
// w2 = log2(e) (ln(alpha_min / opacity) - 1e-4) skips a fragment whose exponent is below the
// alpha_min level by more than 1e-4 (in natural units) before the exponential.  Every rounding
// step is explicit, so the compositing and its derivative compute bit-identical exponents.
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ void stage_splat(const float4& a, const float4& b, float4& sa, float4& sb) {
    sa = make_float4(a.x, a.y, __fmul_rn(-0.5f * kLog2e, a.z), __fmul_rn(-kLog2e, a.w));
    sb = make_float4(__fmul_rn(-0.5f * kLog2e, b.x), b.y, __fmul_rn(kLog2e, __fadd_rn(b.w, -1e-4f)), 0.0f);
}

__device__ __forceinline__ float splat_exponent2(const float4& sa, const float4& sb, float dx, float dy) {
    const float t = __fmaf_rn(sa.z, dx, __fmul_rn(sa.w, dy));         // kA dx + kB dy
    return __fmaf_rn(dx, t, __fmul_rn(__fmul_rn(sb.x, dy), dy));      // dx t + kC dy^2
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// S5 binning refinement.  A splat's tile rectangle (the box of its support ellipse) is pruned,
// row by row, to the tiles whose pixel-centre box meets the ellipse q(d) <= kk.  Within a tile
// row (a horizontal band of pixel-centre offsets y in [y0, y1]) the ellipse is convex, so the
// tiles it meets are those whose pixel-centre columns meet the interval of x it covers over the
// band: [min x_left(y), max x_right(y)] with
//   x_right/left(y) = (cb y +- sqrt(det (cc kk - y^2))) / cc,   |y| <= sqrt(cc kk),
// (Sigma_2D = [[ca, cb], [cb, cc]], det its determinant); x_right is concave with its maximum at
// the ellipse's rightmost point y = cb x_max / ca, x_max = sqrt(ca kk), so its maximum over the
// band is at that y clamped to the band (and symmetrically for x_left).  The projection counts
// with these functions and the duplication writes with them, on the same stored record values
// (conic and det), with every rounding step explicit, so both agree bit for bit.  It is
// conservative: kk is inflated by 1e-4 relative plus 1e-3 and the interval widened by 1e-3 px
// plus 1e-5 relative -- more than the compositing's exponent pre-test margin, and far more than
// the ~1e-7 relative error of the hardware's approximate square root, reciprocal and division
// used for the extents and of the division by cc (a product with its reciprocal) -- so a pruned
// tile holds no pixel the compositing could blend.  The per-splat part (splat_ellipse) is
// computed once per splat, the per-row part (row_tile_span) per tile row.
struct SplatEllipse {
    float u, v;          // mean (pixels)
    float cb, rcc;       // Sigma_2D[0][1], 1 / Sigma_2D[1][1] (rounded)
    float det, ck;       // det Sigma_2D, cc kq (kq: the inflated support level)
    float ymax, yr;      // vertical half-extent sqrt(cc kq); y of the rightmost point
};

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ SplatEllipse splat_ellipse(float u, float v, float A, float B, float C, float det,
                                                      float kk) {
    SplatEllipse e;
    e.u = u; e.v = v;
    const float ca = __fmul_rn(C, det);
    e.cb = __fmul_rn(-B, det);
    const float cc = __fmul_rn(A, det);
    e.det = det;
    const float kq = __fadd_rn(__fmul_rn(kk, 1.0001f), 1e-3f);
    const float xmax = sqrt_approx(__fmul_rn(ca, kq));
    e.ck = __fmul_rn(cc, kq);
    e.ymax = sqrt_approx(e.ck);
    e.yr = __fmul_rn(__fmul_rn(e.cb, xmax), rcp_approx(ca));
    e.rcc = rcp_approx(cc);
    return e;
}

// Tile columns [t0, t1] of tile row ty that the ellipse reaches (t0 > t1: none).  ts is the tile
// size (8, 16 or 32) and rts = 1 / ts, exact for these powers of two.
__device__ __forceinline__ void row_tile_span(const SplatEllipse& e, int ty, int ts, float rts, int& t0, int& t1) {
    const float y0 = __fsub_rn(__fadd_rn((float)(ty * ts), 0.5f), e.v);
    const float y1 = __fsub_rn(__fadd_rn((float)((ty + 1) * ts), -0.5f), e.v);
    const float ya = fmaxf(y0, -e.ymax), yb = fminf(y1, e.ymax);
    if (!(ya <= yb)) { t0 = 1; t1 = 0; return; }
    const float ys = fminf(yb, fmaxf(ya, e.yr));     // band point of the rightmost x
    const float yl = fminf(yb, fmaxf(ya, -e.yr));    // band point of the leftmost x
    const float hr = sqrt_approx(fmaxf(0.0f, __fmul_rn(e.det, __fsub_rn(e.ck, __fmul_rn(ys, ys)))));
    const float hl = sqrt_approx(fmaxf(0.0f, __fmul_rn(e.det, __fsub_rn(e.ck, __fmul_rn(yl, yl)))));
    float xr = __fmul_rn(__fadd_rn(__fmul_rn(e.cb, ys), hr), e.rcc);
    float xl = __fmul_rn(__fsub_rn(__fmul_rn(e.cb, yl), hl), e.rcc);
    const float pad = __fadd_rn(1e-3f, __fmul_rn(1e-5f, __fadd_rn(fabsf(xl), fabsf(xr))));
    xr = __fadd_rn(__fadd_rn(xr, pad), e.u);    // absolute pixel coordinates
    xl = __fsub_rn(__fadd_rn(xl, e.u), pad);
    // tile tx's pixel centres span [tx ts + 0.5, tx ts + ts - 0.5]
    t1 = (int)floorf(__fmul_rn(__fsub_rn(xr, 0.5f), rts));
    t0 = (int)ceilf(__fmul_rn(__fadd_rn(xl, 0.5f - (float)ts), rts));
}

// Exclusive warp prefix of one value per lane; returns the warp total.
__device__ __forceinline__ uint32_t warp_prefix(uint32_t area, uint32_t& pre) {
    const int lane = threadIdx.x & 31;
    uint32_t p = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, p, o);
        if (lane >= o) p += t;
    }
    pre = p - area;
    return __shfl_sync(0xffffffffu, p, 31);
}

// Raw instance as uploaded by nvgs_set_instances.
struct InstanceRaw {
    float R[9], t[3], s;
    int asset;
};

// S1 work item: up to kChunk consecutive Gaussians of one instance.
struct Chunk {
    int inst;
    int g0;
    int count;
    int pad_;
};

// ------------------------------------------------------------------ launch log
// Counts kernel launches and, when `record` is set, brackets each launch with CUDA events on
// its stream so that per-kernel device time can be read back after the frame.
struct LaunchLog {
    static constexpr int kMax = 1024;
    uint64_t count = 0;
    bool record = false;
    bool ready = false;
    int n = 0;
    cudaEvent_t ev[2 * kMax];
    const char* names[kMax];
    void begin(cudaStream_t s, const char* name) {
        if (record && ready && n < kMax) {
            names[n] = name;
            cudaEventRecord(ev[2 * n], s);
        }
    }
    void end(cudaStream_t s) {
        count++;
        if (record && ready && n < kMax) {
            cudaEventRecord(ev[2 * n + 1], s);
            n++;
        }
    }
};
#define NVGS_LAUNCH(log, stream, name, ...) \
    do {                                   \
        (log)->begin(stream, name);        \
        __VA_ARGS__;                       \
        (log)->end(stream);                \
    } while (0)

// ------------------------------------------------------------------ launchers (stream-ordered)
// Each returns cudaGetLastError() after its launches and logs them in *log.
// fi_map (nullable, device, n_fi entries): frame instance k = (view, instance) of a multi-view
// batch, with that view's camera cam_dev[view]; without it frame instance k = instance k, view 0.
cudaError_t launch_instance_setup(const InstanceRaw* inst, int n_inst, const AssetDev* assets,
                                  const CamParams* cam_dev, FrameInst* out, cudaStream_t s, LaunchLog* log,
                                  const int2* fi_map = nullptr, int n_fi = 0);

cudaError_t launch_frustum(const Chunk* chunks, int n_chunks, const FrameInst* fi,
                           const AssetDev* assets, const CamParams* cam_dev, uint32_t* bits,
                           uint32_t* chunk_counts, cudaStream_t s, LaunchLog* log);

// Writes (instance, gaussian) of every set bit, in bit order, at out[chunk_offsets[c] + rank].
cudaError_t launch_expand_chunks(const Chunk* chunks, int n_chunks, const uint32_t* bits,
                                 const uint32_t* chunk_offsets, uint2* out, cudaStream_t s,
                                 LaunchLog* log);

// S2: keep bits over a list of (instance, gaussian) entries.
// Launchers taking n_dev (nullable): the count is read on the device and n is the capacity
// (grids are sized from it; nothing waits for the count on the host).
cudaError_t launch_mlp_fp32(const uint2* list, uint32_t n, const uint32_t* n_dev, const FrameInst* fi,
                            const AssetDev* assets, const float* logits_override,
                            const int64_t* inst_offset, float threshold, uint32_t* keep_bits,
                            float* logits_out, cudaStream_t s, LaunchLog* log);
// FP8 (E4M3) variant; weights packed by mlp_f8_pack_weights (scales_out nullable: the five
// per-tensor scales s_W1, s_W2, s_W3, s_h1, s_h2).
size_t mlp_f8_weight_bytes();
void mlp_f8_pack_weights(const float* w, uint8_t* out, float* scales_out);
cudaError_t launch_mlp_f8(const uint2* list, uint32_t n, const uint32_t* n_dev,
                          const FrameInst* fi, const AssetDev* assets, float threshold, uint32_t* keep_bits,
                          float* logits_out, uint32_t* err_flag, int num_sms, cudaStream_t s, LaunchLog* log);
// The rows' means are read through each entry's instance and asset.  err_flag (device) is set to 1
// if a bounded wait on the tensor-core pipeline gave up.
cudaError_t launch_mlp_tc(const uint2* list, uint32_t n, const uint32_t* n_dev,
                          const FrameInst* fi,
                          const AssetDev* assets, float threshold, uint32_t* keep_bits,
                          float* logits_out, uint32_t* err_flag, int num_sms, int ctas_per_sm,
                          cudaStream_t s, LaunchLog* log);

// BF16 operand tiles of one asset's MLP in the tcgen05 shared-memory layout (host-side packing).
size_t mlp_tc_weight_bytes();
void mlp_tc_pack_weights(const float* w, uint8_t* out);

// One training step of the visibility MLP (k_train.cu); partial needs train_partial_bytes(B).
// bf16: forward and backward on the tcgen05 tensor cores (k_train_tc.cu) instead of FP32 CUDA
// cores; err_flag receives 1 if a bounded tensor-core wait gave up.
size_t train_partial_bytes(uint32_t B);
cudaError_t launch_train_step(const AssetDev* asset_dev, uint32_t n_gauss, const float4* views,
                              uint32_t n_views, const uint8_t* labels, uint32_t B, uint64_t seed,
                              uint32_t step, int32_t* sv, int32_t* sg, int explicit_samples,
                              uint32_t* n_pos, float* loss_sum, float* partial, float* w, float* m,
                              float* v, float lr, float beta1, float beta2, float eps, int bf16,
                              uint32_t* err_flag, cudaStream_t s, LaunchLog* log);
cudaError_t launch_train_fwd_bwd_tc(const float* w, const AssetDev* asset, const float4* views,
                                    const uint8_t* labels, const int32_t* sv, const int32_t* sg, uint32_t B,
                                    uint32_t n_gauss, const uint32_t* n_pos, float* partial, float* loss_sum,
                                    uint32_t* err_flag, cudaStream_t s, LaunchLog* log);

// Per-block popcounts of a bitmask over n items (blocks of kChunk items).
cudaError_t launch_bit_counts(const uint32_t* bits, uint32_t n, const uint32_t* n_dev,
                              uint32_t* block_counts, cudaStream_t s, LaunchLog* log);
// Stable compaction of list[i] for set bits i, using block offsets from the scan.
cudaError_t launch_compact_list(const uint2* list, uint32_t n, const uint32_t* n_dev, const uint32_t* bits,
                                const uint32_t* block_offsets, uint2* out, cudaStream_t s,
                                LaunchLog* log);

// Scatter of per-instanced-Gaussian outputs of nvgs_query_visibility.
cudaError_t launch_scatter_visibility(const uint2* list, uint32_t n, const uint32_t* keep_bits,
                                      const float* logits, const int64_t* inst_offset,
                                      const FrameInst* fi, float* out_logits, uint8_t* out_keep,
                                      cudaStream_t s, LaunchLog* log);

// Projected splat record: kRecF4 float4 = 64 bytes per survivor, so that one aligned 64-byte
// access fetches all of it (the binning and the compositing gather records in depth order):
//   [0] u, v, conic A, conic B
//   [1] conic C, opacity, det Sigma_2D, ln(alpha_min / opacity)
//   [2] r, g, b, camera-space depth
//   [3] tile rectangle x0, y0, x1, y1 (inclusive; int bits; multi-view: w | view << 16)
constexpr int kRecF4 = 4;
__device__ __forceinline__ int4 rec_rect(const float4* __restrict__ rec, size_t i) {
    return __ldg(reinterpret_cast<const int4*>(rec) + kRecF4 * i + 3);
}

// S4: records (with their tile rects) and tile counts; dkey / didx receive the depth sort keys
// (IEEE bits of the camera-space z) and the survivor indices 0..n-1.  multi_view: each survivor's
// camera is cam_dev[its frame instance's view], and the rect's w holds the last tile row | view << 16.
cudaError_t launch_project(const uint2* surv, uint32_t n, const uint32_t* n_dev, const FrameInst* fi,
                           const AssetDev* assets, const CamParams* cam_dev, float4* rec,
                           uint32_t* tile_counts, uint32_t* dkey, uint32_t* didx, int num_sms,
                           cudaStream_t s, LaunchLog* log, int multi_view = 0);

// S5 (k_bin.cu)
cudaError_t launch_gather_counts(const uint32_t* order, const uint32_t* counts, uint32_t n,
                                 const uint32_t* n_dev, uint32_t* counts_sorted, int num_sms,
                                 cudaStream_t s, LaunchLog* log);
// Pairs of the survivors in depth order: the tiles of each rectangle that row_tile_span keeps,
// as the projection counted them.  n_pairs (device) is the total; writes stop at pair_cap, and
// overflow (device, nullable) is set when the total exceeds it.
// multi_view: tile ids are global (the view's tile_base + its local tile id), the view taken
// from the rect (as launch_project writes it in multi-view mode).  keys: key_bytes 2 (uint16 tile
// ids, at most 65536 tiles) or 4 (uint32).
cudaError_t launch_duplicate(const uint32_t* order, const float4* rec,
                             const uint32_t* offsets, uint32_t n, const uint32_t* n_dev,
                             const CamParams* cam_dev, const uint32_t* n_pairs, uint32_t pair_cap,
                             uint32_t* overflow, void* keys, int key_bytes, uint32_t* values, int num_sms,
                             cudaStream_t s, LaunchLog* log, int multi_view = 0);
// keys: the sorted tile ids, key_bytes 2 (uint16) or 4 (uint32).
cudaError_t launch_tile_ranges(const void* keys, int key_bytes, uint32_t n, const uint32_t* n_dev,
                               uint32_t n_tiles, uint32_t* ranges, cudaStream_t s, LaunchLog* log);

// S6
// mark (nullable, per survivor): set to 1 when the survivor is blended at some pixel.  evals
// (nullable, device): receives the number of (pixel, fragment) evaluations (profiling).
// Tiles with more than split_len pairs take the chunked path; scratch must hold
// blend_split_scratch_bytes(...), scan_scratch a scan of n_tiles values.  auto_split_pairs
// (device, nullable): the split length is the automatic one, computed on the device from this pair
// count with the host's rule; split_len is then its lower bound 4096 (scratch sizing) and n_pairs
// the pair capacity.
size_t blend_split_scratch_bytes(int n_tiles, uint64_t n_pairs, int tile_size, uint32_t split_len);
// Multi-view batches (n_views > 1 or images != nullptr): the tiles of all views are global ids
// (cam_dev[v].tile_base), n_tiles_total of them; a tile's view is found from the tile bases and
// it is written to images[view] (a DEVICE array of n_views image pointers); final_T, n_contrib
// and mark must then be null.
cudaError_t launch_blend(const uint32_t* ranges, const uint32_t* values, const float4* rec,
                         const CamParams& cam, const CamParams* cam_dev, float* image, float* final_T,
                         int32_t* n_contrib, uint8_t* mark, uint32_t split_len, uint64_t n_pairs,
                         const uint32_t* auto_split_pairs, void* scratch, void* scan_scratch,
                         int num_sms, unsigned long long* evals, cudaStream_t s, LaunchLog* log,
                         int n_views = 1, float* const* images = nullptr, int n_tiles_total = 0,
                         uint32_t* tile_order = nullptr);
// tile_order (device, nullable; n_tiles entries of scratch): the compositing CTAs then take the
// tiles longest list first (pair counts capped at the split length, in power-of-two classes), so
// that the longest tiles do not start in the grid's last wave.
// labels[row * n_gauss + g] |= mark[s] for survivor s = (instance, g)
cudaError_t launch_mark_labels(const uint2* surv, uint32_t n_surv, const uint8_t* mark,
                               uint8_t* labels_row, cudaStream_t s, LaunchLog* log);

// ------------------------------------------------------------------ generic device primitives
// Exclusive scan of n uint32 values; total (nullable, device) receives the sum.  Needs
// scan_scratch_bytes(n) bytes of scratch.
size_t scan_scratch_bytes(uint64_t n);
// With n_dev, elements at or past *n_dev read as 0 (n is then the capacity); out is written over
// all n.
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* total,
                               void* scratch, cudaStream_t s, LaunchLog* log,
                               const uint32_t* n_dev = nullptr);

// Stable LSD radix sort (8-bit digits) of n (key, value) pairs on bits [0, key_bits); key bits at
// or above key_bits are ignored (they never change the order).
// keys/values hold the input; the alt buffers must hold n entries each.  With copy_back the
// result always lands in keys/values; otherwise *result_in_alt tells where it is.
// Scratch: radix_scratch_bytes(n).
size_t radix_scratch_bytes(uint64_t n);
cudaError_t radix_sort_pairs(unsigned long long* keys, uint32_t* values,
                             unsigned long long* keys_alt, uint32_t* values_alt, uint64_t n,
                             int key_bits, void* scratch, cudaStream_t s, LaunchLog* log,
                             int* passes_out, int copy_back, int* result_in_alt);
// The same sort for 32-bit keys, with digits of digit_bits (1..8) bits.
// With n_dev the element count is read on the device (n is the capacity).
cudaError_t radix_sort_pairs_u32(uint32_t* keys, uint32_t* values, uint32_t* keys_alt,
                                 uint32_t* values_alt, uint64_t n, int key_bits, void* scratch,
                                 cudaStream_t s, LaunchLog* log, int* passes_out, int copy_back,
                                 int* result_in_alt, const uint32_t* n_dev = nullptr,
                                 int digit_bits = 8);
// The same sort for 16-bit keys (key_bits <= 16): the S5 tile sort when the frame (or batch) has
// at most 65536 tiles, at 12 instead of 16 bytes of key + value traffic per element and pass.
cudaError_t radix_sort_pairs_u16(uint16_t* keys, uint32_t* values, uint16_t* keys_alt,
                                 uint32_t* values_alt, uint64_t n, int key_bits, void* scratch,
                                 cudaStream_t s, LaunchLog* log, int* passes_out, int copy_back,
                                 int* result_in_alt, const uint32_t* n_dev = nullptr,
                                 int digit_bits = 8);

// N2: gradients of the render (k_backward.cu).  gsurv: render_backward_scratch_bytes(n_surv).
size_t render_backward_scratch_bytes(uint64_t n_surv);
cudaError_t launch_render_backward(const uint32_t* ranges, const uint32_t* values, const float4* rec,
                                   const CamParams& cam, const CamParams* cam_dev, const float* final_T,
                                   const int32_t* last_pair,
                                   const float* dL_dimg, float* gsurv, const uint2* surv, uint32_t n_surv,
                                   const FrameInst* fi, const AssetDev* assets, int asset_id,
                                   float* g_means, float* g_ls, float* g_quat, float* g_op, float* g_sh,
                                   cudaStream_t s, LaunchLog* log);
cudaError_t launch_pack_asset(uint32_t n, int K, int stride, const float* means, const float* log_scales,
                              const float* quats, const float* opacity_logits, const float* sh,
                              float4* mean_op, float4* scale_quat, float* sh_out,
                              cudaStream_t s, LaunchLog* log);

}  // namespace nvgs
