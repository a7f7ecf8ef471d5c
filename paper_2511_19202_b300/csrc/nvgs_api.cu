// C ABI of libnvgs: context, scene upload and the per-frame orchestration of S1-S6 (NVGS
// Sec. 3.3).  Host code here only validates arguments, sizes buffers and enqueues kernels; every
// step of the pass itself runs in the kernels of the k_*.cu files.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nvgs_internal.cuh"

using namespace nvgs;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct AssetStore {
    DevBuf mean_op, scale_quat, sh, w_fp32, w_tc, w_f8;
    AssetDev dev{};
    int precision = -1;  // -1: no MLP
};

}  // namespace

struct nvgs_ctx {
    int device = 0;
    int num_sms = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    std::vector<AssetStore> assets;
    DevBuf assets_dev;
    bool assets_dirty = true;
    uint64_t scene_gen = 0;   // bumped by every change of assets, MLPs or instances (graph keys)

    std::vector<nvgs_instance> instances;
    std::vector<int64_t> inst_offset_h;
    DevBuf inst_raw, inst_offset, chunks;
    int n_chunks = 0;
    int64_t n_instanced = 0;

    // per-frame buffers
    DevBuf frame_inst, bits, chunk_counts, chunk_offsets, vis_list, keep_bits, logits_tmp,
        block_counts, block_offsets, surv, rec, tile_counts, tile_offsets, keys, vals,
        keys_alt, vals_alt, ranges, scratch, counters, image_tmp, final_T, n_contrib, mark, dkey,
        didx, dkey_alt, didx_alt, split_scratch, grad_surv, tile_order;
    // visibility-MLP training state, per asset (FP32 master weights, Adam moments, views)
    struct Train {
        DevBuf w, m, v, views;
        int n_views = 0;
    };
    std::vector<Train> train;
    DevBuf tr_sv, tr_sg, tr_partial;
    uint32_t* h_counters = nullptr;  // pinned mirror of counters
    // camera parameters of the frame(s) in flight: kernels read them from device memory (so that
    // a captured graph replays with new cameras); staged through pinned host memory
    DevBuf cam_dev;
    CamParams* h_cam = nullptr;
    int h_cam_cap = 0;
    cudaEvent_t cam_ev = nullptr;
    bool cam_ev_pending = false;

    cudaEvent_t ev[NVGS_NUM_STAGES + 1] = {};
    bool events_ready = false;

    // last frame (kept_frame: it kept final T and last-fragment indices and nothing has
    // overwritten its buffers since -- what nvgs_render_backward needs)
    nvgs_frame_view last{};
    CamParams last_cp{};
    bool kept_frame = false;
    // batched rendering: per-view counts (in frustum, survivors, pairs, pad) and the cached graph
    DevBuf view_stats;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint8_t> graph_key;
    // multi-view batches with per-view instance sets: (view, instance) map, chunk list, image
    // pointers, and their cached graph
    DevBuf mv_fimap, mv_chunks, mv_images;
    cudaGraphExec_t mv_graph_exec = nullptr;
    std::vector<uint8_t> mv_graph_key;
    LaunchLog log;
    // per-kernel device time accumulated over profiled frames
    std::vector<std::string> kname;
    std::vector<uint64_t> kcount;
    std::vector<double> kms;
};

namespace {

nvgs_status fail(nvgs_ctx* c, nvgs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? NVGS_ERR_OOM : NVGS_ERR_CUDA,   \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                        __LINE__);                                                            \
    } while (0)

// Host-side fault injection for the tests: the next g_fail_allocs buffer growths fail as if
// cudaMalloc had run out of memory (nvgs_debug_fail_allocs).
std::atomic<int> g_fail_allocs{0};
// Bumped by every device or staging allocation: a captured graph holds raw buffer addresses, so
// its key carries this count and any (re)allocation since the capture forces a new capture.
std::atomic<uint64_t> g_alloc_gen{0};

cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return cudaSuccess;
    for (int left = g_fail_allocs.load(); left > 0;)
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) return cudaErrorMemoryAllocation;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        if (e != cudaSuccess) return e;
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 4;
    want = (want + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.cap = want;
    g_alloc_gen.fetch_add(1);
    return cudaSuccess;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

template <class T>
T* P(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

int bit_width(uint64_t v) {
    int b = 0;
    while (v) { b++; v >>= 1; }
    return b;
}

nvgs_status validate_flags(nvgs_ctx* ctx, const nvgs_render_flags* f) {
    if (!f) return fail(ctx, NVGS_ERR_INVALID_ARG, "flags is NULL");
    if (f->tile_size != 8 && f->tile_size != 16 && f->tile_size != 32)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "tile_size must be 8, 16 or 32 (got %d)", f->tile_size);
    if (!(f->alpha_min > 0.f && f->alpha_min < 1.f) || !(f->alpha_max > 0.f && f->alpha_max <= 1.f) ||
        !(f->t_stop >= 0.f && f->t_stop < 1.f) || !(f->dilation >= 0.f) || !(f->guard_band > 0.f))
        return fail(ctx, NVGS_ERR_INVALID_ARG, "blending constants out of range");
    if (f->mlp_ctas_per_sm < 0 || f->mlp_ctas_per_sm > 4)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "mlp_ctas_per_sm must be 0..4");
    if (!(f->radius_clip_area >= 0.0f) || !std::isfinite(f->radius_clip_area))
        return fail(ctx, NVGS_ERR_INVALID_ARG, "radius_clip_area must be a finite value >= 0");
    if (f->sort_digit_bits != 0 && (f->sort_digit_bits < 4 || f->sort_digit_bits > 8))
        return fail(ctx, NVGS_ERR_INVALID_ARG, "sort_digit_bits must be 0 or 4..8");
    if (f->profile < 0 || f->profile > 2)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "profile must be 0, 1 or 2");
    if (f->blend_split_len > 0 && f->blend_split_len < 256)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "blend_split_len must be 0, negative or >= 256");
    if (f->image_memory != NVGS_MEM_HOST && f->image_memory != NVGS_MEM_DEVICE)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "image_memory must be NVGS_MEM_HOST or NVGS_MEM_DEVICE");
    return NVGS_OK;
}

nvgs_status make_cam(nvgs_ctx* ctx, const nvgs_camera* c, const nvgs_render_flags* f, CamParams* cp) {
    if (!c) return fail(ctx, NVGS_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "image size %dx%d out of range", c->width, c->height);
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !(c->z_near > 0.f) || !std::isfinite(c->cx) ||
        !std::isfinite(c->cy))
        return fail(ctx, NVGS_ERR_INVALID_ARG, "camera intrinsics out of range");
    for (int k = 0; k < 9; k++)
        if (!std::isfinite(c->R[k])) return fail(ctx, NVGS_ERR_INVALID_ARG, "camera R not finite");
    for (int k = 0; k < 3; k++)
        if (!std::isfinite(c->t[k])) return fail(ctx, NVGS_ERR_INVALID_ARG, "camera t not finite");
    CamParams p{};
    memcpy(p.R, c->R, sizeof p.R);
    memcpy(p.t, c->t, sizeof p.t);
    p.fx = c->fx; p.fy = c->fy; p.cx = c->cx; p.cy = c->cy;
    p.W = c->width; p.H = c->height; p.z_near = c->z_near;
    p.lim_x = (float)(f->guard_band * (double)c->width / (2.0 * c->fx));
    p.lim_y = (float)(f->guard_band * (double)c->height / (2.0 * c->fy));
    p.f_r = (float)(2.0 * c->fx / c->width);
    p.alpha_min = f->alpha_min; p.alpha_max = f->alpha_max; p.t_stop = f->t_stop;
    p.dilation = f->dilation;
    for (int k = 0; k < 3; k++) p.bg[k] = f->bg[k];
    p.tile_size = f->tile_size;
    p.tiles_x = (c->width + f->tile_size - 1) / f->tile_size;
    p.tiles_y = (c->height + f->tile_size - 1) / f->tile_size;
    p.mlp_gate = f->mlp_gate ? 1 : 0;
    // the 1-sigma ellipse of Sigma_2D has area pi sqrt(det): area < A  <=>  det < (A / pi)^2
    const double clip = (double)f->radius_clip_area / 3.14159265358979323846;
    p.clip_det = (float)(clip * clip);
    *cp = p;
    return NVGS_OK;
}

nvgs_status upload_assets(nvgs_ctx* ctx) {
    if (!ctx->assets_dirty) return NVGS_OK;
    std::vector<AssetDev> h(ctx->assets.size());
    for (size_t k = 0; k < ctx->assets.size(); k++) h[k] = ctx->assets[k].dev;
    CK(ensure(ctx->assets_dev, h.size() * sizeof(AssetDev)));
    CK(cudaMemcpy(ctx->assets_dev.p, h.data(), h.size() * sizeof(AssetDev), cudaMemcpyHostToDevice));
    ctx->assets_dirty = false;
    return NVGS_OK;
}

// Stage boundaries of a frame: CUDA events when profiling, and always an NVTX range per stage
// (free unless a profiler is attached), so that tools can select S1-S6 by name.
const char* const kStageNvtx[NVGS_NUM_STAGES] = {"nvgs setup", "nvgs S1 cull", "nvgs S2 mlp",
                                                 "nvgs S3 compact", "nvgs S4 project", "nvgs S5 bin",
                                                 "nvgs S5 sort", "nvgs S6 blend"};
struct StageTimer {
    nvgs_ctx* ctx;
    bool on;
    bool range_open = false;
    void mark(int k) {
        if (on) cudaEventRecord(ctx->ev[k], ctx->stream);
        if (range_open) nvtxRangePop();
        range_open = k >= 0 && k < NVGS_NUM_STAGES;
        if (range_open) nvtxRangePushA(kStageNvtx[k]);
    }
    ~StageTimer() {
        if (range_open) nvtxRangePop();
    }
};

// Tensor-core MLP kernel of the frame: BF16 (FP8) when every asset with an MLP has BF16 (FP8)
// tiles and no logits are injected; otherwise -1 (the FP32 CUDA-core kernel).
int tc_mlp_precision(const nvgs_ctx* ctx, const nvgs_render_flags* f) {
    if (f->logits_override) return -1;
    int prec = -1;
    for (auto& a : ctx->assets) {
        if (a.precision < 0) continue;
        if (a.precision == NVGS_PREC_FP32) return -1;
        if (prec >= 0 && prec != a.precision) return -1;
        prec = a.precision;
    }
    return prec;
}

bool uses_tc_mlp(const nvgs_ctx* ctx, const nvgs_render_flags* f) { return tc_mlp_precision(ctx, f) >= 0; }

// S1 (+ S2 when use_mlp, + S3): fills ctx->vis_list / surv and the counts (counters[0] = in
// frustum, counters[1] = survivors).  `query` keeps the per-entry logits for
// nvgs_query_visibility.  Synchronous mode reads the counts back to size what follows; in
// device-count mode (`async`) nothing waits: every later kernel reads the count from the counters
// and the instanced-Gaussian count is the capacity (the MLP's timeout flag is read at the end of
// the batch).
// The frame instances a cull covers: the context's instances under one camera, or (multi-view
// batches) the (view, instance) pairs of fi_map with their chunk list.
struct CullScope {
    const Chunk* chunks;
    int n_chunks;
    int n_fi;
    const int2* fi_map;   // nullable
    uint64_t cap;         // instanced Gaussians over the frame instances
};

nvgs_status run_cull(nvgs_ctx* ctx, const CamParams* cam_dev, const nvgs_render_flags* f,
                     StageTimer& tm, uint32_t* n_vis_out, uint32_t* n_mlp_out, bool want_logits,
                     bool compact, bool async = false, const CullScope* scope = nullptr) {
    cudaStream_t s = ctx->stream;
    const CullScope sc = scope ? *scope
                               : CullScope{P<Chunk>(ctx->chunks), ctx->n_chunks, (int)ctx->instances.size(),
                                           nullptr, (uint64_t)ctx->n_instanced};
    const int n_inst = (int)ctx->instances.size();
    tm.mark(NVGS_STAGE_SETUP);
    CK(ensure(ctx->frame_inst, (size_t)sc.n_fi * sizeof(FrameInst)));
    CK(launch_instance_setup(P<InstanceRaw>(ctx->inst_raw), n_inst, P<AssetDev>(ctx->assets_dev), cam_dev,
                             P<FrameInst>(ctx->frame_inst), s, &ctx->log, sc.fi_map, sc.n_fi));
    tm.mark(NVGS_STAGE_CULL);
    const uint64_t cap = sc.cap;
    CK(ensure(ctx->bits, (size_t)sc.n_chunks * kChunkWords * 4));
    CK(ensure(ctx->chunk_counts, (size_t)sc.n_chunks * 4));
    CK(ensure(ctx->chunk_offsets, (size_t)sc.n_chunks * 4));
    CK(ensure(ctx->vis_list, cap * sizeof(uint2)));
    CK(ensure(ctx->scratch, std::max(scan_scratch_bytes(sc.n_chunks), scan_scratch_bytes(cap / kChunk + 1))));
    CK(launch_frustum(sc.chunks, sc.n_chunks, P<FrameInst>(ctx->frame_inst),
                      P<AssetDev>(ctx->assets_dev), cam_dev, P<uint32_t>(ctx->bits),
                      P<uint32_t>(ctx->chunk_counts), s, &ctx->log));
    uint32_t* counters = P<uint32_t>(ctx->counters);
    CK(exclusive_scan_u32(P<uint32_t>(ctx->chunk_counts), P<uint32_t>(ctx->chunk_offsets), sc.n_chunks,
                          &counters[0], ctx->scratch.p, s, &ctx->log));
    const bool tc_mlp = f->use_mlp && uses_tc_mlp(ctx, f);
    CK(launch_expand_chunks(sc.chunks, sc.n_chunks, P<uint32_t>(ctx->bits),
                            P<uint32_t>(ctx->chunk_offsets), P<uint2>(ctx->vis_list), s, &ctx->log));
    uint32_t n_vis_cap = (uint32_t)cap;
    const uint32_t* n_vis_dev = &counters[0];
    if (!async) {
        CK(cudaMemcpyAsync(ctx->h_counters, counters, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        n_vis_cap = ctx->h_counters[0];
        n_vis_dev = nullptr;
    }
    *n_vis_out = n_vis_cap;
    *n_mlp_out = 0;
    tm.mark(NVGS_STAGE_MLP);
    if (!f->use_mlp) {
        tm.mark(NVGS_STAGE_COMPACT);
        return NVGS_OK;
    }
    CK(ensure(ctx->keep_bits, ((size_t)cap / 32 + 2) * 4));
    if (want_logits) CK(ensure(ctx->logits_tmp, (size_t)cap * 4 + 16));
    if (tc_mlp) {
        if (!async) CK(cudaMemsetAsync(&counters[8], 0, 4, s));
        if (tc_mlp_precision(ctx, f) == NVGS_PREC_FP8)
            CK(launch_mlp_f8(P<uint2>(ctx->vis_list), n_vis_cap, n_vis_dev,
                             P<FrameInst>(ctx->frame_inst), P<AssetDev>(ctx->assets_dev), f->logit_threshold,
                             P<uint32_t>(ctx->keep_bits), want_logits ? P<float>(ctx->logits_tmp) : nullptr,
                             &counters[8], ctx->num_sms, s, &ctx->log));
        else
            CK(launch_mlp_tc(P<uint2>(ctx->vis_list), n_vis_cap, n_vis_dev,
                             P<FrameInst>(ctx->frame_inst),
                             P<AssetDev>(ctx->assets_dev), f->logit_threshold, P<uint32_t>(ctx->keep_bits),
                             want_logits ? P<float>(ctx->logits_tmp) : nullptr, &counters[8],
                             ctx->num_sms, f->mlp_ctas_per_sm, s, &ctx->log));
        if (!async) {
            CK(cudaMemcpyAsync(ctx->h_counters + 8, &counters[8], 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (ctx->h_counters[8])
                return fail(ctx, NVGS_ERR_TIMEOUT, "tensor-core MLP: a bounded mbarrier wait gave up");
        }
    } else {
        CK(launch_mlp_fp32(P<uint2>(ctx->vis_list), n_vis_cap, n_vis_dev, P<FrameInst>(ctx->frame_inst),
                           P<AssetDev>(ctx->assets_dev), f->logits_override, P<int64_t>(ctx->inst_offset),
                           f->logit_threshold, P<uint32_t>(ctx->keep_bits),
                           want_logits ? P<float>(ctx->logits_tmp) : nullptr, s, &ctx->log));
    }
    *n_mlp_out = n_vis_cap;
    tm.mark(NVGS_STAGE_COMPACT);
    if (!compact) return NVGS_OK;
    const uint32_t nb = (n_vis_cap + kChunk - 1) / kChunk;
    CK(ensure(ctx->block_counts, (size_t)nb * 4 + 16));
    CK(ensure(ctx->block_offsets, (size_t)nb * 4 + 16));
    CK(ensure(ctx->surv, cap * sizeof(uint2)));
    if (n_vis_cap > 0) {
        CK(launch_bit_counts(P<uint32_t>(ctx->keep_bits), n_vis_cap, n_vis_dev, P<uint32_t>(ctx->block_counts), s,
                             &ctx->log));
        CK(exclusive_scan_u32(P<uint32_t>(ctx->block_counts), P<uint32_t>(ctx->block_offsets), nb,
                              &counters[1], ctx->scratch.p, s, &ctx->log));
        CK(launch_compact_list(P<uint2>(ctx->vis_list), n_vis_cap, n_vis_dev, P<uint32_t>(ctx->keep_bits),
                               P<uint32_t>(ctx->block_offsets), P<uint2>(ctx->surv), s, &ctx->log));
    } else {
        CK(cudaMemsetAsync(&counters[1], 0, 4, s));
    }
    return NVGS_OK;
}

nvgs_status begin_frame(nvgs_ctx* ctx, bool record) {
    ctx->kept_frame = false;
    ctx->log.count = 0;
    ctx->log.n = 0;
    ctx->log.record = record;
    if (record && !ctx->log.ready) {
        for (int k = 0; k < 2 * LaunchLog::kMax; k++) CK(cudaEventCreate(&ctx->log.ev[k]));
        ctx->log.ready = true;
    }
    return NVGS_OK;
}

// Launch-log reset for calls that enqueue work outside a frame (no timing, kept frame untouched).
void begin_frame_log_only(nvgs_ctx* ctx) {
    ctx->log.count = 0;
    ctx->log.n = 0;
    ctx->log.record = false;
}

// After the frame's final synchronisation: fold the bracketed launches into per-kernel totals.
void end_frame(nvgs_ctx* ctx) {
    LaunchLog& L = ctx->log;
    if (!L.record) return;
    for (int k = 0; k < L.n; k++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, L.ev[2 * k], L.ev[2 * k + 1]) != cudaSuccess) continue;
        size_t j = 0;
        while (j < ctx->kname.size() && ctx->kname[j] != L.names[k]) j++;
        if (j == ctx->kname.size()) {
            ctx->kname.emplace_back(L.names[k]);
            ctx->kcount.push_back(0);
            ctx->kms.push_back(0.0);
        }
        ctx->kcount[j]++;
        ctx->kms[j] += ms;
    }
    L.n = 0;
}

// A graph key with the allocation count and the context's scene generation appended: a graph
// captured before a buffer was reallocated, or before the assets, MLPs or instances changed, never
// matches again.
static std::vector<uint8_t> graph_stamp(const nvgs_ctx* ctx, std::vector<uint8_t> key) {
    const uint64_t a = g_alloc_gen.load(), g = ctx->scene_gen;
    key.insert(key.end(), (const uint8_t*)&a, (const uint8_t*)&a + sizeof a);
    key.insert(key.end(), (const uint8_t*)&g, (const uint8_t*)&g + sizeof g);
    return key;
}

// Stage n camera records and copy them to ctx->cam_dev on the stream (the staging buffer is
// reused only after the previous copy has completed).
nvgs_status upload_cams(nvgs_ctx* ctx, const CamParams* cps, int n) {
    if (n > ctx->h_cam_cap) {
        if (ctx->cam_ev_pending) CK(cudaEventSynchronize(ctx->cam_ev));
        ctx->cam_ev_pending = false;
        if (ctx->h_cam) CK(cudaFreeHost(ctx->h_cam));
        ctx->h_cam = nullptr;
        const int cap = std::max(n, 64);
        CK(cudaMallocHost(&ctx->h_cam, (size_t)cap * sizeof(CamParams)));
        ctx->h_cam_cap = cap;
        g_alloc_gen.fetch_add(1);
        CK(ensure(ctx->cam_dev, (size_t)cap * sizeof(CamParams)));
    }
    if (!ctx->cam_ev) CK(cudaEventCreateWithFlags(&ctx->cam_ev, cudaEventDisableTiming));
    if (ctx->cam_ev_pending) CK(cudaEventSynchronize(ctx->cam_ev));
    memcpy(ctx->h_cam, cps, (size_t)n * sizeof(CamParams));
    CK(cudaMemcpyAsync(ctx->cam_dev.p, ctx->h_cam, (size_t)n * sizeof(CamParams), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaEventRecord(ctx->cam_ev, ctx->stream));
    ctx->cam_ev_pending = true;
    return NVGS_OK;
}

nvgs_status check_scene(nvgs_ctx* ctx) {
    if (ctx->instances.empty()) return fail(ctx, NVGS_ERR_INVALID_ARG, "no instances set");
    return upload_assets(ctx);
}

}  // namespace

// ============================================================================ context
extern "C" int nvgs_abi_version(void) { return NVGS_ABI_VERSION; }

extern "C" void nvgs_default_flags(nvgs_render_flags* f) {
    if (!f) return;
    memset(f, 0, sizeof *f);
    f->use_mlp = 1;
    f->mlp_gate = 1;
    f->logit_threshold = 0.0f;
    f->alpha_min = 1.0f / 255.0f;
    f->alpha_max = 0.99f;
    f->t_stop = 1e-4f;
    f->dilation = 0.3f;
    f->guard_band = 1.3f;
    f->tile_size = 16;
    f->image_memory = NVGS_MEM_DEVICE;
}

extern "C" nvgs_status nvgs_create(nvgs_ctx** out, int device, void* cuda_stream) {
    if (!out) return NVGS_ERR_INVALID_ARG;
    *out = nullptr;
    nvgs_ctx* ctx = new (std::nothrow) nvgs_ctx();
    if (!ctx) return NVGS_ERR_OOM;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || device < 0 || device >= n_dev) {
        delete ctx;
        return e != cudaSuccess ? NVGS_ERR_CUDA : NVGS_ERR_INVALID_ARG;
    }
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return NVGS_ERR_CUDA; }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        // blocking: ordered with the legacy default stream (the default stream of most callers)
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamDefault) != cudaSuccess) {
            delete ctx;
            return NVGS_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    if (ensure(ctx->counters, 128) != cudaSuccess ||
        cudaMallocHost(&ctx->h_counters, 128) != cudaSuccess) {
        delete ctx;
        return NVGS_ERR_OOM;
    }
    *out = ctx;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_destroy(nvgs_ctx* ctx) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& a : ctx->assets) {
        release(a.mean_op); release(a.scale_quat); release(a.sh);
        release(a.w_fp32); release(a.w_tc); release(a.w_f8);
    }
    DevBuf* bufs[] = {&ctx->assets_dev, &ctx->inst_raw, &ctx->inst_offset, &ctx->chunks,
                      &ctx->frame_inst, &ctx->bits, &ctx->chunk_counts, &ctx->chunk_offsets,
                      &ctx->vis_list, &ctx->keep_bits, &ctx->logits_tmp, &ctx->block_counts,
                      &ctx->block_offsets, &ctx->surv, &ctx->rec, &ctx->tile_counts,
                      &ctx->tile_offsets, &ctx->keys, &ctx->vals, &ctx->keys_alt, &ctx->vals_alt,
                      &ctx->ranges, &ctx->scratch, &ctx->counters, &ctx->image_tmp, &ctx->final_T,
                      &ctx->n_contrib, &ctx->mark, &ctx->tr_sv, &ctx->tr_sg, &ctx->tr_partial,
                      &ctx->dkey, &ctx->didx, &ctx->dkey_alt, &ctx->didx_alt, &ctx->split_scratch,
                      &ctx->grad_surv, &ctx->tile_order, &ctx->cam_dev, &ctx->view_stats,
                      &ctx->mv_fimap, &ctx->mv_chunks, &ctx->mv_images};
    for (auto& t : ctx->train) { release(t.w); release(t.m); release(t.v); release(t.views); }
    for (DevBuf* b : bufs) release(*b);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    if (ctx->h_cam) cudaFreeHost(ctx->h_cam);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->mv_graph_exec) cudaGraphExecDestroy(ctx->mv_graph_exec);
    if (ctx->cam_ev) cudaEventDestroy(ctx->cam_ev);
    if (ctx->events_ready)
        for (auto& ev : ctx->ev) cudaEventDestroy(ev);
    if (ctx->log.ready)
        for (int k = 0; k < 2 * LaunchLog::kMax; k++) cudaEventDestroy(ctx->log.ev[k]);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return NVGS_OK;
}

extern "C" const char* nvgs_last_error(const nvgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" void* nvgs_get_stream(const nvgs_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

// ============================================================================ scene
extern "C" nvgs_status nvgs_load_asset(nvgs_ctx* ctx, const nvgs_asset_desc* d, int* asset_id) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (!d || !asset_id) return fail(ctx, NVGS_ERR_INVALID_ARG, "desc / asset_id is NULL");
    if (d->n < 1 || d->n > (int64_t)1 << 31) return fail(ctx, NVGS_ERR_INVALID_ARG, "asset size %lld out of range", (long long)d->n);
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(ctx, NVGS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (!d->means || !d->log_scales || !d->quats || !d->opacity_logits || !d->sh)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset array is NULL");
    if (d->memory != NVGS_MEM_HOST && d->memory != NVGS_MEM_DEVICE)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset memory kind invalid");
    if (!(d->train_fov_x > 0.f && d->train_fov_x < 3.14159f))
        return fail(ctx, NVGS_ERR_INVALID_ARG, "train_fov_x must be in (0, pi)");
    CK(cudaSetDevice(ctx->device));
    const int64_t n = d->n;
    const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
    const int stride = (3 * K + 3) / 4 * 4;
    // stage the five arrays on the host (device inputs are copied down once at load time)
    std::vector<float> mh(n * 3), lh(n * 3), qh(n * 4), oh(n), sh(n * 3 * K);
    auto fetch = [&](std::vector<float>& dst, const float* src) -> cudaError_t {
        if (d->memory == NVGS_MEM_HOST) {
            memcpy(dst.data(), src, dst.size() * 4);
            return cudaSuccess;
        }
        return cudaMemcpy(dst.data(), src, dst.size() * 4, cudaMemcpyDeviceToHost);
    };
    CK(fetch(mh, d->means)); CK(fetch(lh, d->log_scales)); CK(fetch(qh, d->quats));
    CK(fetch(oh, d->opacity_logits)); CK(fetch(sh, d->sh));
    std::vector<float4> m4(n), sq4(2 * (size_t)n);
    std::vector<float> shp((size_t)n * stride, 0.0f);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t g = 0; g < n; g++) {
        for (int k = 0; k < 3; k++) {
            double v = mh[3 * g + k];
            if (!std::isfinite(v)) return fail(ctx, NVGS_ERR_INVALID_ARG, "non-finite mean at %lld", (long long)g);
            lo[k] = std::min(lo[k], v);
            hi[k] = std::max(hi[k], v);
        }
        m4[g] = make_float4(mh[3 * g], mh[3 * g + 1], mh[3 * g + 2], oh[g]);
        sq4[2 * g] = make_float4(lh[3 * g], lh[3 * g + 1], lh[3 * g + 2], 0.0f);
        sq4[2 * g + 1] = make_float4(qh[4 * g], qh[4 * g + 1], qh[4 * g + 2], qh[4 * g + 3]);
        memcpy(&shp[(size_t)g * stride], &sh[(size_t)g * 3 * K], 3 * K * sizeof(float));
    }
    AssetStore as;
    CK(ensure(as.mean_op, n * 16)); CK(ensure(as.scale_quat, n * 32));
    CK(ensure(as.sh, (size_t)n * stride * 4));
    CK(cudaMemcpy(as.mean_op.p, m4.data(), n * 16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(as.scale_quat.p, sq4.data(), n * 32, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(as.sh.p, shp.data(), (size_t)n * stride * 4, cudaMemcpyHostToDevice));
    AssetDev& a = as.dev;
    a.mean_op = P<float4>(as.mean_op); a.scale_quat = P<float4>(as.scale_quat);
    a.sh = P<float>(as.sh);
    a.w_fp32 = nullptr; a.w_tc = nullptr; a.w_f8 = nullptr;
    a.n = n; a.sh_degree = d->sh_degree; a.sh_stride = stride;
    double dd = 0.0;
    for (int k = 0; k < 3; k++) {
        double e = hi[k] - lo[k];
        a.bbox_c[k] = (float)(0.5 * (lo[k] + hi[k]));
        a.bbox_scale[k] = (float)(e > 0.0 ? 2.0 / e : 2.0);
        dd += e * e;
    }
    // half the box diagonal; a single point (zero box) keeps a tiny positive radius
    const double r = std::max(0.5 * std::sqrt(dd), 1e-6);
    // Eq. 1 (Sec. 3.1): d = r / (tan(theta_t / 2) p), p = 0.9 (near) and 0.05 (far)
    const double th = d->train_fov_x;
    const double pn = d->p_near > 0.f ? d->p_near : 0.9, pf = d->p_far > 0.f ? d->p_far : 0.05;
    const double dmin = d->d_min > 0.f ? d->d_min : r / (std::tan(th / 2.0) * pn);
    const double dmax = d->d_max > 0.f ? d->d_max : r / (std::tan(th / 2.0) * pf);
    if (!(dmax > dmin && dmin > 0.0)) return fail(ctx, NVGS_ERR_INVALID_ARG, "need 0 < d_min < d_max");
    a.bbox_r = (float)r;
    a.d_min = (float)dmin; a.d_max = (float)dmax;
    a.log_dmin = (float)std::log(dmin);
    a.inv_log_range = (float)(1.0 / (std::log(dmax) - std::log(dmin)));
    a.train_focal = (float)(1.0 / std::tan(th / 2.0));
    ctx->assets.push_back(as);
    ctx->assets_dirty = true;
    ctx->scene_gen++;
    *asset_id = (int)ctx->assets.size() - 1;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_set_mlp(nvgs_ctx* ctx, int asset_id, const float* w, int precision) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->assets.size())
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset_id %d out of range", asset_id);
    if (!w) return fail(ctx, NVGS_ERR_INVALID_ARG, "weights is NULL");
    if (precision != NVGS_PREC_FP32 && precision != NVGS_PREC_BF16 && precision != NVGS_PREC_FP8)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "precision must be NVGS_PREC_FP32, _BF16 or _FP8");
    for (int k = 0; k < kMlpWeights; k++)
        if (!std::isfinite(w[k])) return fail(ctx, NVGS_ERR_INVALID_ARG, "non-finite weight %d", k);
    CK(cudaSetDevice(ctx->device));
    AssetStore& as = ctx->assets[asset_id];
    CK(ensure(as.w_fp32, kMlpWeights * 4));
    CK(cudaMemcpy(as.w_fp32.p, w, kMlpWeights * 4, cudaMemcpyHostToDevice));
    as.dev.w_fp32 = P<float>(as.w_fp32);
    as.precision = NVGS_PREC_FP32;
    if (precision == NVGS_PREC_BF16) {
        const size_t nb = mlp_tc_weight_bytes();
        std::vector<uint8_t> packed(nb);
        mlp_tc_pack_weights(w, packed.data());
        CK(ensure(as.w_tc, nb));
        CK(cudaMemcpy(as.w_tc.p, packed.data(), nb, cudaMemcpyHostToDevice));
        as.dev.w_tc = P<uint8_t>(as.w_tc);
        as.precision = NVGS_PREC_BF16;
    } else if (precision == NVGS_PREC_FP8) {
        const size_t nb = mlp_f8_weight_bytes();
        std::vector<uint8_t> packed(nb);
        mlp_f8_pack_weights(w, packed.data(), nullptr);
        CK(ensure(as.w_f8, nb));
        CK(cudaMemcpy(as.w_f8.p, packed.data(), nb, cudaMemcpyHostToDevice));
        as.dev.w_f8 = P<uint8_t>(as.w_f8);
        as.precision = NVGS_PREC_FP8;
    }
    ctx->assets_dirty = true;
    ctx->scene_gen++;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_set_instances(nvgs_ctx* ctx, const nvgs_instance* inst, int count) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (count < 1 || !inst) return fail(ctx, NVGS_ERR_INVALID_ARG, "need at least one instance");
    std::vector<InstanceRaw> raw(count);
    std::vector<int64_t> off(count);
    std::vector<Chunk> chunks;
    int64_t total = 0;
    for (int i = 0; i < count; i++) {
        const nvgs_instance& x = inst[i];
        if (x.asset_id < 0 || x.asset_id >= (int)ctx->assets.size())
            return fail(ctx, NVGS_ERR_INVALID_ARG, "instance %d: asset_id %d not loaded", i, x.asset_id);
        if (!(x.s > 0.f) || !std::isfinite(x.s))
            return fail(ctx, NVGS_ERR_INVALID_ARG, "instance %d: scale must be > 0", i);
        for (int k = 0; k < 9; k++)
            if (!std::isfinite(x.R[k])) return fail(ctx, NVGS_ERR_INVALID_ARG, "instance %d: R not finite", i);
        memcpy(raw[i].R, x.R, sizeof raw[i].R);
        memcpy(raw[i].t, x.t, sizeof raw[i].t);
        raw[i].s = x.s;
        raw[i].asset = x.asset_id;
        off[i] = total;
        const int64_t n = ctx->assets[x.asset_id].dev.n;
        for (int64_t g0 = 0; g0 < n; g0 += kChunk)
            chunks.push_back(Chunk{i, (int)g0, (int)std::min<int64_t>(kChunk, n - g0), 0});
        total += n;
    }
    if (total >= ((int64_t)1 << 32) - 1)
        return fail(ctx, NVGS_ERR_CAPACITY, "more than 2^32 instanced Gaussians");
    CK(cudaSetDevice(ctx->device));
    CK(ensure(ctx->inst_raw, raw.size() * sizeof(InstanceRaw)));
    CK(ensure(ctx->inst_offset, off.size() * sizeof(int64_t)));
    CK(ensure(ctx->chunks, chunks.size() * sizeof(Chunk)));
    CK(cudaMemcpy(ctx->inst_raw.p, raw.data(), raw.size() * sizeof(InstanceRaw), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->inst_offset.p, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->chunks.p, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
    ctx->kept_frame = false;
    ctx->instances.assign(inst, inst + count);
    ctx->inst_offset_h = off;
    ctx->n_chunks = (int)chunks.size();
    ctx->n_instanced = total;
    ctx->scene_gen++;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_scene_info(const nvgs_ctx* ctx, int64_t* n_instanced, int* n_assets,
                                       int* n_instances) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (n_instanced) *n_instanced = ctx->n_instanced;
    if (n_assets) *n_assets = (int)ctx->assets.size();
    if (n_instances) *n_instances = (int)ctx->instances.size();
    return NVGS_OK;
}

// ============================================================================ per frame
extern "C" nvgs_status nvgs_query_visibility(nvgs_ctx* ctx, const nvgs_camera* cam,
                                             const nvgs_render_flags* f, float* logits,
                                             uint8_t* keep, nvgs_frame_stats* stats) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    nvgs_status st = validate_flags(ctx, f);
    if (st != NVGS_OK) return st;
    CamParams cp;
    if ((st = make_cam(ctx, cam, f, &cp)) != NVGS_OK) return st;
    CK(cudaSetDevice(ctx->device));
    if ((st = check_scene(ctx)) != NVGS_OK) return st;
    begin_frame(ctx, false);
    StageTimer tm{ctx, false};
    uint32_t n_vis = 0, n_mlp = 0;
    if ((st = upload_cams(ctx, &cp, 1)) != NVGS_OK) return st;
    if ((st = run_cull(ctx, P<CamParams>(ctx->cam_dev), f, tm, &n_vis, &n_mlp, true, false)) != NVGS_OK)
        return st;
    cudaStream_t s = ctx->stream;
    const uint64_t N = (uint64_t)ctx->n_instanced;
    if (keep) CK(cudaMemsetAsync(keep, 0, N, s));
    if (logits) CK(cudaMemsetAsync(logits, 0xff, N * 4, s));  // NaN pattern
    if (!f->use_mlp) {
        // keep = in frustum; no logits
        CK(ensure(ctx->keep_bits, (N / 32 + 2) * 4));
        CK(cudaMemsetAsync(ctx->keep_bits.p, 0xff, ((size_t)n_vis + 31) / 32 * 4, s));
    }
    CK(launch_scatter_visibility(P<uint2>(ctx->vis_list), n_vis, P<uint32_t>(ctx->keep_bits),
                                 f->use_mlp ? P<float>(ctx->logits_tmp) : nullptr,
                                 P<int64_t>(ctx->inst_offset), P<FrameInst>(ctx->frame_inst),
                                 f->use_mlp ? logits : nullptr, keep, s, &ctx->log));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->n_instanced = N;
        stats->n_in_frustum = n_vis;
        stats->n_mlp_queries = n_mlp;
        stats->kernel_launches = ctx->log.count;
    }
    return NVGS_OK;
}

// The whole pass for one camera.  labels_row (nullable, device, one byte per Gaussian of the
// scene's single instance) receives 1 for every Gaussian blended at some pixel (the labeller).
// S5 after the depth order: the survivors' pairs in that order (k_duplicate), sorted stably by tile
// id, and each tile's range.  Tile ids are 16-bit when the frame (or batch) has at most 65536
// tiles (12 instead of 16 bytes of key + value traffic per pair and radix pass).  n / n_dev: the
// survivor count (host, or a capacity with the count on the device); pair_cap: the pairs' count
// (synchronous path) or capacity; n_pairs_dev: the pair total on the device; sort_n_dev: null
// when pair_cap is the exact count, else n_pairs_dev.
struct SortedPairs {
    void* keys = nullptr;
    int key_bytes = 4;
    uint32_t* vals = nullptr;
    int passes = 0;
};
static nvgs_status bin_and_sort(nvgs_ctx* ctx, const uint32_t* order, uint32_t n, const uint32_t* n_dev,
                                const CamParams* cam_dev, const uint32_t* n_pairs_dev, uint64_t pair_cap,
                                uint32_t* overflow, const uint32_t* sort_n_dev, int n_tiles, int digit_bits,
                                int multi_view, cudaStream_t s, SortedPairs& out, StageTimer* tm = nullptr) {
    const int tile_bits = std::max(1, bit_width((uint64_t)n_tiles - 1));
    const int kb = n_tiles <= 65536 ? 2 : 4;
    CK(ensure(ctx->keys, (size_t)pair_cap * 4 + 16));
    CK(ensure(ctx->vals, (size_t)pair_cap * 4 + 16));
    CK(ensure(ctx->keys_alt, (size_t)pair_cap * 4 + 16));
    CK(ensure(ctx->vals_alt, (size_t)pair_cap * 4 + 16));
    CK(ensure(ctx->ranges, (size_t)n_tiles * 8));
    if (radix_scratch_bytes(pair_cap) > ctx->scratch.cap) CK(ensure(ctx->scratch, radix_scratch_bytes(pair_cap)));
    CK(launch_duplicate(order, P<float4>(ctx->rec), P<uint32_t>(ctx->tile_offsets), n, n_dev, cam_dev,
                        n_pairs_dev, (uint32_t)pair_cap, overflow, ctx->keys.p, kb, P<uint32_t>(ctx->vals),
                        ctx->num_sms, s, &ctx->log, multi_view));
    if (tm) tm->mark(NVGS_STAGE_SORT);
    int in_alt = 0;
    if (kb == 2)
        CK(radix_sort_pairs_u16(P<uint16_t>(ctx->keys), P<uint32_t>(ctx->vals), P<uint16_t>(ctx->keys_alt),
                                P<uint32_t>(ctx->vals_alt), pair_cap, tile_bits, ctx->scratch.p, s, &ctx->log,
                                &out.passes, 0, &in_alt, sort_n_dev, digit_bits));
    else
        CK(radix_sort_pairs_u32(P<uint32_t>(ctx->keys), P<uint32_t>(ctx->vals), P<uint32_t>(ctx->keys_alt),
                                P<uint32_t>(ctx->vals_alt), pair_cap, tile_bits, ctx->scratch.p, s, &ctx->log,
                                &out.passes, 0, &in_alt, sort_n_dev, digit_bits));
    out.keys = in_alt ? ctx->keys_alt.p : ctx->keys.p;
    out.vals = in_alt ? P<uint32_t>(ctx->vals_alt) : P<uint32_t>(ctx->vals);
    out.key_bytes = kb;
    CK(launch_tile_ranges(out.keys, kb, (uint32_t)pair_cap, sort_n_dev, (uint32_t)n_tiles,
                          P<uint32_t>(ctx->ranges), s, &ctx->log));
    return NVGS_OK;
}

static nvgs_status do_render(nvgs_ctx* ctx, const nvgs_camera* cam, const nvgs_render_flags* f,
                             float* image, nvgs_frame_stats* stats, uint8_t* labels_row) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    nvgs_status st = validate_flags(ctx, f);
    if (st != NVGS_OK) return st;
    if (!image) return fail(ctx, NVGS_ERR_INVALID_ARG, "image is NULL");
    CamParams cp;
    if ((st = make_cam(ctx, cam, f, &cp)) != NVGS_OK) return st;
    CK(cudaSetDevice(ctx->device));
    if ((st = check_scene(ctx)) != NVGS_OK) return st;
    cudaStream_t s = ctx->stream;
    if ((st = begin_frame(ctx, f->profile != 0)) != NVGS_OK) return st;
    if (f->profile && !ctx->events_ready) {
        for (auto& ev : ctx->ev) CK(cudaEventCreate(&ev));
        ctx->events_ready = true;
    }
    StageTimer tm{ctx, f->profile != 0};

    uint32_t n_vis = 0, n_mlp = 0;
    if ((st = upload_cams(ctx, &cp, 1)) != NVGS_OK) return st;
    const CamParams* cam_dev = P<CamParams>(ctx->cam_dev);
    if ((st = run_cull(ctx, cam_dev, f, tm, &n_vis, &n_mlp, false, true)) != NVGS_OK) return st;
    uint32_t* counters = P<uint32_t>(ctx->counters);
    uint32_t n_surv = n_vis;
    const uint2* surv = P<uint2>(ctx->vis_list);
    if (f->use_mlp) {
        CK(cudaMemcpyAsync(ctx->h_counters + 1, counters + 1, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        n_surv = ctx->h_counters[1];
        surv = P<uint2>(ctx->surv);
    }

    // ---- S4
    tm.mark(NVGS_STAGE_PROJECT);
    const uint64_t cap = (uint64_t)ctx->n_instanced;
    CK(ensure(ctx->rec, cap * 64 + 64));
    CK(ensure(ctx->tile_counts, cap * 4 + 16));
    CK(ensure(ctx->tile_offsets, cap * 4 + 16));
    CK(ensure(ctx->dkey, cap * 4 + 16));
    CK(ensure(ctx->didx, cap * 4 + 16));
    CK(ensure(ctx->dkey_alt, cap * 4 + 16));
    CK(ensure(ctx->didx_alt, cap * 4 + 16));
    CK(ensure(ctx->scratch, std::max({scan_scratch_bytes(ctx->n_chunks), scan_scratch_bytes(cap + 1),
                                      radix_scratch_bytes(n_surv)})));
    CK(launch_project(surv, n_surv, nullptr, P<FrameInst>(ctx->frame_inst), P<AssetDev>(ctx->assets_dev), cam_dev,
                      P<float4>(ctx->rec), P<uint32_t>(ctx->tile_counts),
                      P<uint32_t>(ctx->dkey), P<uint32_t>(ctx->didx), ctx->num_sms, s, &ctx->log));

    // ---- S5: survivors by depth, pairs in that order, pairs by tile, tile ranges
    tm.mark(NVGS_STAGE_BIN);
    int dpasses = 0, d_alt = 0;
    CK(radix_sort_pairs_u32(P<uint32_t>(ctx->dkey), P<uint32_t>(ctx->didx), P<uint32_t>(ctx->dkey_alt),
                            P<uint32_t>(ctx->didx_alt), n_surv, 32, ctx->scratch.p, s, &ctx->log,
                            &dpasses, 0, &d_alt, nullptr, f->sort_digit_bits ? f->sort_digit_bits : 8));
    const uint32_t* order = d_alt ? P<uint32_t>(ctx->didx_alt) : P<uint32_t>(ctx->didx);
    if (n_surv <= 1) order = P<uint32_t>(ctx->didx);
    CK(launch_gather_counts(order, P<uint32_t>(ctx->tile_counts), n_surv, nullptr, P<uint32_t>(ctx->tile_offsets),
                            ctx->num_sms, s, &ctx->log));
    CK(exclusive_scan_u32(P<uint32_t>(ctx->tile_offsets), P<uint32_t>(ctx->tile_offsets), n_surv,
                          counters + 2, ctx->scratch.p, s, &ctx->log));
    CK(cudaMemcpyAsync(ctx->h_counters + 2, counters + 2, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t n_pairs = n_surv ? ctx->h_counters[2] : 0u;
    const int n_tiles = cp.tiles_x * cp.tiles_y;
    SortedPairs sp;
    {
        const nvgs_status st = bin_and_sort(ctx, order, n_surv, nullptr, cam_dev, counters + 2, n_pairs, nullptr,
                                            nullptr, n_tiles, f->sort_digit_bits ? f->sort_digit_bits : 8, 0, s, sp,
                                            &tm);
        if (st != NVGS_OK) return st;
    }
    uint32_t* svals = sp.vals;
    int passes = sp.passes + dpasses;
    const int depth_bits = 0;

    // ---- S6
    tm.mark(NVGS_STAGE_BLEND);
    const size_t npx = (size_t)cp.W * cp.H;
    float* img_dev = image;
    bool copy_back = false;
    if (f->image_memory == NVGS_MEM_HOST) {
        // a page-locked host image that the device can address (and whose floats are aligned) is
        // written by the compositing kernels themselves (the transfer overlaps the compositing);
        // any other goes through a device buffer and one copy after the last kernel
        cudaPointerAttributes pa{};
        if (((uintptr_t)image & 3u) == 0 && cudaPointerGetAttributes(&pa, image) == cudaSuccess &&
            pa.type == cudaMemoryTypeHost && pa.devicePointer && ((uintptr_t)pa.devicePointer & 3u) == 0) {
            img_dev = static_cast<float*>(pa.devicePointer);
        } else {
            (void)cudaGetLastError();
            CK(ensure(ctx->image_tmp, npx * 12));
            img_dev = P<float>(ctx->image_tmp);
            copy_back = true;
        }
    }
    float* fT = nullptr;
    int32_t* nc = nullptr;
    if (f->keep_outputs) {
        CK(ensure(ctx->final_T, npx * 4));
        CK(ensure(ctx->n_contrib, npx * 4));
        fT = P<float>(ctx->final_T);
        nc = P<int32_t>(ctx->n_contrib);
    }
    uint8_t* mark = nullptr;
    if (labels_row) {
        CK(ensure(ctx->mark, (size_t)n_surv + 16));
        mark = P<uint8_t>(ctx->mark);
        CK(cudaMemsetAsync(mark, 0, (size_t)n_surv + 1, s));
    }
    // dense tiles: chunks of split_len pairs on separate CTAs (flags.blend_split_len; < 0 = never
    // split; 0 = automatic: tiles longer than four times the mean, and at least 4096 pairs --
    // splitting pays only where a few tiles would otherwise hold up the whole grid)
    const uint64_t auto_len = std::max<uint64_t>(4096, 4 * ((uint64_t)n_pairs / (uint64_t)n_tiles + 1));
    const uint32_t split_len = f->blend_split_len < 0 ? 0xffffffffu
                               : (f->blend_split_len == 0 ? (uint32_t)std::min<uint64_t>(auto_len, 0x7fffffffu)
                                                          : (uint32_t)f->blend_split_len);
    if (n_pairs > split_len) {
        CK(ensure(ctx->split_scratch, blend_split_scratch_bytes(n_tiles, n_pairs, cp.tile_size, split_len)));
        CK(ensure(ctx->scratch, scan_scratch_bytes(n_tiles)));
    }
    // profile 2: S6's (pixel, fragment) evaluations and composited fragments in counters[16..19]
    unsigned long long* evals = f->profile >= 2 ? reinterpret_cast<unsigned long long*>(counters + 16) : nullptr;
    if (evals) CK(cudaMemsetAsync(evals, 0, 16, s));
    CK(ensure(ctx->tile_order, (size_t)n_tiles * 4 + 16));
    CK(launch_blend(P<uint32_t>(ctx->ranges), svals, P<float4>(ctx->rec), cp, cam_dev, img_dev, fT, nc, mark,
                    split_len, n_pairs, nullptr, ctx->split_scratch.p, ctx->scratch.p, ctx->num_sms, evals,
                    s, &ctx->log, 1, nullptr, 0, P<uint32_t>(ctx->tile_order)));
    if (evals) CK(cudaMemcpyAsync(ctx->h_counters + 16, counters + 16, 16, cudaMemcpyDeviceToHost, s));
    if (labels_row) CK(launch_mark_labels(surv, n_surv, mark, labels_row, s, &ctx->log));
    tm.mark(NVGS_NUM_STAGES);
    if (copy_back) CK(cudaMemcpyAsync(image, img_dev, npx * 12, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    end_frame(ctx);

    nvgs_frame_view& L = ctx->last;
    L.survivors = reinterpret_cast<const uint32_t*>(surv);
    L.records = P<float>(ctx->rec);
    L.tile_rects = P<int32_t>(ctx->rec) + 12;   // inside the records, 16 int32 apart
    L.pair_values = svals;
    L.pair_keys = sp.keys;
    L.pair_key_bytes = sp.key_bytes;
    L.tile_ranges = P<uint32_t>(ctx->ranges);
    L.final_T = fT;
    L.n_contrib = nc;
    L.n_survivors = n_surv;
    L.n_pairs = n_pairs;
    L.tiles_x = cp.tiles_x; L.tiles_y = cp.tiles_y; L.tile_size = cp.tile_size;
    L.depth_bits = depth_bits;
    ctx->last_cp = cp;
    ctx->kept_frame = f->keep_outputs != 0 && !labels_row;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->n_instanced = (uint64_t)ctx->n_instanced;
        stats->n_in_frustum = n_vis;
        stats->n_mlp_queries = n_mlp;
        stats->n_survivors = n_surv;
        stats->n_pairs = n_pairs;
        stats->sort_passes = (uint32_t)passes;
        stats->kernel_launches = ctx->log.count;
        if (f->profile) {
            if (f->profile >= 2) {
                uint64_t ev[2] = {0, 0};
                memcpy(ev, ctx->h_counters + 16, 16);
                stats->blend_evaluations = ev[0];
                stats->blend_composited = ev[1];
            }
            for (int k = 0; k < NVGS_NUM_STAGES; k++) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ctx->ev[k], ctx->ev[k + 1]);
                stats->stage_ms[k] = ms;
            }
        }
    }
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_render(nvgs_ctx* ctx, const nvgs_camera* cam, const nvgs_render_flags* f,
                                   float* image, nvgs_frame_stats* stats) {
    return do_render(ctx, cam, f, image, stats, nullptr);
}

// ============================================================================ N1: labeller + trainer
extern "C" nvgs_status nvgs_label_visibility(nvgs_ctx* ctx, int asset_id, const nvgs_camera* views,
                                             int n_views, int group, const nvgs_render_flags* flags,
                                             uint8_t* labels) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->assets.size())
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset_id %d out of range", asset_id);
    if (!views || n_views < 1 || group < 1 || n_views % group != 0 || !labels)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "need views, n_views >= 1 divisible by group >= 1, labels");
    nvgs_status st = validate_flags(ctx, flags);
    if (st != NVGS_OK) return st;
    CK(cudaSetDevice(ctx->device));
    // render the asset alone (identity instance, no MLP), then restore the caller's scene
    const std::vector<nvgs_instance> saved = ctx->instances;
    nvgs_instance one{};
    one.asset_id = asset_id;
    one.R[0] = one.R[4] = one.R[8] = 1.0f;
    one.s = 1.0f;
    if ((st = nvgs_set_instances(ctx, &one, 1)) != NVGS_OK) return st;
    nvgs_render_flags fl = *flags;
    fl.use_mlp = 0;
    fl.image_memory = NVGS_MEM_DEVICE;
    fl.logits_override = nullptr;
    fl.keep_outputs = 0;
    const int64_t n = ctx->assets[asset_id].dev.n;
    CK(cudaMemsetAsync(labels, 0, (size_t)(n_views / group) * n, ctx->stream));
    for (int v = 0; v < n_views && st == NVGS_OK; v++) {
        const size_t npx = (size_t)views[v].width * views[v].height;
        if (ensure(ctx->image_tmp, npx * 12) != cudaSuccess) { st = fail(ctx, NVGS_ERR_OOM, "labeller image"); break; }
        st = do_render(ctx, &views[v], &fl, P<float>(ctx->image_tmp), nullptr,
                       labels + (size_t)(v / group) * n);
    }
    nvgs_status st2 = saved.empty() ? NVGS_OK : nvgs_set_instances(ctx, saved.data(), (int)saved.size());
    if (saved.empty()) { ctx->instances.clear(); ctx->n_instanced = 0; ctx->n_chunks = 0; ctx->scene_gen++; }
    return st != NVGS_OK ? st : st2;
}

extern "C" nvgs_status nvgs_train_init(nvgs_ctx* ctx, int asset_id, const float* w0,
                                       const nvgs_camera* views, int n_views) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->assets.size())
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset_id %d out of range", asset_id);
    if (!w0 || !views || n_views < 1) return fail(ctx, NVGS_ERR_INVALID_ARG, "weights / views missing");
    CK(cudaSetDevice(ctx->device));
    if (ctx->train.size() < ctx->assets.size()) ctx->train.resize(ctx->assets.size());
    auto& T = ctx->train[asset_id];
    CK(ensure(T.w, kMlpWeights * 4));
    CK(ensure(T.m, kMlpWeights * 4));
    CK(ensure(T.v, kMlpWeights * 4));
    CK(ensure(T.views, (size_t)n_views * 16));
    CK(cudaMemcpy(T.w.p, w0, kMlpWeights * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(T.m.p, 0, kMlpWeights * 4));
    CK(cudaMemset(T.v.p, 0, kMlpWeights * 4));
    const float f_t = ctx->assets[asset_id].dev.train_focal;
    std::vector<float4> vt(n_views);
    for (int v = 0; v < n_views; v++) {
        const nvgs_camera& c = views[v];
        if (!(c.fx > 0.f) || c.width < 1) return fail(ctx, NVGS_ERR_INVALID_ARG, "view %d invalid", v);
        double cc[3];
        for (int q = 0; q < 3; q++)   // camera centre -R^T t (the asset frame is the world frame)
            cc[q] = -((double)c.R[q] * c.t[0] + (double)c.R[3 + q] * c.t[1] + (double)c.R[6 + q] * c.t[2]);
        const double f_view = 2.0 * c.fx / c.width;
        vt[v] = make_float4((float)cc[0], (float)cc[1], (float)cc[2], (float)(f_t / f_view));
    }
    CK(cudaMemcpy(T.views.p, vt.data(), (size_t)n_views * 16, cudaMemcpyHostToDevice));
    T.n_views = n_views;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_train_visibility_step(nvgs_ctx* ctx, int asset_id, const nvgs_train_batch* b,
                                                  const nvgs_adam_cfg* adam, float* loss_out) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->train.size() || !ctx->train[asset_id].n_views)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset %d has no training state (nvgs_train_init)", asset_id);
    if (!b || !adam || !b->labels || b->batch < 1 || (!b->sample_view) != (!b->sample_gauss))
        return fail(ctx, NVGS_ERR_INVALID_ARG, "bad batch");
    if (b->precision != NVGS_PREC_FP32 && b->precision != NVGS_PREC_BF16)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "batch precision must be NVGS_PREC_FP32 or NVGS_PREC_BF16");
    if (!(adam->lr >= 0.f) || !(adam->beta1 >= 0.f && adam->beta1 < 1.f) ||
        !(adam->beta2 >= 0.f && adam->beta2 < 1.f) || !(adam->eps > 0.f) || adam->step < 0)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "bad Adam configuration");
    CK(cudaSetDevice(ctx->device));
    auto& T = ctx->train[asset_id];
    const uint32_t B = (uint32_t)b->batch;
    const bool expl = b->sample_view != nullptr;
    CK(ensure(ctx->tr_sv, (size_t)B * 4));
    CK(ensure(ctx->tr_sg, (size_t)B * 4));
    CK(ensure(ctx->tr_partial, train_partial_bytes(B)));
    cudaStream_t s = ctx->stream;
    if (expl) {
        CK(cudaMemcpyAsync(ctx->tr_sv.p, b->sample_view, (size_t)B * 4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->tr_sg.p, b->sample_gauss, (size_t)B * 4, cudaMemcpyDeviceToDevice, s));
    }
    {
        const nvgs_status ust = upload_assets(ctx);
        if (ust != NVGS_OK) return ust;
    }
    uint32_t* counters = P<uint32_t>(ctx->counters);
    ctx->log.count = 0;
    const bool tc = b->precision == NVGS_PREC_BF16;
    if (tc) CK(cudaMemsetAsync(&counters[12], 0, 4, s));
    CK(launch_train_step(P<AssetDev>(ctx->assets_dev) + asset_id, (uint32_t)ctx->assets[asset_id].dev.n,
                         P<float4>(T.views), (uint32_t)T.n_views, b->labels, B, b->seed,
                         (uint32_t)adam->step, P<int32_t>(ctx->tr_sv), P<int32_t>(ctx->tr_sg), expl ? 1 : 0,
                         &counters[10], reinterpret_cast<float*>(&counters[11]), P<float>(ctx->tr_partial),
                         P<float>(T.w), P<float>(T.m), P<float>(T.v), adam->lr, adam->beta1, adam->beta2,
                         adam->eps, tc ? 1 : 0, &counters[12], s, &ctx->log));
    if (loss_out) {
        CK(cudaMemcpyAsync(ctx->h_counters + 11, &counters[11], 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        memcpy(loss_out, ctx->h_counters + 11, 4);
        if (tc && ctx->h_counters[12])
            return fail(ctx, NVGS_ERR_TIMEOUT, "tensor-core training step: a bounded mbarrier wait gave up");
    }
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_train_get_weights(nvgs_ctx* ctx, int asset_id, float* w_out) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->train.size() || !ctx->train[asset_id].n_views || !w_out)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset %d has no training state", asset_id);
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(w_out, ctx->train[asset_id].w.p, kMlpWeights * 4, cudaMemcpyDeviceToHost));
    return NVGS_OK;
}

static_assert(NVGS_TRAIN_STATE_FLOATS == 3 * kMlpWeights, "checkpoint size");

extern "C" nvgs_status nvgs_train_save_state(nvgs_ctx* ctx, int asset_id, float* out) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->train.size() || !ctx->train[asset_id].n_views || !out)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset %d has no training state", asset_id);
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const auto& T = ctx->train[asset_id];
    CK(cudaMemcpy(out, T.w.p, kMlpWeights * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out + kMlpWeights, T.m.p, kMlpWeights * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out + 2 * kMlpWeights, T.v.p, kMlpWeights * 4, cudaMemcpyDeviceToHost));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_train_load_state(nvgs_ctx* ctx, int asset_id, const float* in) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->train.size() || !ctx->train[asset_id].n_views || !in)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset %d has no training state", asset_id);
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    auto& T = ctx->train[asset_id];
    CK(cudaMemcpy(T.w.p, in, kMlpWeights * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(T.m.p, in + kMlpWeights, kMlpWeights * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(T.v.p, in + 2 * kMlpWeights, kMlpWeights * 4, cudaMemcpyHostToDevice));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_get_asset_info(const nvgs_ctx* ctx, int asset_id, nvgs_asset_info* out) {
    if (!ctx || !out || asset_id < 0 || asset_id >= (int)ctx->assets.size()) return NVGS_ERR_INVALID_ARG;
    const AssetDev& a = ctx->assets[asset_id].dev;
    out->n = a.n;
    out->sh_degree = a.sh_degree;
    for (int k = 0; k < 3; k++) {
        out->bbox_center[k] = a.bbox_c[k];
        out->bbox_half_extent[k] = 1.0f / a.bbox_scale[k];
    }
    out->d_min = a.d_min;
    out->d_max = a.d_max;
    out->train_fov_x = (float)(2.0 * std::atan(1.0 / a.train_focal));
    out->has_mlp = ctx->assets[asset_id].precision;
    return NVGS_OK;
}

// Training cameras of Sec. 3.1 / 4.1: n_dirs directions on a Fibonacci sphere around the box
// centre, each at n_dist distances log-spaced from d_min to d_max (one distance: d_min), looking
// at the centre with the asset's training field of view.  Direction-major order.
extern "C" nvgs_status nvgs_training_views(const nvgs_ctx* ctx, int asset_id, int n_dirs, int n_dist,
                                           int width, int height, nvgs_camera* out) {
    if (!ctx || !out || asset_id < 0 || asset_id >= (int)ctx->assets.size() || n_dirs < 1 ||
        n_dist < 1 || width < 1 || height < 1)
        return NVGS_ERR_INVALID_ARG;
    const AssetDev& a = ctx->assets[asset_id].dev;
    const double golden = M_PI * (3.0 - std::sqrt(5.0));
    const double fx = (width / 2.0) * a.train_focal;   // (W/2) / tan(theta_t / 2)
    for (int k = 0; k < n_dirs; k++) {
        const double y = 1.0 - 2.0 * (k + 0.5) / n_dirs;
        const double rad = std::sqrt(std::max(0.0, 1.0 - y * y));
        const double ph = golden * k;
        const double dir[3] = {rad * std::cos(ph), y, rad * std::sin(ph)};
        for (int j = 0; j < n_dist; j++) {
            const double u = n_dist > 1 ? (double)j / (n_dist - 1) : 0.0;
            const double d = a.d_min * std::pow((double)a.d_max / a.d_min, u);
            double eye[3], f[3], r[3], dn[3];
            for (int q = 0; q < 3; q++) { eye[q] = a.bbox_c[q] + d * dir[q]; f[q] = -dir[q]; }
            // right = f x up (up = +y, or +z when looking along y), down = f x right
            double up[3] = {0.0, 1.0, 0.0};
            if (std::fabs(f[1]) > 0.999) { up[1] = 0.0; up[2] = 1.0; }
            r[0] = f[1] * up[2] - f[2] * up[1]; r[1] = f[2] * up[0] - f[0] * up[2]; r[2] = f[0] * up[1] - f[1] * up[0];
            const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            for (int q = 0; q < 3; q++) r[q] /= rn;
            dn[0] = f[1] * r[2] - f[2] * r[1]; dn[1] = f[2] * r[0] - f[0] * r[2]; dn[2] = f[0] * r[1] - f[1] * r[0];
            nvgs_camera& c = out[k * n_dist + j];
            const double* rows[3] = {r, dn, f};
            for (int p = 0; p < 3; p++) {
                for (int q = 0; q < 3; q++) c.R[3 * p + q] = (float)rows[p][q];
                c.t[p] = (float)(-(rows[p][0] * eye[0] + rows[p][1] * eye[1] + rows[p][2] * eye[2]));
            }
            c.fx = c.fy = (float)fx;
            c.cx = width / 2.0f;
            c.cy = height / 2.0f;
            c.width = width;
            c.height = height;
            c.z_near = 0.2f;
        }
    }
    return NVGS_OK;
}

namespace {
// Camera at `eye` looking along f (unit): rows right, down, forward (right = f x up, with up = +y,
// or +z when looking along y).
void look_along(const double* eye, const double* f, int width, int height, double fx, nvgs_camera& c,
                double* right = nullptr, double* down = nullptr) {
    double r[3], dn[3];
    double up[3] = {0.0, 1.0, 0.0};
    if (std::fabs(f[1]) > 0.999) { up[1] = 0.0; up[2] = 1.0; }
    r[0] = f[1] * up[2] - f[2] * up[1]; r[1] = f[2] * up[0] - f[0] * up[2]; r[2] = f[0] * up[1] - f[1] * up[0];
    const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int q = 0; q < 3; q++) r[q] /= rn;
    dn[0] = f[1] * r[2] - f[2] * r[1]; dn[1] = f[2] * r[0] - f[0] * r[2]; dn[2] = f[0] * r[1] - f[1] * r[0];
    const double* rows[3] = {r, dn, f};
    for (int p = 0; p < 3; p++) {
        for (int q = 0; q < 3; q++) c.R[3 * p + q] = (float)rows[p][q];
        c.t[p] = (float)(-(rows[p][0] * eye[0] + rows[p][1] * eye[1] + rows[p][2] * eye[2]));
    }
    c.fx = c.fy = (float)fx;
    c.cx = width / 2.0f;
    c.cy = height / 2.0f;
    c.width = width;
    c.height = height;
    c.z_near = 0.2f;
    if (right) for (int q = 0; q < 3; q++) right[q] = r[q];
    if (down) for (int q = 0; q < 3; q++) down[q] = dn[q];
}

// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", 2014).
uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
double unit_uniform(uint64_t bits) { return (double)(bits >> 11) * (1.0 / 9007199254740992.0); }
}  // namespace

extern "C" nvgs_status nvgs_training_views_ex(const nvgs_ctx* ctx, int asset_id, const nvgs_view_opts* o,
                                              nvgs_camera* out) {
    if (!ctx || !o || !out || asset_id < 0 || asset_id >= (int)ctx->assets.size() || o->n_dirs < 1 ||
        o->n_dist < 1 || o->width < 1 || o->height < 1 || o->n_aux < 0 || o->n_aux > 64 ||
        (o->n_aux > 0 && !(o->aux_angle > 0.0f && o->aux_angle < 1.5f)))
        return NVGS_ERR_INVALID_ARG;
    const AssetDev& a = ctx->assets[asset_id].dev;
    const double golden = M_PI * (3.0 - std::sqrt(5.0));
    const double fx = (o->width / 2.0) * a.train_focal;   // (W/2) / tan(theta_t / 2)
    const int group = 1 + o->n_aux;
    for (int k = 0; k < o->n_dirs; k++) {
        const double y = 1.0 - 2.0 * (k + 0.5) / o->n_dirs;
        const double rad = std::sqrt(std::max(0.0, 1.0 - y * y));
        const double ph = golden * k;
        const double dir[3] = {rad * std::cos(ph), y, rad * std::sin(ph)};
        for (int j = 0; j < o->n_dist; j++) {
            const double u = o->n_dist > 1 ? (double)j / (o->n_dist - 1) : 0.0;
            const double d = a.d_min * std::pow((double)a.d_max / a.d_min, u);
            const int view = k * o->n_dist + j;
            double eye[3], f[3], r[3], dn[3];
            for (int q = 0; q < 3; q++) { eye[q] = a.bbox_c[q] + d * dir[q]; f[q] = -dir[q]; }
            nvgs_camera& c = out[(size_t)view * group];
            look_along(eye, f, o->width, o->height, fx, c, r, dn);
            if (o->random_offset) {
                // s(d): 0 at d_min, d_min / d_max at d_max, linear in d
                const double t = a.d_max > a.d_min ? (d - a.d_min) / ((double)a.d_max - a.d_min) : 0.0;
                const double s = t * (double)a.d_min / a.d_max;
                const uint64_t h = splitmix64(o->seed ^ splitmix64((uint64_t)view));
                const double oa = 2.0 * unit_uniform(h) - 1.0, ob = 2.0 * unit_uniform(splitmix64(h)) - 1.0;
                for (int q = 0; q < 3; q++) eye[q] += (oa * r[q] + ob * dn[q]) * s * d;
                look_along(eye, f, o->width, o->height, fx, c);
            }
            // auxiliary views: directions on the cone of half-angle aux_angle around dir, same distance
            for (int m = 0; m < o->n_aux; m++) {
                const double phi = 2.0 * M_PI * m / o->n_aux;
                const double cb = std::cos((double)o->aux_angle), sb = std::sin((double)o->aux_angle);
                double ad[3], aeye[3], af[3];
                for (int q = 0; q < 3; q++) ad[q] = cb * dir[q] + sb * (std::cos(phi) * r[q] + std::sin(phi) * dn[q]);
                const double an = std::sqrt(ad[0] * ad[0] + ad[1] * ad[1] + ad[2] * ad[2]);
                for (int q = 0; q < 3; q++) { ad[q] /= an; aeye[q] = a.bbox_c[q] + d * ad[q]; af[q] = -ad[q]; }
                look_along(aeye, af, o->width, o->height, fx, out[(size_t)view * group + 1 + m]);
            }
        }
    }
    return NVGS_OK;
}

extern "C" float nvgs_lr_schedule(int step, int total, float lr0, float lr1, float warmup_frac) {
    if (total <= 0) return lr0;
    const double tw = std::max(1.0, (double)warmup_frac * total);
    if (step < tw) return (float)(lr0 * 0.5 * (1.0 - std::cos(M_PI * (step + 1) / tw)));
    const double u = std::min(1.0, (step - tw) / std::max(1.0, total - tw));
    return (float)(lr0 * std::pow((double)lr1 / lr0, u));
}

// ============================================================================ batched views
// One view of a batch in device-count mode: the S1-S6 pass of do_render with every count read on
// the device (counters) and every size a capacity, so that nothing here waits for the GPU.
static nvgs_status enqueue_view_async(nvgs_ctx* ctx, const CamParams& cp, const CamParams* cam_dev,
                                      const nvgs_render_flags* f, float* image, uint64_t pair_cap,
                                      uint32_t* view_counts) {
    cudaStream_t s = ctx->stream;
    StageTimer tm{ctx, false};
    uint32_t n_vis = 0, n_mlp = 0;
    nvgs_status st = run_cull(ctx, cam_dev, f, tm, &n_vis, &n_mlp, false, true, true);
    if (st != NVGS_OK) return st;
    uint32_t* counters = P<uint32_t>(ctx->counters);
    const uint64_t cap = (uint64_t)ctx->n_instanced;
    const uint2* surv = f->use_mlp ? P<uint2>(ctx->surv) : P<uint2>(ctx->vis_list);
    const uint32_t* n_surv_dev = f->use_mlp ? &counters[1] : &counters[0];
    // S4
    CK(ensure(ctx->rec, cap * 64 + 64));
    CK(ensure(ctx->tile_counts, cap * 4 + 16));
    CK(ensure(ctx->tile_offsets, cap * 4 + 16));
    CK(ensure(ctx->dkey, cap * 4 + 16));
    CK(ensure(ctx->didx, cap * 4 + 16));
    CK(ensure(ctx->dkey_alt, cap * 4 + 16));
    CK(ensure(ctx->didx_alt, cap * 4 + 16));
    CK(ensure(ctx->scratch, std::max({scan_scratch_bytes(ctx->n_chunks), scan_scratch_bytes(cap + 1),
                                      radix_scratch_bytes(cap), radix_scratch_bytes(pair_cap)})));
    CK(launch_project(surv, (uint32_t)cap, n_surv_dev, P<FrameInst>(ctx->frame_inst), P<AssetDev>(ctx->assets_dev),
                      cam_dev, P<float4>(ctx->rec), P<uint32_t>(ctx->tile_counts),
                      P<uint32_t>(ctx->dkey), P<uint32_t>(ctx->didx), ctx->num_sms, s, &ctx->log));
    // S5
    int dpasses = 0, d_alt = 0;
    CK(radix_sort_pairs_u32(P<uint32_t>(ctx->dkey), P<uint32_t>(ctx->didx), P<uint32_t>(ctx->dkey_alt),
                            P<uint32_t>(ctx->didx_alt), cap, 32, ctx->scratch.p, s, &ctx->log, &dpasses, 0,
                            &d_alt, n_surv_dev, f->sort_digit_bits ? f->sort_digit_bits : 8));
    const uint32_t* order = d_alt ? P<uint32_t>(ctx->didx_alt) : P<uint32_t>(ctx->didx);
    CK(launch_gather_counts(order, P<uint32_t>(ctx->tile_counts), (uint32_t)cap, n_surv_dev,
                            P<uint32_t>(ctx->tile_offsets), ctx->num_sms, s, &ctx->log));
    CK(exclusive_scan_u32(P<uint32_t>(ctx->tile_offsets), P<uint32_t>(ctx->tile_offsets), cap, counters + 2,
                          ctx->scratch.p, s, &ctx->log, n_surv_dev));
    const int n_tiles = cp.tiles_x * cp.tiles_y;
    SortedPairs sp;
    {
        const nvgs_status st = bin_and_sort(ctx, order, (uint32_t)cap, n_surv_dev, cam_dev, counters + 2, pair_cap,
                                            counters + 9, counters + 2, n_tiles,
                                            f->sort_digit_bits ? f->sort_digit_bits : 8, 0, s, sp);
        if (st != NVGS_OK) return st;
    }
    uint32_t* svals = sp.vals;
    // S6.  The automatic split length depends on the frame's pair count, which only the device
    // knows here: it is resolved there with the synchronous path's rule (so both paths split the
    // same tiles and give the same image), and the scratch is sized for its lower bound 4096.
    const bool auto_split = f->blend_split_len == 0;
    const uint32_t split_len = f->blend_split_len < 0 ? 0xffffffffu
                               : (auto_split ? 4096u : (uint32_t)f->blend_split_len);
    if (pair_cap > split_len) {
        CK(ensure(ctx->split_scratch, blend_split_scratch_bytes(n_tiles, pair_cap, cp.tile_size, split_len)));
        CK(ensure(ctx->scratch, scan_scratch_bytes(n_tiles)));
    }
    CK(ensure(ctx->tile_order, (size_t)n_tiles * 4 + 16));
    CK(launch_blend(P<uint32_t>(ctx->ranges), svals, P<float4>(ctx->rec), cp, cam_dev, image, nullptr, nullptr,
                    nullptr, split_len, pair_cap, auto_split ? counters + 2 : nullptr, ctx->split_scratch.p,
                    ctx->scratch.p, ctx->num_sms, nullptr, s, &ctx->log, 1, nullptr, 0, P<uint32_t>(ctx->tile_order)));
    // this view's counts
    CK(cudaMemcpyAsync(view_counts, counters, 3 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return NVGS_OK;
}

static nvgs_status enqueue_batch(nvgs_ctx* ctx, const std::vector<CamParams>& cps, float* const* images,
                                 const nvgs_render_flags* f, uint64_t pair_cap) {
    cudaStream_t s = ctx->stream;
    uint32_t* counters = P<uint32_t>(ctx->counters);
    CK(cudaMemsetAsync(&counters[8], 0, 8, s));   // MLP timeout flag, pair overflow flag
    for (size_t v = 0; v < cps.size(); v++) {
        nvgs_status st = enqueue_view_async(ctx, cps[v], P<CamParams>(ctx->cam_dev) + v, f, images[v], pair_cap,
                                            P<uint32_t>(ctx->view_stats) + 4 * v);
        if (st != NVGS_OK) return st;
    }
    CK(cudaMemcpyAsync(P<uint32_t>(ctx->view_stats) + 4 * cps.size(), &counters[8], 8, cudaMemcpyDeviceToDevice, s));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_render_batch(nvgs_ctx* ctx, const nvgs_camera* cams, int n_views,
                                         float* const* images, const nvgs_render_flags* f,
                                         const nvgs_batch_opts* opts, nvgs_frame_stats* stats) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    nvgs_status st = validate_flags(ctx, f);
    if (st != NVGS_OK) return st;
    if (!cams || !images || n_views < 1 || n_views > 4096)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "need 1..4096 cameras and image pointers");
    if (f->image_memory != NVGS_MEM_DEVICE || f->keep_outputs || f->profile)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "batched views need device images, no kept outputs, no profiling");
    for (int v = 0; v < n_views; v++)
        if (!images[v]) return fail(ctx, NVGS_ERR_INVALID_ARG, "image %d is NULL", v);
    nvgs_batch_opts o{};
    if (opts) o = *opts;
    if (o.max_pairs < 0) return fail(ctx, NVGS_ERR_INVALID_ARG, "max_pairs must be >= 0");
    std::vector<CamParams> cps(n_views);
    for (int v = 0; v < n_views; v++)
        if ((st = make_cam(ctx, &cams[v], f, &cps[v])) != NVGS_OK) return st;
    CK(cudaSetDevice(ctx->device));
    if ((st = check_scene(ctx)) != NVGS_OK) return st;
    const uint64_t pair_cap = std::min<uint64_t>(o.max_pairs > 0 ? (uint64_t)o.max_pairs
                                                                 : 8ull * (uint64_t)ctx->n_instanced,
                                                 0xffffffffull - 16);
    if (ctx->n_instanced >= ((int64_t)1 << 31))
        return fail(ctx, NVGS_ERR_CAPACITY, "batched views take at most 2^31 instanced Gaussians");
    begin_frame(ctx, false);
    cudaStream_t s = ctx->stream;
    CK(ensure(ctx->view_stats, (size_t)(n_views + 1) * 16));
    // graph key: view sizes, flags, options and capacities
    std::vector<uint8_t> key;
    auto put = [&](const void* p, size_t n) { key.insert(key.end(), (const uint8_t*)p, (const uint8_t*)p + n); };
    put(&n_views, sizeof n_views);
    for (auto& c : cps) { put(&c.W, sizeof c.W); put(&c.H, sizeof c.H); }
    put(f, sizeof *f);
    put(&o, sizeof o);
    put(&pair_cap, sizeof pair_cap);
    for (int v = 0; v < n_views; v++) put(&images[v], sizeof(float*));
    const std::vector<uint8_t> key_now = graph_stamp(ctx, key);
    const bool replay = o.use_graph && ctx->graph_exec && key_now == ctx->graph_key;
    if (replay) {
        // the graph's first node copies the staged cameras; restage them once the last copy is done
        if (ctx->cam_ev_pending) CK(cudaEventSynchronize(ctx->cam_ev));
        memcpy(ctx->h_cam, cps.data(), cps.size() * sizeof(CamParams));
        CK(cudaGraphLaunch(ctx->graph_exec, s));
        CK(cudaEventRecord(ctx->cam_ev, s));
        ctx->cam_ev_pending = true;
    } else {
        if ((st = upload_cams(ctx, cps.data(), n_views)) != NVGS_OK) return st;
        if ((st = enqueue_batch(ctx, cps, images, f, pair_cap)) != NVGS_OK) return st;
        if (o.use_graph) {
            // every buffer now has its size: capture the same work (cameras copied inside)
            CK(cudaStreamSynchronize(s));
            if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
            ctx->graph_key.clear();
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaMemcpyAsync(ctx->cam_dev.p, ctx->h_cam, cps.size() * sizeof(CamParams),
                                             cudaMemcpyHostToDevice, s);
            nvgs_status cs = ce == cudaSuccess ? enqueue_batch(ctx, cps, images, f, pair_cap)
                                               : fail(ctx, NVGS_ERR_CUDA, "capture: %s", cudaGetErrorString(ce));
            cudaGraph_t g = nullptr;
            cudaError_t ee = cudaStreamEndCapture(s, &g);
            if (cs != NVGS_OK) { if (g) cudaGraphDestroy(g); return cs; }
            if (ee != cudaSuccess) return fail(ctx, NVGS_ERR_CUDA, "capture: %s", cudaGetErrorString(ee));
            cudaError_t ie = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                ctx->graph_exec = nullptr;
                return fail(ctx, NVGS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
            ctx->graph_key = graph_stamp(ctx, key);   // the buffers as captured
        }
    }
    if (!stats) return NVGS_OK;
    std::vector<uint32_t> h((size_t)(n_views + 1) * 4);
    CK(cudaMemcpyAsync(h.data(), ctx->view_stats.p, h.size() * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int v = 0; v < n_views; v++) {
        memset(&stats[v], 0, sizeof stats[v]);
        stats[v].n_instanced = (uint64_t)ctx->n_instanced;
        stats[v].n_in_frustum = h[4 * v];
        stats[v].n_mlp_queries = f->use_mlp ? h[4 * v] : 0;
        stats[v].n_survivors = f->use_mlp ? h[4 * v + 1] : h[4 * v];
        stats[v].n_pairs = h[4 * v + 2];
    }
    if (h[4 * n_views]) return fail(ctx, NVGS_ERR_TIMEOUT, "tensor-core MLP: a bounded mbarrier wait gave up");
    if (h[4 * n_views + 1])
        return fail(ctx, NVGS_ERR_CAPACITY, "a view needed more than max_pairs = %llu pairs",
                    (unsigned long long)pair_cap);
    return NVGS_OK;
}

// ============================================================================ N3: views with own instance sets
// All views of the batch as one flattened frame: frame instance k = (view, instance) with the
// view's camera, the in-frustum and survivor lists of every view in one list, tile ids made global
// by each view's tile_base (the depth sort of all survivors and the tile sort of all pairs then
// give every tile its pairs front to back), and one launch per stage for the whole batch; nothing
// waits for the GPU, so the batch can be captured into a CUDA graph.
static nvgs_status enqueue_views(nvgs_ctx* ctx, const CullScope& scope, const CamParams& cp0, int n_views,
                                 int n_tiles, const nvgs_render_flags* f, uint64_t pair_cap, int digit_bits) {
    cudaStream_t s = ctx->stream;
    const CamParams* cam_dev = P<CamParams>(ctx->cam_dev);
    uint32_t* counters = P<uint32_t>(ctx->counters);
    CK(cudaMemsetAsync(&counters[8], 0, 8, s));   // MLP timeout flag, pair overflow flag
    StageTimer tm{ctx, false};
    uint32_t n_vis = 0, n_mlp = 0;
    nvgs_status st = run_cull(ctx, cam_dev, f, tm, &n_vis, &n_mlp, false, true, true, &scope);
    if (st != NVGS_OK) return st;
    const uint64_t cap = scope.cap;
    const uint2* surv = f->use_mlp ? P<uint2>(ctx->surv) : P<uint2>(ctx->vis_list);
    const uint32_t* n_surv_dev = f->use_mlp ? &counters[1] : &counters[0];
    // S4
    CK(ensure(ctx->rec, cap * 64 + 64));
    CK(ensure(ctx->tile_counts, cap * 4 + 16));
    CK(ensure(ctx->tile_offsets, cap * 4 + 16));
    CK(ensure(ctx->dkey, cap * 4 + 16));
    CK(ensure(ctx->didx, cap * 4 + 16));
    CK(ensure(ctx->dkey_alt, cap * 4 + 16));
    CK(ensure(ctx->didx_alt, cap * 4 + 16));
    CK(ensure(ctx->scratch, std::max({scan_scratch_bytes(scope.n_chunks), scan_scratch_bytes(cap + 1),
                                      radix_scratch_bytes(cap), radix_scratch_bytes(pair_cap),
                                      scan_scratch_bytes((uint64_t)n_tiles)})));
    CK(launch_project(surv, (uint32_t)cap, n_surv_dev, P<FrameInst>(ctx->frame_inst), P<AssetDev>(ctx->assets_dev),
                      cam_dev, P<float4>(ctx->rec), P<uint32_t>(ctx->tile_counts),
                      P<uint32_t>(ctx->dkey), P<uint32_t>(ctx->didx), ctx->num_sms, s, &ctx->log, 1));
    // S5: every survivor of the batch by depth, the pairs in that order with global tile ids, the
    // pairs by tile id
    int dpasses = 0, d_alt = 0;
    CK(radix_sort_pairs_u32(P<uint32_t>(ctx->dkey), P<uint32_t>(ctx->didx), P<uint32_t>(ctx->dkey_alt),
                            P<uint32_t>(ctx->didx_alt), cap, 32, ctx->scratch.p, s, &ctx->log, &dpasses, 0,
                            &d_alt, n_surv_dev, digit_bits));
    const uint32_t* order = d_alt ? P<uint32_t>(ctx->didx_alt) : P<uint32_t>(ctx->didx);
    CK(launch_gather_counts(order, P<uint32_t>(ctx->tile_counts), (uint32_t)cap, n_surv_dev,
                            P<uint32_t>(ctx->tile_offsets), ctx->num_sms, s, &ctx->log));
    CK(exclusive_scan_u32(P<uint32_t>(ctx->tile_offsets), P<uint32_t>(ctx->tile_offsets), cap, counters + 2,
                          ctx->scratch.p, s, &ctx->log, n_surv_dev));
    SortedPairs sp;
    {
        const nvgs_status st = bin_and_sort(ctx, order, (uint32_t)cap, n_surv_dev, cam_dev, counters + 2, pair_cap,
                                            counters + 9, counters + 2, n_tiles, digit_bits, 1, s, sp);
        if (st != NVGS_OK) return st;
    }
    uint32_t* svals = sp.vals;
    // S6 over the tiles of every view; the automatic split length takes the batch's pair count and
    // tile count (the rule of nvgs_render over the whole batch)
    const bool auto_split = f->blend_split_len == 0;
    const uint32_t split_len = f->blend_split_len < 0 ? 0xffffffffu
                               : (auto_split ? 4096u : (uint32_t)f->blend_split_len);
    if (pair_cap > split_len)
        CK(ensure(ctx->split_scratch, blend_split_scratch_bytes(n_tiles, pair_cap, cp0.tile_size, split_len)));
    // longest tiles first, while one CTA orders them quickly (a batch of up to 256K tiles)
    uint32_t* tile_order = nullptr;
    if (n_tiles <= (1 << 18)) {
        CK(ensure(ctx->tile_order, (size_t)n_tiles * 4 + 16));
        tile_order = P<uint32_t>(ctx->tile_order);
    }
    CK(launch_blend(P<uint32_t>(ctx->ranges), svals, P<float4>(ctx->rec), cp0, cam_dev, nullptr, nullptr, nullptr,
                    nullptr, split_len, pair_cap, auto_split ? counters + 2 : nullptr, ctx->split_scratch.p,
                    ctx->scratch.p, ctx->num_sms, nullptr, s, &ctx->log, n_views, P<float*>(ctx->mv_images),
                    n_tiles, tile_order));
    // batch counts (in frustum, survivors, pairs) and the flags, for the stats
    CK(cudaMemcpyAsync(P<uint32_t>(ctx->view_stats), counters, 3 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(P<uint32_t>(ctx->view_stats) + 4, &counters[8], 8, cudaMemcpyDeviceToDevice, s));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_render_views(nvgs_ctx* ctx, const nvgs_camera* cams,
                                         const nvgs_view_instances* sets, int n_views, float* const* images,
                                         const nvgs_render_flags* f, const nvgs_batch_opts* opts,
                                         nvgs_frame_stats* stats) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    nvgs_status st = validate_flags(ctx, f);
    if (st != NVGS_OK) return st;
    if (!cams || !images || n_views < 1 || n_views > 4096)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "need 1..4096 cameras and image pointers");
    if (f->image_memory != NVGS_MEM_DEVICE || f->keep_outputs || f->profile || f->logits_override)
        return fail(ctx, NVGS_ERR_INVALID_ARG,
                    "views need device images, no kept outputs, no profiling, no injected logits");
    for (int v = 0; v < n_views; v++)
        if (!images[v]) return fail(ctx, NVGS_ERR_INVALID_ARG, "image %d is NULL", v);
    nvgs_batch_opts o{};
    if (opts) o = *opts;
    if (o.max_pairs < 0) return fail(ctx, NVGS_ERR_INVALID_ARG, "max_pairs must be >= 0");
    CK(cudaSetDevice(ctx->device));
    if ((st = check_scene(ctx)) != NVGS_OK) return st;
    const int n_inst = (int)ctx->instances.size();
    // frame instances (view, instance) and their chunks; cameras with their global tile bases
    std::vector<int2> fimap;
    std::vector<Chunk> chunks;
    std::vector<CamParams> cps(n_views);
    uint64_t total = 0;
    int n_tiles = 0;
    for (int v = 0; v < n_views; v++) {
        if ((st = make_cam(ctx, &cams[v], f, &cps[v])) != NVGS_OK) return st;
        cps[v].tile_base = n_tiles;
        n_tiles += cps[v].tiles_x * cps[v].tiles_y;
        const bool all = !sets || !sets[v].instances;
        const int count = all ? n_inst : sets[v].count;
        if (count < 0) return fail(ctx, NVGS_ERR_INVALID_ARG, "view %d: negative instance count", v);
        for (int j = 0; j < count; j++) {
            const int i = all ? j : sets[v].instances[j];
            if (i < 0 || i >= n_inst)
                return fail(ctx, NVGS_ERR_INVALID_ARG, "view %d: instance %d out of range", v, i);
            const int fi = (int)fimap.size();
            fimap.push_back(make_int2(v, i));
            const int64_t n = ctx->assets[ctx->instances[i].asset_id].dev.n;
            for (int64_t g0 = 0; g0 < n; g0 += kChunk)
                chunks.push_back(Chunk{fi, (int)g0, (int)std::min<int64_t>(kChunk, n - g0), 0});
            total += (uint64_t)n;
        }
        if (n_tiles > (1 << 26)) return fail(ctx, NVGS_ERR_CAPACITY, "more than 2^26 tiles in the batch");
    }
    if (fimap.empty()) return fail(ctx, NVGS_ERR_INVALID_ARG, "no instance in any view");
    if (total >= ((uint64_t)1 << 31))
        return fail(ctx, NVGS_ERR_CAPACITY, "a batch takes at most 2^31 instanced Gaussians (has %llu)",
                    (unsigned long long)total);
    const uint64_t pair_cap = std::min<uint64_t>(o.max_pairs > 0 ? (uint64_t)o.max_pairs : 8ull * total,
                                                 0xffffffffull - 16);
    const int digit_bits = f->sort_digit_bits ? f->sort_digit_bits : 8;
    begin_frame(ctx, false);
    ctx->kept_frame = false;
    cudaStream_t s = ctx->stream;
    CK(ensure(ctx->view_stats, 32));
    // graph key: cameras' sizes, the instance sets, flags, options and image pointers
    std::vector<uint8_t> key;
    auto put = [&](const void* p, size_t n) { key.insert(key.end(), (const uint8_t*)p, (const uint8_t*)p + n); };
    put(&n_views, sizeof n_views);
    for (auto& c : cps) { put(&c.W, sizeof c.W); put(&c.H, sizeof c.H); }
    put(fimap.data(), fimap.size() * sizeof(int2));
    put(f, sizeof *f);
    put(&o, sizeof o);
    put(&pair_cap, sizeof pair_cap);
    for (int v = 0; v < n_views; v++) put(&images[v], sizeof(float*));
    const std::vector<uint8_t> key_now = graph_stamp(ctx, key);
    const bool replay = o.use_graph && ctx->mv_graph_exec && key_now == ctx->mv_graph_key;
    if (replay) {
        if (ctx->cam_ev_pending) CK(cudaEventSynchronize(ctx->cam_ev));
        memcpy(ctx->h_cam, cps.data(), cps.size() * sizeof(CamParams));
        CK(cudaGraphLaunch(ctx->mv_graph_exec, s));
        CK(cudaEventRecord(ctx->cam_ev, s));
        ctx->cam_ev_pending = true;
    } else {
        CK(ensure(ctx->mv_fimap, fimap.size() * sizeof(int2)));
        CK(ensure(ctx->mv_chunks, chunks.size() * sizeof(Chunk)));
        CK(ensure(ctx->mv_images, (size_t)n_views * sizeof(float*)));
        CK(cudaMemcpyAsync(ctx->mv_fimap.p, fimap.data(), fimap.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->mv_chunks.p, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->mv_images.p, images, (size_t)n_views * sizeof(float*), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));   // the host vectors go out of scope
        if ((st = upload_cams(ctx, cps.data(), n_views)) != NVGS_OK) return st;
        const CullScope scope{P<Chunk>(ctx->mv_chunks), (int)chunks.size(), (int)fimap.size(), P<int2>(ctx->mv_fimap),
                              total};
        if ((st = enqueue_views(ctx, scope, cps[0], n_views, n_tiles, f, pair_cap, digit_bits)) != NVGS_OK) return st;
        if (o.use_graph) {
            CK(cudaStreamSynchronize(s));
            if (ctx->mv_graph_exec) { cudaGraphExecDestroy(ctx->mv_graph_exec); ctx->mv_graph_exec = nullptr; }
            ctx->mv_graph_key.clear();
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaMemcpyAsync(ctx->cam_dev.p, ctx->h_cam, cps.size() * sizeof(CamParams),
                                             cudaMemcpyHostToDevice, s);
            nvgs_status cs = ce == cudaSuccess
                                 ? enqueue_views(ctx, scope, cps[0], n_views, n_tiles, f, pair_cap, digit_bits)
                                 : fail(ctx, NVGS_ERR_CUDA, "capture: %s", cudaGetErrorString(ce));
            cudaGraph_t g = nullptr;
            cudaError_t ee = cudaStreamEndCapture(s, &g);
            if (cs != NVGS_OK) { if (g) cudaGraphDestroy(g); return cs; }
            if (ee != cudaSuccess) return fail(ctx, NVGS_ERR_CUDA, "capture: %s", cudaGetErrorString(ee));
            cudaError_t ie = cudaGraphInstantiate(&ctx->mv_graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                ctx->mv_graph_exec = nullptr;
                return fail(ctx, NVGS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
            ctx->mv_graph_key = graph_stamp(ctx, key);   // the buffers as captured
        }
    }
    if (!stats) return NVGS_OK;
    uint32_t h[8] = {};
    CK(cudaMemcpyAsync(h, ctx->view_stats.p, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memset(stats, 0, sizeof *stats);
    stats->n_instanced = total;
    stats->n_in_frustum = h[0];
    stats->n_mlp_queries = f->use_mlp ? h[0] : 0;
    stats->n_survivors = f->use_mlp ? h[1] : h[0];
    stats->n_pairs = h[2];
    stats->kernel_launches = ctx->log.count;
    if (h[4]) return fail(ctx, NVGS_ERR_TIMEOUT, "tensor-core MLP: a bounded mbarrier wait gave up");
    if (h[5])
        return fail(ctx, NVGS_ERR_CAPACITY, "the batch needed more than max_pairs = %llu pairs",
                    (unsigned long long)pair_cap);
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_autotune(nvgs_ctx* ctx, const nvgs_camera* cams, int n_views,
                                     float* const* images, const nvgs_render_flags* f,
                                     const nvgs_batch_opts* opts, nvgs_render_flags* best,
                                     nvgs_tune_result* results, int max_results, int* n_results) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (!f || !best) return fail(ctx, NVGS_ERR_INVALID_ARG, "flags / best is NULL");
    nvgs_batch_opts o{};
    if (opts) o = *opts;
    o.use_graph = 0;   // plain batches: the graph cache keeps whatever the caller captured
    const bool tc = f->use_mlp && uses_tc_mlp(ctx, f);
    const int tiles[3] = {8, 16, 32};
    const int splits[2] = {0, -1};
    const int digits[3] = {8, 6, 4};
    const int n_ctas = tc ? 4 : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaSetDevice(ctx->device));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = INFINITY;
    int count = 0;
    nvgs_status st = NVGS_OK;
    for (int ti = 0; ti < 3 && st == NVGS_OK; ti++)
        for (int ci = 0; ci < n_ctas && st == NVGS_OK; ci++)
            for (int si = 0; si < 2 && st == NVGS_OK; si++)
            for (int di = 0; di < 3 && st == NVGS_OK; di++) {
                nvgs_render_flags c = *f;
                c.tile_size = tiles[ti];
                c.mlp_ctas_per_sm = tc ? ci + 1 : f->mlp_ctas_per_sm;
                c.blend_split_len = splits[si];
                c.sort_digit_bits = digits[di];
                std::vector<nvgs_frame_stats> stv(n_views);
                st = nvgs_render_batch(ctx, cams, n_views, images, &c, &o, stv.data());   // warm-up
                if (st == NVGS_ERR_CAPACITY) {   // needs more pairs than max_pairs: not a candidate
                    if (results && count < max_results)
                        results[count] = nvgs_tune_result{c.tile_size, c.mlp_ctas_per_sm, c.blend_split_len, INFINITY,
                                                          c.sort_digit_bits, 0};
                    count++;
                    st = NVGS_OK;
                    continue;
                }
                if (st != NVGS_OK) break;
                cudaEventRecord(e0, ctx->stream);
                for (int rep = 0; rep < 3 && st == NVGS_OK; rep++)
                    st = nvgs_render_batch(ctx, cams, n_views, images, &c, &o, nullptr);
                if (st != NVGS_OK) break;
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= 3.0f * (float)n_views;
                if (results && count < max_results)
                    results[count] = nvgs_tune_result{c.tile_size, c.mlp_ctas_per_sm, c.blend_split_len, ms,
                                                      c.sort_digit_bits, 0};
                count++;
                if (ms < best_ms) { best_ms = ms; *best = c; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_results) *n_results = count;
    return st;
}

extern "C" nvgs_status nvgs_device_bytes(const nvgs_ctx* ctx, uint64_t* bytes) {
    if (!ctx || !bytes) return NVGS_ERR_INVALID_ARG;
    uint64_t t = 0;
    for (auto& a : ctx->assets)
        for (const DevBuf* b : {&a.mean_op, &a.scale_quat, &a.sh, &a.w_fp32, &a.w_tc, &a.w_f8}) t += b->cap;
    const DevBuf* bufs[] = {&ctx->assets_dev, &ctx->inst_raw, &ctx->inst_offset, &ctx->chunks,
                            &ctx->frame_inst, &ctx->bits, &ctx->chunk_counts, &ctx->chunk_offsets,
                            &ctx->vis_list, &ctx->keep_bits, &ctx->logits_tmp, &ctx->block_counts,
                            &ctx->block_offsets, &ctx->surv, &ctx->rec, &ctx->tile_counts,
                            &ctx->tile_offsets, &ctx->keys, &ctx->vals, &ctx->keys_alt, &ctx->vals_alt,
                            &ctx->ranges, &ctx->scratch, &ctx->counters, &ctx->image_tmp, &ctx->final_T,
                            &ctx->n_contrib, &ctx->mark, &ctx->tr_sv, &ctx->tr_sg, &ctx->tr_partial,
                            &ctx->dkey, &ctx->didx, &ctx->dkey_alt, &ctx->didx_alt, &ctx->split_scratch,
                            &ctx->grad_surv, &ctx->tile_order, &ctx->cam_dev, &ctx->view_stats};
    for (const DevBuf* b : bufs) t += b->cap;
    for (auto& tr : ctx->train) t += tr.w.cap + tr.m.cap + tr.v.cap + tr.views.cap;
    *bytes = t;
    return NVGS_OK;
}

// ============================================================================ gradients
extern "C" nvgs_status nvgs_render_backward(nvgs_ctx* ctx, const float* dL_dimage, int asset_id,
                                            const nvgs_asset_grads* g) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->assets.size())
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset_id %d not loaded", asset_id);
    if (!dL_dimage || !g || !g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "dL_dimage / gradient array is NULL");
    if (!ctx->kept_frame)
        return fail(ctx, NVGS_ERR_UNSUPPORTED,
                    "no kept frame: render with keep_outputs = 1 right before the backward");
    CK(cudaSetDevice(ctx->device));
    const nvgs_frame_view& L = ctx->last;
    const uint32_t n_surv = (uint32_t)L.n_survivors;
    CK(ensure(ctx->grad_surv, render_backward_scratch_bytes(n_surv)));
    begin_frame_log_only(ctx);
    CK(launch_render_backward(L.tile_ranges, L.pair_values, reinterpret_cast<const float4*>(L.records),
                              ctx->last_cp, P<CamParams>(ctx->cam_dev), L.final_T, L.n_contrib, dL_dimage,
                              P<float>(ctx->grad_surv),
                              reinterpret_cast<const uint2*>(L.survivors), n_surv,
                              P<FrameInst>(ctx->frame_inst), P<AssetDev>(ctx->assets_dev), asset_id,
                              g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, ctx->stream,
                              &ctx->log));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_update_asset(nvgs_ctx* ctx, int asset_id, const float* means,
                                         const float* log_scales, const float* quats,
                                         const float* opacity_logits, const float* sh) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (asset_id < 0 || asset_id >= (int)ctx->assets.size())
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset_id %d not loaded", asset_id);
    if (!means || !log_scales || !quats || !opacity_logits || !sh)
        return fail(ctx, NVGS_ERR_INVALID_ARG, "asset array is NULL");
    CK(cudaSetDevice(ctx->device));
    AssetStore& a = ctx->assets[asset_id];
    const int K = (a.dev.sh_degree + 1) * (a.dev.sh_degree + 1);
    ctx->kept_frame = false;
    begin_frame_log_only(ctx);
    CK(launch_pack_asset((uint32_t)a.dev.n, K, a.dev.sh_stride, means, log_scales, quats, opacity_logits,
                         sh, P<float4>(a.mean_op), P<float4>(a.scale_quat), P<float>(a.sh),
                         ctx->stream, &ctx->log));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_last_frame(const nvgs_ctx* ctx, nvgs_frame_view* out) {
    if (!ctx || !out) return NVGS_ERR_INVALID_ARG;
    *out = ctx->last;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_sort_pairs(nvgs_ctx* ctx, uint64_t* keys, uint32_t* values, int64_t n,
                                       int key_bits) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    if (n < 0 || n > 0xffffffffLL) return fail(ctx, NVGS_ERR_INVALID_ARG, "n out of range");
    if (key_bits < 0 || key_bits > 64) return fail(ctx, NVGS_ERR_INVALID_ARG, "key_bits must be 0..64");
    if (n > 0 && (!keys || !values)) return fail(ctx, NVGS_ERR_INVALID_ARG, "keys / values NULL");
    CK(cudaSetDevice(ctx->device));
    if (n <= 1 || key_bits == 0) return NVGS_OK;
    CK(ensure(ctx->keys_alt, (size_t)n * 8));
    CK(ensure(ctx->vals_alt, (size_t)n * 4));
    CK(ensure(ctx->scratch, radix_scratch_bytes((uint64_t)n)));
    int passes = 0, in_alt = 0;
    begin_frame(ctx, false);
    CK(radix_sort_pairs(reinterpret_cast<unsigned long long*>(keys), values,
                        P<unsigned long long>(ctx->keys_alt), P<uint32_t>(ctx->vals_alt), (uint64_t)n,
                        key_bits, ctx->scratch.p, ctx->stream, &ctx->log, &passes, 1, &in_alt));
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_kernel_stats(const nvgs_ctx* ctx, nvgs_kernel_stat* out, int cap,
                                         int* n_out) {
    if (!ctx || !n_out || cap < 0 || (cap > 0 && !out)) return NVGS_ERR_INVALID_ARG;
    const int n = (int)ctx->kname.size();
    for (int k = 0; k < n && k < cap; k++) {
        memset(out[k].name, 0, sizeof out[k].name);
        strncpy(out[k].name, ctx->kname[k].c_str(), sizeof out[k].name - 1);
        out[k].launches = ctx->kcount[k];
        out[k].total_ms = ctx->kms[k];
    }
    *n_out = n;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_reset_kernel_stats(nvgs_ctx* ctx) {
    if (!ctx) return NVGS_ERR_INVALID_ARG;
    ctx->kname.clear();
    ctx->kcount.clear();
    ctx->kms.clear();
    return NVGS_OK;
}

extern "C" void nvgs_debug_fail_allocs(int n) { g_fail_allocs.store(n > 0 ? n : 0); }
