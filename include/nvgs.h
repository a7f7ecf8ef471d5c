/*
 * nvgs.h — C ABI of the NVGS per-frame render pass on one NVIDIA B300 (sm_103a).
 *
 * The library renders composed scenes of instanced 3D Gaussian Splatting assets with the
 * occlusion culling of "NVGS: Neural Visibility for Occlusion Culling in 3D Gaussian Splatting":
 *
 *   S1  frustum culling of every instanced Gaussian on its mean            (Sec. 3.3)
 *   S2  the per-asset visibility MLP, queried for in-frustum Gaussians     (Sec. 3.2, 3.3, Eq. 2)
 *   S3  stream compaction: a Gaussian is instantiated only if it survives  (Sec. 3.3)
 *   S4  EWA projection to 2D conics and SH colour                          (Sec. 3.3 -> 3DGS)
 *   S5  tile binning and a radix sort on (tile, depth) keys                (Sec. 3.3 -> 3DGS)
 *   S6  front-to-back alpha compositing with the blending rules of         (Sec. 4.1)
 *       alpha < 1/255 skipped and T < 1e-4 stopping the pixel
 *
 * Every call is asynchronous on the context's CUDA stream unless stated otherwise.  Device
 * pointers passed in are borrowed for the duration of the enqueued work; the caller keeps
 * ownership of everything it passes.  No C++ exception crosses this boundary: each call returns
 * an nvgs_status and the text of the last error is kept per context (nvgs_last_error).
 *
 * Conventions (the same as the test-side oracle's):
 *   - instance: a local point mu lands at R (s mu) + t in the world (R orthonormal, s > 0);
 *   - camera: x_c = R x_w + t, x right / y down / z forward; pixel (i, j) is sampled at its centre
 *     (i + 0.5, j + 0.5); u = fx x_c / z_c + cx, v = fy y_c / z_c + cy;
 *   - images are row-major H x W x 3 float32 (RGB innermost);
 *   - "instanced index" of Gaussian g of instance i = sum_{k<i} N(asset of k) + g.
 */
#ifndef NVGS_H
#define NVGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NVGS_ABI_VERSION 1

typedef enum {
    NVGS_OK = 0,
    NVGS_ERR_INVALID_ARG = 1,  /* a pointer, size or enum is out of range; nothing was enqueued */
    NVGS_ERR_OOM = 2,          /* device allocation failed */
    NVGS_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    NVGS_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    NVGS_ERR_CAPACITY = 5,     /* a fixed-capacity buffer would overflow */
    NVGS_ERR_UNSUPPORTED = 6   /* a valid request the library does not implement */
} nvgs_status;

typedef enum { NVGS_MEM_HOST = 0, NVGS_MEM_DEVICE = 1 } nvgs_memory;

/* Arithmetic of the visibility MLP (Sec. 3.2): FP32 on CUDA cores; BF16 operands with FP32
 * accumulation on the tcgen05 tensor cores; or E4M3 (FP8) operands with FP32 accumulation on
 * the tensor cores, one scale per tensor: weights max|W| / 448, inputs x 256 (|x| <= 1), hidden
 * activations (their bound for |x| <= 1) / 448. */
typedef enum { NVGS_PREC_FP32 = 0, NVGS_PREC_BF16 = 1, NVGS_PREC_FP8 = 2 } nvgs_precision;

typedef struct nvgs_ctx nvgs_ctx;

/* One 3DGS asset (Sec. 3.3: every distinct asset is held once, however often it is placed).  Arrays are read during the
 * call and copied into the library's own layout. */
typedef struct {
    int64_t n;                   /* Gaussians, >= 1 */
    int32_t sh_degree;           /* 0..3 */
    int32_t memory;              /* nvgs_memory of the five arrays below */
    const float* means;          /* n x 3 */
    const float* log_scales;     /* n x 3 */
    const float* quats;          /* n x 4, (w, x, y, z), need not be normalised */
    const float* opacity_logits; /* n; opacity = sigmoid(logit) */
    const float* sh;             /* n x (deg+1)^2 x 3, coefficient-major, RGB innermost */
    float train_fov_x;           /* training field of view theta_t in radians (Eq. 1, Eq. 2) */
    float d_min, d_max;          /* camera distance bounds; <= 0 selects Eq. 1 on the means' box */
    float p_near, p_far;         /* Eq. 1 coverage fractions; <= 0 selects 0.9 / 0.05 (Sec. 3.1) */
} nvgs_asset_desc;

/* A rigid, uniformly scaled placement of an asset (Sec. 3.3: the scene is a list of such
 * transforms over the stored assets). */
typedef struct {
    int32_t asset_id;
    float R[9];                  /* row-major rotation */
    float t[3];
    float s;                     /* uniform scale > 0 (the s of Eq. 2) */
} nvgs_instance;

/* Pinhole camera.  The field of view is fixed by fx, fy and the image size. */
typedef struct {
    float R[9];                  /* world -> camera rotation, row-major */
    float t[3];
    float fx, fy, cx, cy;        /* pixels */
    int32_t width, height;       /* 1 .. 16384 */
    float z_near;                /* > 0 */
} nvgs_camera;

/* Per-frame switches.  nvgs_default_flags() fills the paper's values. */
typedef struct {
    int32_t use_mlp;             /* 0: unculled plain path (S1, S4-S6); 1: MLP culling (S1-S6) */
    int32_t mlp_gate;            /* 1: bypass the MLP for instances closer than d_min (Sec. 3.3) */
    float logit_threshold;       /* keep iff logit > threshold (default 0) */
    float alpha_min;             /* 1/255 (Sec. 4.1) */
    float alpha_max;             /* 0.99 (3DGS) */
    float t_stop;                /* 1e-4 (Sec. 4.1) */
    float dilation;              /* 0.3 px^2 added to the 2D covariance (3DGS) */
    float guard_band;            /* 1.3: frustum half-width multiplier */
    float bg[3];                 /* background colour */
    int32_t tile_size;           /* 8, 16 or 32 */
    int32_t image_memory;        /* nvgs_memory of the output image */
    int32_t profile;             /* 1: time each stage and kernel with CUDA events
                                    (nvgs_frame_stats, nvgs_kernel_stats); 2: the same and count
                                    S6's (pixel, fragment) evaluations, which runs an instrumented
                                    compositing kernel (so its times are not those of 1) */
    const float* logits_override;/* nullable DEVICE array of per-instanced-Gaussian logits used
                                    instead of the MLP (tests inject fixed decisions with it) */
    int32_t keep_outputs;        /* 1: keep final T and the last blended pair per pixel for
                                    nvgs_render_backward */
    int32_t blend_split_len;     /* tiles with more pairs are composited in chunks of this many
                                    pairs on separate CTAs (0: automatic, max(4096, 4 x the
                                    mean pairs per tile); < 0: never; else >= 256) */
    int32_t mlp_ctas_per_sm;     /* resident CTAs per SM of the BF16 tensor-core MLP (0: default
                                    4; 1..4) -- a tuning knob, results do not depend on it */
    float radius_clip_area;      /* radius clipping (Sec. 4.4), lossy: a splat whose 1-sigma
                                    ellipse is smaller than this many px^2, i.e. whose
                                    pi sqrt(det Sigma_2D) (dilation included) is below it, is not
                                    binned.  0 (default): off.  >= 0 */
    int32_t sort_digit_bits;     /* digit width of the S5 radix sorts, 4..8 bits (0: default 8) --
                                    a tuning knob, results do not depend on it */
    int32_t reserved[3];
} nvgs_render_flags;

#define NVGS_NUM_STAGES 8
/* Stage indices of nvgs_frame_stats.stage_ms */
enum { NVGS_STAGE_SETUP = 0, NVGS_STAGE_CULL = 1, NVGS_STAGE_MLP = 2, NVGS_STAGE_COMPACT = 3,
       NVGS_STAGE_PROJECT = 4, NVGS_STAGE_BIN = 5, NVGS_STAGE_SORT = 6, NVGS_STAGE_BLEND = 7 };

typedef struct {
    uint64_t n_instanced;        /* instanced Gaussians before culling */
    uint64_t n_in_frustum;       /* after S1 */
    uint64_t n_mlp_queries;      /* Gaussians the MLP evaluated (in frustum, not gated) */
    uint64_t n_survivors;        /* after S2/S3 = instantiated Gaussians */
    uint64_t n_pairs;            /* (tile, Gaussian) pairs sorted in S5 */
    uint32_t n_instances_visible;/* instances whose bounding sphere meets the frustum */
    uint32_t sort_passes;        /* radix passes run in S5 */
    float stage_ms[NVGS_NUM_STAGES]; /* filled when flags.profile >= 1 (synchronises) */
    uint64_t kernel_launches;    /* kernels this frame enqueued */
    uint64_t blend_evaluations;  /* (pixel, fragment) evaluations of S6 up to each pixel's stop,
                                    when flags.profile = 2 */
    uint64_t blend_composited;   /* of those, the fragments composited (alpha >= alpha_min, not
                                    stopped), when flags.profile = 2 */
} nvgs_frame_stats;

/* ------------------------------------------------------------------ context */
/* Creates a context on CUDA device `device`; `cuda_stream` is a cudaStream_t to enqueue on,
 * or NULL for a stream the context creates and owns.  That stream is a blocking one: it orders
 * itself with the legacy default stream (work enqueued there before a call finishes before the
 * call's kernels start, and work enqueued there after waits for them), which is how callers
 * that use the default stream -- such as PyTorch by default -- see the library's results. */
nvgs_status nvgs_create(nvgs_ctx** out, int device, void* cuda_stream);
nvgs_status nvgs_destroy(nvgs_ctx* ctx);
/* Text of the last error on this context ("" if none).  Owned by the context. */
const char* nvgs_last_error(const nvgs_ctx* ctx);
/* The cudaStream_t the context enqueues on. */
void* nvgs_get_stream(const nvgs_ctx* ctx);
/* Fills the paper's defaults: MLP on, gate on, threshold 0, alpha in [1/255, 0.99],
 * T stop 1e-4, dilation 0.3, guard band 1.3, black background, 16x16 tiles, device image. */
void nvgs_default_flags(nvgs_render_flags* flags);
int nvgs_abi_version(void);

/* ------------------------------------------------------------------ scene */
/* Copies an asset into device memory (structure-of-arrays, 16-byte vectors), computes its
 * means' bounding box and the Eq. 1 distance bounds (Sec. 3.1).  Synchronous.  *asset_id
 * receives the new asset's index (0, 1, ...). */
nvgs_status nvgs_load_asset(nvgs_ctx* ctx, const nvgs_asset_desc* desc, int* asset_id);

/* Sets the asset's visibility MLP (Sec. 3.2): 32 -> 64 -> 64 -> 64 -> 1 with ReLU.  `weights`
 * is a HOST array of 10497 floats: W1 (64x32, row = output), b1 (64), W2 (64x64), b2, W3 (64x64),
 * b3, W4 (1x64), b4 (1).  The library keeps an FP32 copy and, for NVGS_PREC_BF16, BF16 operand
 * tiles in the tcgen05 shared-memory layout.  Synchronous. */
nvgs_status nvgs_set_mlp(nvgs_ctx* ctx, int asset_id, const float* weights, int precision);

/* Replaces the instance list (HOST array).  Every asset_id must name a loaded asset. */
nvgs_status nvgs_set_instances(nvgs_ctx* ctx, const nvgs_instance* instances, int count);

/* Totals of the current scene. */
nvgs_status nvgs_scene_info(const nvgs_ctx* ctx, int64_t* n_instanced, int* n_assets,
                            int* n_instances);

/* ------------------------------------------------------------------ per frame */
/* S1 + S2 only (Sec. 3.3): per instanced Gaussian, the MLP logit (NaN outside the frustum,
 * +inf where the instance bypasses the MLP) and the keep decision (0/1 bytes: in frustum and
 * kept).  Both outputs are nullable DEVICE arrays of n_instanced entries.  stats (HOST,
 * nullable) is written after the call synchronises. */
nvgs_status nvgs_query_visibility(nvgs_ctx* ctx, const nvgs_camera* cam,
                                  const nvgs_render_flags* flags, float* logits,
                                  uint8_t* keep, nvgs_frame_stats* stats);

/* The whole pass S1-S6 for one camera into `image` (H x W x 3 float32 in flags.image_memory).
 * A HOST image that is page-locked and mapped for the device (cudaHostAlloc, or a pinned torch
 * tensor) is written directly by the compositing kernels, overlapping the transfer with the
 * compositing; a pageable HOST image is copied back from a device buffer.  Either way it is
 * complete when the call returns.  stats (HOST, nullable) is filled after the call
 * synchronises. */
nvgs_status nvgs_render(nvgs_ctx* ctx, const nvgs_camera* cam, const nvgs_render_flags* flags,
                        float* image, nvgs_frame_stats* stats);

/* ------------------------------------------------------------------ visibility MLP: labels, training */
/* GPU labeller (Sec. 3.1): renders asset `asset_id` alone (identity transform, no culling) from
 * each of the n_views HOST cameras and writes labels[(v / group) * N + g] = 1 for every Gaussian g
 * that is blended at one or more pixels of view v (contribution alpha * T > 0), else 0.  Views are
 * taken in groups of `group` consecutive cameras whose labels are OR-ed: a main view followed by
 * its auxiliary cone views (Sec. 3.1).  labels is a DEVICE array of (n_views / group) * N bytes.
 * flags supplies the blending constants and tile size (use_mlp is ignored).  The caller's scene
 * (instances) is restored afterwards.  Synchronous. */
nvgs_status nvgs_label_visibility(nvgs_ctx* ctx, int asset_id, const nvgs_camera* views, int n_views,
                                  int group, const nvgs_render_flags* flags, uint8_t* labels);

/* Per-asset constants computed at load (Sec. 3.1). */
typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t has_mlp;             /* -1 none, else the nvgs_precision set */
    float bbox_center[3];        /* centre of the means' bounding box */
    float bbox_half_extent[3];
    float d_min, d_max;          /* Eq. 1 camera distance bounds */
    float train_fov_x;           /* theta_t */
} nvgs_asset_info;
nvgs_status nvgs_get_asset_info(const nvgs_ctx* ctx, int asset_id, nvgs_asset_info* out);

/* Training views (Sec. 3.1, 4.1): n_dirs Fibonacci-sphere directions around the asset's box
 * centre, each at n_dist distances log-spaced from d_min to d_max (n_dist = 3 gives d_min, their
 * geometric mean and d_max), looking at the centre with the asset's training field of view, at
 * width x height pixels.  out: HOST array of n_dirs * n_dist cameras, direction-major. */
nvgs_status nvgs_training_views(const nvgs_ctx* ctx, int asset_id, int n_dirs, int n_dist, int width,
                                int height, nvgs_camera* out);

/* Training views with the paper's robustness variants (Sec. 3.1, 4.1).  Main views as for
 * nvgs_training_views, each followed by n_aux auxiliary views: cameras at the same distance whose
 * directions lie on the cone of half-angle aux_angle around the main direction (equally spaced
 * around it), looking at the box centre; nvgs_label_visibility with group = 1 + n_aux OR-s a main
 * view with its auxiliary views.  random_offset = 1 shifts every main camera in its image plane
 * so that the asset does not sit at the image centre: the shift is (a r + b d_n) s(d) d with
 * (a, b) uniform in [-1, 1]^2 (SplitMix64 of seed and the view index), r / d_n the camera's right
 * and down axes and s(d) growing linearly from 0 at d_min to d_min / d_max at d_max.  out: HOST
 * array of n_dirs * n_dist * (1 + n_aux) cameras, main-view-major. */
typedef struct {
    int32_t n_dirs, n_dist;      /* Fibonacci directions, log-spaced distances per direction */
    int32_t width, height;
    int32_t n_aux;               /* auxiliary views per main view (0: none; the paper's figures: 6) */
    float aux_angle;             /* cone half-angle, radians (> 0 when n_aux > 0) */
    int32_t random_offset;       /* 0 / 1 */
    int32_t pad_;
    uint64_t seed;
} nvgs_view_opts;
nvgs_status nvgs_training_views_ex(const nvgs_ctx* ctx, int asset_id, const nvgs_view_opts* opts,
                                   nvgs_camera* out);

/* Starts training the MLP of `asset_id` (Sec. 3.2, 4.1): FP32 master weights from `w0` (HOST,
 * 10497 floats, the nvgs_set_mlp layout), zero Adam moments, and the n_views HOST cameras the
 * label rows refer to (one per label row; their centre and focal length give each sample's view
 * direction and Eq. 2 distance). */
nvgs_status nvgs_train_init(nvgs_ctx* ctx, int asset_id, const float* w0, const nvgs_camera* views,
                            int n_views);

typedef struct {
    const uint8_t* labels;       /* DEVICE, n_views x N bytes from nvgs_label_visibility */
    int32_t batch;               /* samples per step (B) */
    int32_t precision;           /* NVGS_PREC_FP32 (0): forward and backward in FP32 on the CUDA
                                    cores; NVGS_PREC_BF16: BF16 operands with FP32 accumulation on
                                    the tcgen05 tensor cores, blocks of 128 samples.  Master
                                    weights, moments and the Adam update are FP32 either way */
    const int32_t* sample_view;  /* nullable DEVICE [B]: explicit (view, gaussian) samples; NULL */
    const int32_t* sample_gauss; /*   draws them on the device from seed and step (SplitMix64) */
    uint64_t seed;
} nvgs_train_batch;

typedef struct {
    float lr, beta1, beta2, eps; /* Adam (Sec. 4.1: Adam, lr 2e-3 decaying to 2e-4) */
    int32_t step;                /* 0-based step index (bias correction, sample stream) */
} nvgs_adam_cfg;

/* One Adam step on the class-balanced binary cross-entropy of B samples (a sample of class c
 * weighs B / (2 N_c), N_c = its class count in the batch: the class-frequency weighting of
 * Sec. 4.1).  loss_out (HOST, nullable) receives the batch loss; reading it
 * synchronises, and then a BF16 step whose bounded tensor-core wait gave up returns
 * NVGS_ERR_TIMEOUT (its update must be discarded: reload a checkpoint). */
nvgs_status nvgs_train_visibility_step(nvgs_ctx* ctx, int asset_id, const nvgs_train_batch* batch,
                                       const nvgs_adam_cfg* adam, float* loss_out);

/* Copies the FP32 master weights (HOST, 10497 floats).  Pass them to nvgs_set_mlp to use them. */
nvgs_status nvgs_train_get_weights(nvgs_ctx* ctx, int asset_id, float* w_out);

/* Training checkpoint for resume: the FP32 master weights and both Adam moments of `asset_id`'s
 * training state, as 3 x 10497 HOST floats in the order w, m, v (each in the nvgs_set_mlp layout).
 * nvgs_train_load_state replaces them in a training state that nvgs_train_init created (with the
 * same views).  Training is deterministic given (seed, step), so a run that saves after step k - 1
 * and resumes at step k repeats the uninterrupted run bit for bit.  NVGS_ERR_INVALID_ARG if the
 * asset has no training state or a pointer is NULL. */
#define NVGS_TRAIN_STATE_FLOATS (3 * 10497)
nvgs_status nvgs_train_save_state(nvgs_ctx* ctx, int asset_id, float* state_out);
nvgs_status nvgs_train_load_state(nvgs_ctx* ctx, int asset_id, const float* state);

/* Learning rate at `step` of `total` (Sec. 4.1): cosine warm-up from 0 to lr0 over the first
 * warmup_frac of the steps, then exponential decay to lr1 at the last step. */
float nvgs_lr_schedule(int step, int total, float lr0, float lr1, float warmup_frac);

/* ------------------------------------------------------------------ per-kernel timing */
/* Device time of each kernel, accumulated over every nvgs_render call made with
 * flags.profile = 1 since the last reset (CUDA events bracket each launch on the context's
 * stream).  Writes up to `cap` entries and the number of distinct kernels to *n. */
typedef struct {
    char name[40];
    uint64_t launches;
    double total_ms;
} nvgs_kernel_stat;
nvgs_status nvgs_kernel_stats(const nvgs_ctx* ctx, nvgs_kernel_stat* out, int cap, int* n);
nvgs_status nvgs_reset_kernel_stats(nvgs_ctx* ctx);

/* ------------------------------------------------------------------ batched, sync-free rendering */
/* Several views in one call with no host synchronisation between (or inside) them: every count
 * (in-frustum, survivors, pairs) stays on the device and each kernel reads it there, buffers are
 * sized for capacities instead of the counts, and the camera records are copied to the device on
 * the stream.  The whole batch can therefore be captured into a CUDA graph: with use_graph = 1
 * the first call renders the batch and captures it; later calls with the same number of views,
 * the same view sizes, flags and options replay the graph with the new cameras (one graph launch
 * per batch).  A call after the assets, MLPs or instances changed, or after any call of the
 * library (re)allocated a buffer, captures anew instead of replaying (a graph holds the scene's
 * lists and raw buffer addresses).  The paper runs one view per frame (Sec. 3.3); batching serves
 * multi-view use such as training-view rendering or several cameras per frame. */
typedef struct {
    int64_t max_pairs;           /* capacity of (tile, Gaussian) pairs per view; 0: 8 x the
                                    instanced Gaussians */
    int32_t use_graph;           /* 1: capture on first use, replay on later calls */
    int32_t reserved[5];
} nvgs_batch_opts;

/* cams: n_views cameras (host); images: n_views DEVICE pointers to H x W x 3 float32 (each the
 * size of its camera); flags as for nvgs_render except that image_memory must be DEVICE and
 * keep_outputs, profile and labelling are not available (NVGS_ERR_INVALID_ARG).  With
 * blend_split_len = 0 the split length is nvgs_render's automatic one, max(4096, 4 x (the view's
 * pair count / tiles + 1)), computed on the device from the view's own count, so every view equals
 * its synchronous render bit for bit.  opts: nullable
 * (defaults).  stats: NULL (the call returns without waiting for the GPU; capacity overflows are
 * then not reported) or n_views records, in which case the call waits for the batch and returns
 * NVGS_ERR_CAPACITY if some view needed more than max_pairs pairs (that view's image is
 * incomplete) or NVGS_ERR_TIMEOUT if the tensor-core MLP gave up a wait. */
nvgs_status nvgs_render_batch(nvgs_ctx* ctx, const nvgs_camera* cams, int n_views,
                              float* const* images, const nvgs_render_flags* flags,
                              const nvgs_batch_opts* opts, nvgs_frame_stats* stats);

/* Batches of views that each render their own subset of the context's instances (Sec. 3.3 per
 * view; the paper renders one view per frame).  All views of the batch run as one flattened
 * frame: every (view, instance) pair is a frame instance with that view's transforms, the
 * in-frustum and survivor lists hold the Gaussians of every view, tile ids are global (each view's
 * tiles follow the previous view's), and every stage -- frustum, MLP, compaction, projection, both
 * sorts, duplication, compositing -- is ONE launch for the whole batch.  Nothing waits for the GPU,
 * so the batch can be captured into a CUDA graph (opts.use_graph, as for nvgs_render_batch: the
 * first call renders and captures, later calls with the same views, instance sets, flags, options
 * and images replay it with the new cameras).
 *   cams    : n_views HOST cameras (1..4096), any sizes; the tile size is flags.tile_size for all
 *   sets    : nullable HOST array of n_views instance sets; a NULL array or a set whose `instances`
 *             is NULL renders every instance of the context in that view
 *   images  : n_views DEVICE pointers to H x W x 3 float32 (each the size of its camera)
 *   flags   : as for nvgs_render_batch, and no injected logits; with blend_split_len = 0 the split
 *             length follows the automatic rule over the whole batch's pairs and tiles
 *   opts    : nullable; max_pairs is the pair capacity of the whole batch (0: 8 x its instanced
 *             Gaussians)
 *   stats   : NULL (no wait) or ONE record with the batch's totals; then the call waits and returns
 *             NVGS_ERR_CAPACITY (pairs beyond max_pairs: images incomplete) or NVGS_ERR_TIMEOUT (a
 *             bounded tensor-core wait gave up).
 * Each view's image equals nvgs_render of that view with the same instances, up to FP32 rounding of
 * the dense-tile split (bit for bit with blend_split_len < 0).  At most 2^31 instanced Gaussians
 * per batch (NVGS_ERR_CAPACITY). */
typedef struct {
    const int32_t* instances;    /* HOST: indices into the context's instances (nvgs_set_instances) */
    int32_t count;               /* number of indices */
    int32_t pad_;
} nvgs_view_instances;
nvgs_status nvgs_render_views(nvgs_ctx* ctx, const nvgs_camera* cams, const nvgs_view_instances* sets,
                              int n_views, float* const* images, const nvgs_render_flags* flags,
                              const nvgs_batch_opts* opts, nvgs_frame_stats* stats);

/* Autotuner: times nvgs_render_batch of the given views under every candidate configuration --
 * tile size {8, 16, 32} x tensor-core MLP CTAs per SM {1, 2, 3, 4} (when flags.use_mlp and every
 * MLP is BF16) x dense-tile split {automatic, never} x radix digit width {8, 6, 4} bits -- and
 * returns the fastest flags (all other
 * fields copied from `flags`).  Images do not depend on these choices.  Each candidate runs one
 * untimed batch and three timed ones (CUDA events on the context's stream); the call waits.
 * results (nullable, up to max_results entries) receives every candidate with its time per
 * view (infinity for a candidate that needs more than max_pairs pairs -- smaller tiles make more
 * pairs); n_results the number of candidates. */
typedef struct {
    int32_t tile_size, mlp_ctas_per_sm, blend_split_len;
    float ms_per_view;
    int32_t sort_digit_bits, pad_;
} nvgs_tune_result;
nvgs_status nvgs_autotune(nvgs_ctx* ctx, const nvgs_camera* cams, int n_views, float* const* images,
                          const nvgs_render_flags* flags, const nvgs_batch_opts* opts,
                          nvgs_render_flags* best, nvgs_tune_result* results, int max_results,
                          int* n_results);

/* ------------------------------------------------------------------ gradients of the render */
/* Derivatives of a loss L(image) of the last rendered frame with respect to one asset's
 * parameters: the backward pass of the 3DGS rasteriser that Sec. 3.3 hands the survivors to
 * (compositing of Sec. 4.1, EWA projection, SH colour).  Culled Gaussians (frustum, MLP) and
 * fragments the forward skipped or cut off receive nothing; the alpha clamp, the 1/255 skip, the
 * stop rule and the support cut-off are treated as constants (piecewise-smooth derivative).
 * Every array is DEVICE float32 in the layout of nvgs_asset_desc; the call ADDS into them (zero
 * them first), so several instances of the asset accumulate. */
typedef struct {
    float* means;            /* n x 3 */
    float* log_scales;       /* n x 3 */
    float* quats;            /* n x 4, with respect to the stored (unnormalised) quaternion */
    float* opacity_logits;   /* n */
    float* sh;               /* n x (sh_degree+1)^2 x 3 */
} nvgs_asset_grads;

/* dL_dimage: DEVICE H x W x 3 float32, dL/d(image) of the most recent nvgs_render on this
 * context.  That render must have used keep_outputs = 1, and no render, query or labelling call
 * may come between the two (the backward reuses its survivors, records, sorted pairs, final
 * transmittance and last-fragment indices).  Returns NVGS_ERR_INVALID_ARG for a bad asset id or
 * NULL pointer and NVGS_ERR_UNSUPPORTED when no kept frame is available. */
nvgs_status nvgs_render_backward(nvgs_ctx* ctx, const float* dL_dimage, int asset_id,
                                 const nvgs_asset_grads* grads);

/* Replace the parameters of an asset in place from DEVICE arrays (layout of nvgs_asset_desc,
 * same n and sh_degree) -- the update step of an optimiser.  The bounding box and the distance
 * range of Sec. 3.1 (the MLP's input normalisation) are those computed at load time. */
nvgs_status nvgs_update_asset(nvgs_ctx* ctx, int asset_id, const float* means,
                              const float* log_scales, const float* quats,
                              const float* opacity_logits, const float* sh);

/* Device memory the context holds (assets, MLP tiles, per-frame and training buffers), bytes. */
nvgs_status nvgs_device_bytes(const nvgs_ctx* ctx, uint64_t* bytes);

/* ------------------------------------------------------------------ internals of the last frame */
/* Device pointers into the library's buffers after the last nvgs_render (valid until the next
 * call on this context).  For tests and debugging: the survivor list (S3), projected records
 * (S4), sorted pair values and per-tile ranges (S5). */
typedef struct {
    const uint32_t* survivors;   /* 2 x n_survivors: (instance, gaussian) */
    const float* records;        /* 16 x n_survivors: u, v, conic a, b, c, opacity, det Sigma_2D,
                                    ln(alpha_min / opacity), r, g, b, depth, then the tile
                                    rectangle x0, y0, x1, y1 (inclusive) as int32 bits; a
                                    survivor without tiles has only its (empty: 1, 1, 0, 0)
                                    rectangle written */
    const int32_t* tile_rects;   /* the rectangles inside the records: 4 int32 every 16 */
    const uint32_t* pair_values; /* n_pairs survivor indices in (tile, depth) order */
    const void* pair_keys;       /* n_pairs tile ids of those pairs (non-decreasing), uint16 when
                                    pair_key_bytes = 2 (frames of at most 65536 tiles), else uint32 */
    const uint32_t* tile_ranges; /* 2 x n_tiles: [start, end) into pair_values */
    const float* final_T;        /* W x H, when flags.keep_outputs */
    const int32_t* n_contrib;    /* W x H, when flags.keep_outputs: 1 + index (into the sorted
                                    pairs) of the last fragment blended at the pixel, 0 if none */
    uint64_t n_survivors, n_pairs;
    int32_t tiles_x, tiles_y, tile_size, depth_bits; /* depth_bits: 0 (pair_keys hold tile ids) */
    int32_t pair_key_bytes, pad_;
} nvgs_frame_view;
nvgs_status nvgs_last_frame(const nvgs_ctx* ctx, nvgs_frame_view* out);

/* ------------------------------------------------------------------ building blocks */
/* Stable LSD radix sort of n (key, value) pairs on the low `key_bits` bits of the keys, in
 * place, on DEVICE arrays (the library's scratch is used for the ping-pong buffers).  Bits at or
 * above key_bits may be set; they do not influence the order.  The S5 sort of nvgs_render is this
 * routine. */
nvgs_status nvgs_sort_pairs(nvgs_ctx* ctx, uint64_t* keys, uint32_t* values, int64_t n,
                            int key_bits);

/* Allocation-free variant of nvgs_sort_pairs (the paper has no counterpart: this is a library
 * service).  For callers that cannot call cudaMalloc -- a plugin whose host application owns all
 * device memory, a real-time loop that cannot afford cudaMalloc's implicit synchronisation, or
 * code that must leave the allocator alone while its stream is recorded.  It takes no context
 * and allocates nothing: its scratch is a fixed array of about 13 MB compiled into the library,
 * held on every GPU that loads the library until the process exits.
 *   keys, values : DEVICE arrays of n pairs, sorted in place (stable, low key_bits bits)
 *   n            : 0 .. NVGS_SORT_NOALLOC_MAX_PAIRS; larger n returns NVGS_ERR_CAPACITY and
 *                  enqueues nothing
 *   cuda_stream  : cudaStream_t to enqueue on (NULL = the legacy default stream); it must
 *                  belong to the current device, else NVGS_ERR_INVALID_ARG
 * Keys may carry bits at or above key_bits; they do not influence the order.
 * The first call on a device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  The address is kept
 * for the life of the process, which assumes that every device keeps its primary context: do not
 * call this entry point after cudaDeviceReset or under another driver-API context.  All calls share
 * the one array and leave their data in it; calls that overlap on the GPU race, so serialise
 * them.  Returns NVGS_ERR_INVALID_ARG for bad arguments and NVGS_ERR_CUDA if a launch fails. */
#define NVGS_SORT_NOALLOC_MAX_PAIRS (1u << 20)
nvgs_status nvgs_sort_pairs_noalloc(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                    void* cuda_stream);

/* Self-test of the failure path of the bounded device-side waits (a library service; the paper
 * has no counterpart).  On `device`, one warp waits on an mbarrier that nothing arrives on, with
 * the helper the tensor-core MLP kernels use for their mbarrier waits (bounded by an iteration
 * count and by one second of the GPU's global timer).  Returns NVGS_OK if the wait gave up, the
 * kernel recorded it and returned; seconds_waited (HOST, nullable) receives how long it waited.
 * NVGS_ERR_INVALID_ARG for a bad device, NVGS_ERR_CUDA if a CUDA call failed or the wait did not
 * give up.  Blocks the calling thread for about a second; no fault, trap or hang is involved. */
nvgs_status nvgs_selftest_wait_timeout(int device, double* seconds_waited);

/* Measured FP32 FMA throughput of `device` in TFLOP/s (HOST *tflops; a fused multiply-add counts
 * as 2 flops): a kernel of independent FMA chains on every SM, timed with CUDA events after a
 * warm-up launch (~20 ms).  The compositing kernel's ALU roofline is quoted against it.  Returns
 * NVGS_ERR_INVALID_ARG for a bad device or NULL tflops, NVGS_ERR_CUDA if a CUDA call failed. */
nvgs_status nvgs_measure_fp32_fma(int device, double* tflops);

/* Host-side fault injection for tests: the library's next n device-buffer growths (in any
 * context of the process) fail as if cudaMalloc had run out of memory, so the calls that need them
 * return NVGS_ERR_OOM; n = 0 turns it off.  A context stays usable after such a failure. */
void nvgs_debug_fail_allocs(int n);

#ifdef __cplusplus
}
#endif
#endif /* NVGS_H */
