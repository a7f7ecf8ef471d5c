"""Thin ctypes binding of libnvgs (include/nvgs.h): argument marshalling only.

Every function below has the name of the C entry point it calls.  Pointers may be given as
torch tensors (their ``data_ptr()``; CUDA tensors for device arguments), numpy arrays (host
arguments) or ``None`` for NULL.  PyTorch only provides device memory and the stream; all work is
done by the library's CUDA kernels.  Importing this module raises if the library is missing: there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnvgs.so")

NVGS_OK, NVGS_ERR_INVALID_ARG, NVGS_ERR_OOM, NVGS_ERR_CUDA = 0, 1, 2, 3
NVGS_ERR_TIMEOUT, NVGS_ERR_CAPACITY, NVGS_ERR_UNSUPPORTED = 4, 5, 6
NVGS_MEM_HOST, NVGS_MEM_DEVICE = 0, 1
NVGS_PREC_FP32, NVGS_PREC_BF16, NVGS_PREC_FP8 = 0, 1, 2
NVGS_NUM_STAGES = 8
STAGE_NAMES = ("setup", "cull", "mlp", "compact", "project", "bin", "sort", "blend")
MLP_WEIGHTS = 10497


class NvgsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"nvgs status {status}: {msg}")
        self.status = status


class AssetDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("memory", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("train_fov_x", C.c_float),
                ("d_min", C.c_float), ("d_max", C.c_float), ("p_near", C.c_float),
                ("p_far", C.c_float)]


class Instance(C.Structure):
    _fields_ = [("asset_id", C.c_int32), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("s", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("z_near", C.c_float)]


class RenderFlags(C.Structure):
    _fields_ = [("use_mlp", C.c_int32), ("mlp_gate", C.c_int32), ("logit_threshold", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_stop", C.c_float),
                ("dilation", C.c_float), ("guard_band", C.c_float), ("bg", C.c_float * 3),
                ("tile_size", C.c_int32), ("image_memory", C.c_int32), ("profile", C.c_int32),
                ("logits_override", C.c_void_p), ("keep_outputs", C.c_int32),
                ("blend_split_len", C.c_int32), ("mlp_ctas_per_sm", C.c_int32),
                ("radius_clip_area", C.c_float), ("sort_digit_bits", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class FrameStats(C.Structure):
    _fields_ = [("n_instanced", C.c_uint64), ("n_in_frustum", C.c_uint64),
                ("n_mlp_queries", C.c_uint64), ("n_survivors", C.c_uint64),
                ("n_pairs", C.c_uint64), ("n_instances_visible", C.c_uint32),
                ("sort_passes", C.c_uint32), ("stage_ms", C.c_float * NVGS_NUM_STAGES),
                ("kernel_launches", C.c_uint64), ("blend_evaluations", C.c_uint64),
                ("blend_composited", C.c_uint64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "stage_ms"}
        d["stage_ms"] = dict(zip(STAGE_NAMES, list(self.stage_ms)))
        return d


class FrameView(C.Structure):
    _fields_ = [("survivors", C.c_void_p), ("records", C.c_void_p), ("tile_rects", C.c_void_p),
                ("pair_values", C.c_void_p), ("pair_keys", C.c_void_p), ("tile_ranges", C.c_void_p),
                ("final_T", C.c_void_p), ("n_contrib", C.c_void_p), ("n_survivors", C.c_uint64),
                ("n_pairs", C.c_uint64), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32),
                ("tile_size", C.c_int32), ("depth_bits", C.c_int32), ("pair_key_bytes", C.c_int32),
                ("pad_", C.c_int32)]


class AssetInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("has_mlp", C.c_int32),
                ("bbox_center", C.c_float * 3), ("bbox_half_extent", C.c_float * 3),
                ("d_min", C.c_float), ("d_max", C.c_float), ("train_fov_x", C.c_float)]


class TrainBatch(C.Structure):
    _fields_ = [("labels", C.c_void_p), ("batch", C.c_int32), ("precision", C.c_int32),
                ("sample_view", C.c_void_p), ("sample_gauss", C.c_void_p), ("seed", C.c_uint64)]


class AdamCfg(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32)]


class BatchOpts(C.Structure):
    _fields_ = [("max_pairs", C.c_int64), ("use_graph", C.c_int32), ("reserved", C.c_int32 * 5)]


class TuneResult(C.Structure):
    _fields_ = [("tile_size", C.c_int32), ("mlp_ctas_per_sm", C.c_int32), ("blend_split_len", C.c_int32),
                ("ms_per_view", C.c_float), ("sort_digit_bits", C.c_int32), ("pad_", C.c_int32)]


class ViewOpts(C.Structure):
    _fields_ = [("n_dirs", C.c_int32), ("n_dist", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("n_aux", C.c_int32), ("aux_angle", C.c_float), ("random_offset", C.c_int32),
                ("pad_", C.c_int32), ("seed", C.c_uint64)]


class AssetGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_uint64), ("total_ms", C.c_double)]


EXPORTS = ("nvgs_create", "nvgs_destroy", "nvgs_last_error", "nvgs_get_stream", "nvgs_default_flags",
           "nvgs_abi_version", "nvgs_load_asset", "nvgs_set_mlp", "nvgs_set_instances",
           "nvgs_scene_info", "nvgs_query_visibility", "nvgs_render", "nvgs_last_frame",
           "nvgs_sort_pairs", "nvgs_kernel_stats", "nvgs_reset_kernel_stats",
           "nvgs_sort_pairs_noalloc", "nvgs_label_visibility", "nvgs_train_init",
           "nvgs_train_visibility_step", "nvgs_train_get_weights", "nvgs_lr_schedule",
           "nvgs_get_asset_info", "nvgs_training_views", "nvgs_render_backward",
           "nvgs_update_asset", "nvgs_render_batch", "nvgs_render_views", "nvgs_autotune", "nvgs_device_bytes",
           "nvgs_selftest_wait_timeout", "nvgs_measure_fp32_fma", "nvgs_training_views_ex",
           "nvgs_train_save_state", "nvgs_train_load_state", "nvgs_debug_fail_allocs")
NVGS_SORT_NOALLOC_MAX_PAIRS = 1 << 20


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2511_19202_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, P = C.c_void_p, C.POINTER
    L.nvgs_create.argtypes = [P(vp), C.c_int, vp]
    L.nvgs_destroy.argtypes = [vp]
    L.nvgs_last_error.argtypes = [vp]
    L.nvgs_last_error.restype = C.c_char_p
    L.nvgs_get_stream.argtypes = [vp]
    L.nvgs_get_stream.restype = vp
    L.nvgs_default_flags.argtypes = [P(RenderFlags)]
    L.nvgs_default_flags.restype = None
    L.nvgs_abi_version.restype = C.c_int
    L.nvgs_load_asset.argtypes = [vp, P(AssetDesc), P(C.c_int)]
    L.nvgs_set_mlp.argtypes = [vp, C.c_int, vp, C.c_int]
    L.nvgs_set_instances.argtypes = [vp, vp, C.c_int]
    L.nvgs_scene_info.argtypes = [vp, P(C.c_int64), P(C.c_int), P(C.c_int)]
    L.nvgs_query_visibility.argtypes = [vp, P(Camera), P(RenderFlags), vp, vp, P(FrameStats)]
    L.nvgs_render.argtypes = [vp, P(Camera), P(RenderFlags), vp, P(FrameStats)]
    L.nvgs_last_frame.argtypes = [vp, P(FrameView)]
    L.nvgs_sort_pairs.argtypes = [vp, vp, vp, C.c_int64, C.c_int]
    L.nvgs_kernel_stats.argtypes = [vp, vp, C.c_int, P(C.c_int)]
    L.nvgs_reset_kernel_stats.argtypes = [vp]
    L.nvgs_sort_pairs_noalloc.argtypes = [vp, vp, C.c_int64, C.c_int, vp]
    L.nvgs_selftest_wait_timeout.argtypes = [C.c_int, P(C.c_double)]
    L.nvgs_measure_fp32_fma.argtypes = [C.c_int, P(C.c_double)]
    L.nvgs_label_visibility.argtypes = [vp, C.c_int, vp, C.c_int, C.c_int, P(RenderFlags), vp]
    L.nvgs_train_init.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.nvgs_train_visibility_step.argtypes = [vp, C.c_int, P(TrainBatch), P(AdamCfg), P(C.c_float)]
    L.nvgs_train_get_weights.argtypes = [vp, C.c_int, vp]
    L.nvgs_lr_schedule.argtypes = [C.c_int, C.c_int, C.c_float, C.c_float, C.c_float]
    L.nvgs_lr_schedule.restype = C.c_float
    L.nvgs_get_asset_info.argtypes = [vp, C.c_int, P(AssetInfo)]
    L.nvgs_training_views.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]
    L.nvgs_training_views_ex.argtypes = [vp, C.c_int, P(ViewOpts), vp]
    L.nvgs_train_save_state.argtypes = [vp, C.c_int, vp]
    L.nvgs_debug_fail_allocs.argtypes = [C.c_int]
    L.nvgs_debug_fail_allocs.restype = None
    L.nvgs_train_load_state.argtypes = [vp, C.c_int, vp]
    L.nvgs_render_backward.argtypes = [vp, vp, C.c_int, P(AssetGrads)]
    L.nvgs_device_bytes.argtypes = [vp, P(C.c_uint64)]
    L.nvgs_render_batch.argtypes = [vp, vp, C.c_int, vp, P(RenderFlags), P(BatchOpts), vp]
    L.nvgs_render_views.argtypes = [vp, vp, vp, C.c_int, vp, P(RenderFlags), P(BatchOpts), vp]
    L.nvgs_autotune.argtypes = [vp, vp, C.c_int, vp, P(RenderFlags), P(BatchOpts), P(RenderFlags), vp, C.c_int,
                                P(C.c_int)]
    L.nvgs_update_asset.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("nvgs_default_flags", "nvgs_abi_version", "nvgs_last_error", "nvgs_get_stream",
                        "nvgs_lr_schedule"):
            getattr(L, name).restype = C.c_int
    return L


lib = _load()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(ctx, st):
    if st != NVGS_OK:
        msg = lib.nvgs_last_error(ctx).decode() if ctx else ""
        raise NvgsError(st, msg)


# ----------------------------------------------------------------------------- C entry points
def nvgs_create(device: int = 0, stream=None):
    h = C.c_void_p()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(None, lib.nvgs_create(C.byref(h), int(device), s))
    return h


def nvgs_destroy(ctx):
    _check(None, lib.nvgs_destroy(ctx))


def nvgs_last_error(ctx) -> str:
    return lib.nvgs_last_error(ctx).decode()


def nvgs_get_stream(ctx) -> int:
    return lib.nvgs_get_stream(ctx)


def nvgs_default_flags(**overrides) -> RenderFlags:
    f = RenderFlags()
    lib.nvgs_default_flags(C.byref(f))
    for k, v in overrides.items():
        if k == "bg":
            f.bg[:] = [float(x) for x in v]
        elif k == "logits_override":
            f.logits_override = _ptr(v)
        else:
            setattr(f, k, v)
    return f


def nvgs_abi_version() -> int:
    return lib.nvgs_abi_version()


def nvgs_load_asset(ctx, asset, d_min=0.0, d_max=0.0, p_near=0.0, p_far=0.0) -> int:
    """``asset`` has means, log_scales, quats, opacity_logits, sh (numpy float32, host) and
    sh_degree, train_fov_x attributes."""
    arrs = [np.ascontiguousarray(getattr(asset, k), np.float32)
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    d = AssetDesc()
    d.n = int(arrs[0].shape[0])
    d.sh_degree = int(asset.sh_degree)
    d.memory = NVGS_MEM_HOST
    d.means, d.log_scales, d.quats, d.opacity_logits, d.sh = [a.ctypes.data for a in arrs]
    d.train_fov_x = float(asset.train_fov_x)
    d.d_min, d.d_max, d.p_near, d.p_far = float(d_min), float(d_max), float(p_near), float(p_far)
    out = C.c_int(-1)
    _check(ctx, lib.nvgs_load_asset(ctx, C.byref(d), C.byref(out)))
    return out.value


def flat_weights(w) -> np.ndarray:
    if isinstance(w, dict):
        parts = []
        for k in range(1, 5):
            parts += [np.asarray(w[f"W{k}"], np.float32).ravel(), np.asarray(w[f"b{k}"], np.float32).ravel()]
        w = np.concatenate(parts)
    w = np.ascontiguousarray(w, np.float32)
    assert w.size == MLP_WEIGHTS
    return w


def nvgs_set_mlp(ctx, asset_id: int, weights, precision: int = NVGS_PREC_FP32):
    w = flat_weights(weights)
    _check(ctx, lib.nvgs_set_mlp(ctx, int(asset_id), w.ctypes.data, int(precision)))


def nvgs_set_instances(ctx, instances):
    arr = (Instance * len(instances))()
    for k, i in enumerate(instances):
        arr[k].asset_id = int(i.asset_id)
        arr[k].R[:] = [float(x) for x in np.asarray(i.R, np.float32).ravel()]
        arr[k].t[:] = [float(x) for x in np.asarray(i.t, np.float32).ravel()]
        arr[k].s = float(i.s)
    _check(ctx, lib.nvgs_set_instances(ctx, C.cast(arr, C.c_void_p), len(instances)))


def nvgs_scene_info(ctx):
    n = C.c_int64()
    a = C.c_int()
    i = C.c_int()
    _check(ctx, lib.nvgs_scene_info(ctx, C.byref(n), C.byref(a), C.byref(i)))
    return n.value, a.value, i.value


def camera(cam) -> Camera:
    c = Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).ravel()]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).ravel()]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.z_near = int(cam.width), int(cam.height), float(cam.z_near)
    return c


def nvgs_query_visibility(ctx, cam, flags: RenderFlags, logits=None, keep=None) -> FrameStats:
    st = FrameStats()
    _check(ctx, lib.nvgs_query_visibility(ctx, C.byref(camera(cam)), C.byref(flags), _ptr(logits),
                                          _ptr(keep), C.byref(st)))
    return st


def nvgs_render(ctx, cam, flags: RenderFlags, image) -> FrameStats:
    st = FrameStats()
    _check(ctx, lib.nvgs_render(ctx, C.byref(camera(cam)), C.byref(flags), _ptr(image), C.byref(st)))
    return st


def nvgs_last_frame(ctx) -> FrameView:
    v = FrameView()
    _check(ctx, lib.nvgs_last_frame(ctx, C.byref(v)))
    return v


def nvgs_sort_pairs(ctx, keys, values, n: int, key_bits: int):
    _check(ctx, lib.nvgs_sort_pairs(ctx, _ptr(keys), _ptr(values), int(n), int(key_bits)))


def nvgs_kernel_stats(ctx):
    """{kernel name: (launches, total device ms)} over the profiled frames since the last reset."""
    n = C.c_int(0)
    _check(ctx, lib.nvgs_kernel_stats(ctx, None, 0, C.byref(n)))
    arr = (KernelStat * max(1, n.value))()
    _check(ctx, lib.nvgs_kernel_stats(ctx, C.cast(arr, C.c_void_p), n.value, C.byref(n)))
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms)) for k in range(n.value)}


def nvgs_reset_kernel_stats(ctx):
    _check(ctx, lib.nvgs_reset_kernel_stats(ctx))


def nvgs_sort_pairs_noalloc(keys, values, n: int, key_bits: int, stream=None) -> int:
    """Allocation-free sort (fixed scratch inside the library, at most
    NVGS_SORT_NOALLOC_MAX_PAIRS pairs).  Returns the nvgs status code; raises nothing, so that
    callers can test the capacity error."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return lib.nvgs_sort_pairs_noalloc(_ptr(keys), _ptr(values), int(n), int(key_bits), s)


def nvgs_selftest_wait_timeout(device: int = 0):
    """(status, seconds waited) of the bounded-wait self-test (NVGS_OK: the wait gave up as it
    must, the kernel returned)."""
    sec = C.c_double(0.0)
    st = lib.nvgs_selftest_wait_timeout(int(device), C.byref(sec))
    return st, sec.value


def nvgs_measure_fp32_fma(device: int = 0) -> float:
    """Measured FP32 FMA throughput of the device, TFLOP/s."""
    t = C.c_double(0.0)
    _check(None, lib.nvgs_measure_fp32_fma(int(device), C.byref(t)))
    return t.value


def _cam_array(cams):
    if isinstance(cams, C.Array):
        return cams
    arr = (Camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = c if isinstance(c, Camera) else camera(c)
    return arr


def nvgs_label_visibility(ctx, asset_id: int, views, flags: RenderFlags, labels, group: int = 1):
    arr = _cam_array(views)
    _check(ctx, lib.nvgs_label_visibility(ctx, int(asset_id), C.cast(arr, C.c_void_p), len(arr),
                                          int(group), C.byref(flags), _ptr(labels)))


def nvgs_train_init(ctx, asset_id: int, w0, views):
    w = flat_weights(w0)
    arr = _cam_array(views)
    _check(ctx, lib.nvgs_train_init(ctx, int(asset_id), w.ctypes.data, C.cast(arr, C.c_void_p), len(arr)))


def nvgs_train_visibility_step(ctx, asset_id: int, labels, batch: int, step: int, lr: float,
                               seed: int = 0, sample_view=None, sample_gauss=None,
                               beta1=0.9, beta2=0.999, eps=1e-8, want_loss=False, precision=0):
    b = TrainBatch()
    b.labels = _ptr(labels)
    b.batch = int(batch)
    b.precision = int(precision)
    b.sample_view = _ptr(sample_view)
    b.sample_gauss = _ptr(sample_gauss)
    b.seed = int(seed)
    a = AdamCfg()
    a.lr, a.beta1, a.beta2, a.eps, a.step = float(lr), float(beta1), float(beta2), float(eps), int(step)
    loss = C.c_float(float("nan"))
    _check(ctx, lib.nvgs_train_visibility_step(ctx, int(asset_id), C.byref(b), C.byref(a),
                                               C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def nvgs_train_get_weights(ctx, asset_id: int) -> np.ndarray:
    w = np.zeros(MLP_WEIGHTS, np.float32)
    _check(ctx, lib.nvgs_train_get_weights(ctx, int(asset_id), w.ctypes.data))
    return w


def nvgs_lr_schedule(step: int, total: int, lr0: float, lr1: float, warmup_frac: float) -> float:
    return lib.nvgs_lr_schedule(int(step), int(total), float(lr0), float(lr1), float(warmup_frac))


def nvgs_get_asset_info(ctx, asset_id: int) -> AssetInfo:
    out = AssetInfo()
    _check(ctx, lib.nvgs_get_asset_info(ctx, int(asset_id), C.byref(out)))
    return out


def nvgs_training_views(ctx, asset_id: int, n_dirs: int, n_dist: int, width: int, height: int):
    arr = (Camera * (n_dirs * n_dist))()
    _check(ctx, lib.nvgs_training_views(ctx, int(asset_id), int(n_dirs), int(n_dist), int(width),
                                        int(height), C.cast(arr, C.c_void_p)))
    return arr


def nvgs_debug_fail_allocs(n: int) -> None:
    """Test hook: the library's next n device-buffer growths fail as out-of-memory (0: off)."""
    lib.nvgs_debug_fail_allocs(int(n))


NVGS_TRAIN_STATE_FLOATS = 3 * 10497


def nvgs_train_save_state(ctx, asset_id: int) -> np.ndarray:
    """Training checkpoint: FP32 master weights and Adam moments (w, m, v) as one float32 array."""
    out = np.empty(NVGS_TRAIN_STATE_FLOATS, np.float32)
    _check(ctx, lib.nvgs_train_save_state(ctx, int(asset_id), out.ctypes.data))
    return out


def nvgs_train_load_state(ctx, asset_id: int, state) -> None:
    st = np.ascontiguousarray(state, dtype=np.float32)
    if st.size != NVGS_TRAIN_STATE_FLOATS:
        raise ValueError(f"state must hold {NVGS_TRAIN_STATE_FLOATS} floats")
    _check(ctx, lib.nvgs_train_load_state(ctx, int(asset_id), st.ctypes.data))


def nvgs_training_views_ex(ctx, asset_id: int, n_dirs: int, n_dist: int, width: int, height: int,
                           n_aux: int = 0, aux_angle: float = 0.0, random_offset: bool = False,
                           seed: int = 0):
    """Main views, each followed by its n_aux auxiliary cone views (label with group = 1 + n_aux)."""
    o = ViewOpts(int(n_dirs), int(n_dist), int(width), int(height), int(n_aux), float(aux_angle),
                 1 if random_offset else 0, 0, int(seed) & 0xFFFFFFFFFFFFFFFF)
    arr = (Camera * (n_dirs * n_dist * (1 + n_aux)))()
    _check(ctx, lib.nvgs_training_views_ex(ctx, int(asset_id), C.byref(o), C.cast(arr, C.c_void_p)))
    return arr


def nvgs_render_backward(ctx, dL_dimage, asset_id: int, means, log_scales, quats, opacity_logits, sh):
    """Adds dL/d(parameters) of asset `asset_id` into the five device arrays, for dL/d(image) of
    the last render (which must have kept its outputs)."""
    g = AssetGrads(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh))
    _check(ctx, lib.nvgs_render_backward(ctx, _ptr(dL_dimage), int(asset_id), C.byref(g)))


def nvgs_update_asset(ctx, asset_id: int, means, log_scales, quats, opacity_logits, sh):
    _check(ctx, lib.nvgs_update_asset(ctx, int(asset_id), _ptr(means), _ptr(log_scales), _ptr(quats),
                                      _ptr(opacity_logits), _ptr(sh)))


def nvgs_render_batch(ctx, cams, flags: RenderFlags, images, max_pairs: int = 0, use_graph: bool = False,
                      want_stats: bool = True):
    """Renders len(cams) views into the device images (one per camera) without host synchronisation;
    with want_stats the call waits and returns one stats dict per view."""
    n = len(cams)
    arr = (Camera * n)(*[camera(c) for c in cams])
    ptrs = (C.c_void_p * n)(*[_ptr(im) for im in images])
    o = BatchOpts(int(max_pairs), 1 if use_graph else 0)
    st = (FrameStats * n)() if want_stats else None
    _check(ctx, lib.nvgs_render_batch(ctx, C.cast(arr, C.c_void_p), n, C.cast(ptrs, C.c_void_p), C.byref(flags),
                                      C.byref(o), C.cast(st, C.c_void_p) if st is not None else None))
    return [st[k].as_dict() for k in range(n)] if st is not None else None


def nvgs_autotune(ctx, cams, flags: RenderFlags, images, max_pairs: int = 0):
    """(best flags, [ {tile_size, mlp_ctas_per_sm, blend_split_len, sort_digit_bits, ms_per_view}
    ... ])."""
    n = len(cams)
    arr = (Camera * n)(*[camera(c) for c in cams])
    ptrs = (C.c_void_p * n)(*[_ptr(im) for im in images])
    o = BatchOpts(int(max_pairs), 0)
    best = RenderFlags()
    cap = 256
    res = (TuneResult * cap)()
    cnt = C.c_int(0)
    _check(ctx, lib.nvgs_autotune(ctx, C.cast(arr, C.c_void_p), n, C.cast(ptrs, C.c_void_p), C.byref(flags),
                                  C.byref(o), C.byref(best), C.cast(res, C.c_void_p), cap, C.byref(cnt)))
    table = [dict(tile_size=res[k].tile_size, mlp_ctas_per_sm=res[k].mlp_ctas_per_sm,
                  blend_split_len=res[k].blend_split_len, sort_digit_bits=res[k].sort_digit_bits,
                  ms_per_view=res[k].ms_per_view)
             for k in range(min(cnt.value, cap))]
    return best, table


class ViewInstances(C.Structure):
    _fields_ = [("instances", C.c_void_p), ("count", C.c_int32), ("pad_", C.c_int32)]


def nvgs_render_views(ctx, cams, instance_sets, flags: RenderFlags, images, max_pairs: int = 0,
                      use_graph: bool = False, want_stats: bool = True):
    """Views with their own instance subsets (None: every instance), one launch per stage for the
    whole batch; returns the batch's totals (or None without stats)."""
    n = len(cams)
    arr = (Camera * n)(*[camera(c) for c in cams])
    ptrs = (C.c_void_p * n)(*[_ptr(im) for im in images])
    keep = []
    sets = (ViewInstances * n)()
    for k, idx in enumerate(instance_sets if instance_sets is not None else [None] * n):
        if idx is not None:
            a = np.ascontiguousarray(idx, np.int32)
            keep.append(a)
            sets[k].instances = a.ctypes.data
            sets[k].count = a.size
    o = BatchOpts(int(max_pairs), 1 if use_graph else 0)
    st = FrameStats() if want_stats else None
    _check(ctx, lib.nvgs_render_views(ctx, C.cast(arr, C.c_void_p), C.cast(sets, C.c_void_p), n,
                                      C.cast(ptrs, C.c_void_p), C.byref(flags), C.byref(o),
                                      C.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def nvgs_device_bytes(ctx) -> int:
    b = C.c_uint64(0)
    _check(ctx, lib.nvgs_device_bytes(ctx, C.byref(b)))
    return int(b.value)
