"""FP64 CPU oracle of the NVGS render pass — TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline / reference leg may
import this package.  The CUDA library never calls it and shares no code with it; both only read
the seeded inputs drawn by the ``scenes`` package.

The arithmetic lives in ``nvgs_oracle.c`` (plain C, double precision, OpenMP over pixel rows);
this module only marshals numpy arrays into it.  Each wrapper names the part of the paper it
restates:

* ``distance_bound``         Sec. 3.1, Eq. 1
* ``prepare``                Sec. 3.1 (bounding box of the means, near / far distances)
* ``frustum``                Sec. 3.3 (frustum culling on the Gaussian mean)
* ``visibility``/``features``/``mlp_forward``  Sec. 3.2-3.3 and Eq. 2 (MLP inputs, forward)
* ``project``                Sec. 3.3 -> original 3DGS preprocessing (EWA splat, SH colour)
* ``composite``/``render``   Sec. 4.1 blending rules, exact per-pixel depth-sorted compositing
* ``labels``                 Sec. 3.1 (contribution alpha * T; visible iff it blends)
* ``tile_lists``/``tile_lists_ellipse``  Sec. 3.3 -> tiled rasterisation: per-tile lists in blend
  order (support rectangle, exact pixel support, and the support ellipse met by each tile's
  pixel-centre box, with the band a conservative binner may take either way)

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force or independent library routines.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nvgs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrAsset(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("pad_", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p),
                ("bbox_min", C.c_double * 3), ("bbox_max", C.c_double * 3),
                ("d_min", C.c_double), ("d_max", C.c_double), ("train_focal", C.c_double)]


class OrInstance(C.Structure):
    _fields_ = [("asset_id", C.c_int32), ("pad_", C.c_int32), ("R", C.c_double * 9),
                ("t", C.c_double * 3), ("s", C.c_double)]


class OrCamera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("z_near", C.c_double)]


class OrOpts(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double), ("t_stop", C.c_double),
                ("dilation", C.c_double), ("guard_band", C.c_double), ("bg", C.c_double * 3),
                ("tile_size", C.c_int32), ("pad_", C.c_int32), ("eps_alpha", C.c_double),
                ("eps_t", C.c_double), ("eps_depth", C.c_double), ("eps_frustum", C.c_double),
                ("eps_px", C.c_double), ("swap_tol", C.c_double),
                ("radius_clip_area", C.c_double), ("eps_clip", C.c_double)]


SPLAT_DTYPE = np.dtype([
    ("valid", np.int32), ("ambiguous", np.int32), ("instance", np.int32), ("gaussian", np.int32),
    ("u", np.float64), ("v", np.float64), ("depth", np.float64), ("cov", np.float64, 3),
    ("conic", np.float64, 3), ("opacity", np.float64), ("rgb", np.float64, 3),
    ("x_ext", np.float64), ("y_ext", np.float64), ("px_min", np.int32, 2),
    ("px_max", np.int32, 2), ("tile_min", np.int32, 2), ("tile_max", np.int32, 2)], align=True)
assert SPLAT_DTYPE.itemsize == 168


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            vp = C.c_void_p
            L.or_distance_bound.restype = C.c_double
            L.or_distance_bound.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_asset_prepare.argtypes = [P(OrAsset), C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_double]
            L.or_frustum.argtypes = [P(OrAsset), P(OrInstance), C.c_int, P(OrCamera), P(OrOpts),
                                     vp, vp]
            L.or_normalised_distance.restype = C.c_double
            L.or_normalised_distance.argtypes = [C.c_double] * 5
            L.or_mlp_features.argtypes = [P(OrAsset), vp, vp, C.c_double, vp]
            L.or_mlp_forward.argtypes = [vp, C.c_int64, vp, vp]
            L.or_visibility.argtypes = [P(OrAsset), P(OrInstance), C.c_int, P(OrCamera), vp,
                                        C.c_int, vp, vp, vp]
            L.or_visibility_at.restype = C.c_int
            L.or_visibility_at.argtypes = [P(OrAsset), P(OrInstance), C.c_int, P(OrCamera), vp,
                                           C.c_int, vp, C.c_int64, vp, vp, vp]
            L.or_sh_basis.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, vp]
            L.or_quat_to_rot.argtypes = [vp, vp]
            L.or_cov3d.argtypes = [vp, vp, vp]
            L.or_project.argtypes = [P(OrAsset), P(OrInstance), C.c_int, P(OrCamera), P(OrOpts),
                                     vp, vp, vp]
            L.or_composite.argtypes = [vp, C.c_int64, P(OrCamera), P(OrOpts), vp, C.c_int, vp, vp,
                                       vp, vp, C.c_int]
            L.or_render_rows.restype = C.c_int64
            L.or_render_rows.argtypes = [P(OrAsset), P(OrInstance), C.c_int, P(OrCamera), P(OrOpts),
                                         vp, vp, vp, C.c_int, vp, vp, vp]
            L.or_pixel_weights.restype = C.c_int
            L.or_pixel_weights.argtypes = [vp, C.c_int64, P(OrCamera), P(OrOpts), C.c_int,
                                           C.c_int, vp, C.c_int, P(C.c_double)]
            L.or_train_loss_grad.restype = C.c_double
            L.or_train_loss_grad.argtypes = [P(OrAsset), vp, vp, C.c_int64, vp, vp, C.c_int64, vp, vp]
            L.or_train_step.restype = C.c_double
            L.or_train_step.argtypes = [P(OrAsset), vp, vp, C.c_int64, vp, vp, C.c_int64, vp, vp, vp,
                                        C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]
            L.or_num_threads.restype = C.c_int
            L.or_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ----------------------------------------------------------------------------- options
def opts(alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4, dilation=0.3, guard_band=1.3,
         bg=(0.0, 0.0, 0.0), tile_size=16, eps_alpha=2e-4, eps_t=2e-4, eps_depth=4e-7,
         eps_frustum=1e-6, eps_px=1e-3, swap_tol=5e-4, radius_clip_area=0.0,
         eps_clip=1e-3) -> OrOpts:
    """Blending constants of Sec. 4.1 and the 3DGS conventions, radius clipping (Sec. 4.4; 0:
    off), plus ambiguity-band widths."""
    o = OrOpts()
    o.alpha_min, o.alpha_max, o.t_stop = alpha_min, alpha_max, t_stop
    o.dilation, o.guard_band = dilation, guard_band
    o.bg[:] = [float(b) for b in bg]
    o.tile_size = int(tile_size)
    o.eps_alpha, o.eps_t, o.eps_depth = eps_alpha, eps_t, eps_depth
    o.eps_frustum, o.eps_px, o.swap_tol = eps_frustum, eps_px, swap_tol
    o.radius_clip_area, o.eps_clip = radius_clip_area, eps_clip
    return o


# ----------------------------------------------------------------------------- scene marshalling
class OracleScene:
    """FP64 copy of a ``scenes.Scene`` plus the per-asset constants of Sec. 3.1."""

    def __init__(self, scene, theta_t=None, p_near=0.9, p_far=0.05, d_min=0.0, d_max=0.0):
        L = lib()
        self.scene = scene
        self._keep = []
        self.assets = (OrAsset * len(scene.assets))()
        for k, a in enumerate(scene.assets):
            arrs = [np.ascontiguousarray(x, np.float64) for x in
                    (a.means, a.log_scales, a.quats, a.opacity_logits, a.sh)]
            self._keep.append(arrs)
            s = self.assets[k]
            s.n, s.sh_degree = a.n, a.sh_degree
            s.means, s.log_scales, s.quats, s.opacity_logits, s.sh = [x.ctypes.data for x in arrs]
            th = a.train_fov_x if theta_t is None else theta_t
            L.or_asset_prepare(C.byref(s), th, p_near, p_far, d_min, d_max)
        self.instances = (OrInstance * len(scene.instances))()
        for k, i in enumerate(scene.instances):
            d = self.instances[k]
            d.asset_id = i.asset_id
            d.R[:] = [float(x) for x in np.asarray(i.R, np.float64).ravel()]
            d.t[:] = [float(x) for x in np.asarray(i.t, np.float64)]
            d.s = float(i.s)
        self.n_inst = len(scene.instances)
        self.n_instanced = scene.n_instanced

    def asset_constants(self, k):
        s = self.assets[k]
        return dict(bbox_min=np.array(s.bbox_min[:]), bbox_max=np.array(s.bbox_max[:]),
                    d_min=s.d_min, d_max=s.d_max, train_focal=s.train_focal)


def camera(cam) -> OrCamera:
    c = OrCamera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float64).ravel()]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float64)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.z_near = int(cam.width), int(cam.height), float(cam.z_near)
    return c


def flat_weights(w: dict) -> np.ndarray:
    parts = []
    for li in range(1, 5):
        parts += [np.asarray(w[f"W{li}"], np.float64).ravel(), np.asarray(w[f"b{li}"], np.float64).ravel()]
    out = np.concatenate(parts)
    assert out.size == 10497
    return out


# ----------------------------------------------------------------------------- wrappers
def distance_bound(r, theta, p):
    """Eq. 1: d = r / (tan(theta / 2) p)."""
    return lib().or_distance_bound(float(r), float(theta), float(p))


def normalised_distance(d_local, f_t, f_r, d_min, d_max):
    """Eq. 2 then the min-max map of Sec. 3.3 on log distance, clamped to [-1, 1]."""
    return lib().or_normalised_distance(float(d_local), float(f_t), float(f_r), float(d_min), float(d_max))


def frustum(osc: OracleScene, cam, o=None):
    o = o or opts()
    n = osc.n_instanced
    inside = np.zeros(n, np.uint8)
    amb = np.zeros(n, np.uint8)
    lib().or_frustum(osc.assets, osc.instances, osc.n_inst, C.byref(camera(cam)), C.byref(o),
                     _ptr(inside), _ptr(amb))
    return inside.astype(bool), amb.astype(bool)


def visibility(osc: OracleScene, cam, weights=None, gate=False, return_features=False):
    """Per instanced Gaussian: MLP logit, whether the instance bypasses the MLP, and features."""
    n = osc.n_instanced
    logits = np.zeros(n, np.float64)
    gated = np.zeros(n, np.uint8)
    feats = np.zeros((n, 32), np.float64) if return_features else None
    w = flat_weights(weights) if weights is not None else None
    lib().or_visibility(osc.assets, osc.instances, osc.n_inst, C.byref(camera(cam)), _ptr(w),
                        int(bool(gate)), _ptr(logits), _ptr(gated), _ptr(feats))
    out = dict(logits=logits, gated=gated.astype(bool))
    if return_features:
        out["features"] = feats
    return out


def visibility_at(osc: OracleScene, cam, idx, weights=None, gate=False, return_features=False):
    """visibility() at the instanced Gaussians `idx` (instance-major indices) only, each value
    computed exactly as visibility() computes it."""
    idx = np.ascontiguousarray(idx, np.int64)
    n = idx.size
    logits = np.zeros(n, np.float64)
    gated = np.zeros(n, np.uint8)
    feats = np.zeros((n, 32), np.float64) if return_features else None
    w = flat_weights(weights) if weights is not None else None
    rc = lib().or_visibility_at(osc.assets, osc.instances, osc.n_inst, C.byref(camera(cam)), _ptr(w),
                                int(bool(gate)), _ptr(idx), n, _ptr(logits), _ptr(gated), _ptr(feats))
    if rc != 0:
        raise ValueError("visibility_at: index out of range or allocation failed")
    out = dict(logits=logits, gated=gated.astype(bool))
    if return_features:
        out["features"] = feats
    return out


def features(osc: OracleScene, asset_k: int, mu, cam_local, f_r):
    f = np.zeros(32, np.float64)
    mu = np.ascontiguousarray(mu, np.float64)
    cl = np.ascontiguousarray(cam_local, np.float64)
    lib().or_mlp_features(C.byref(osc.assets[asset_k]), _ptr(mu), _ptr(cl), float(f_r), _ptr(f))
    return f


def mlp_forward(weights: dict, feats: np.ndarray) -> np.ndarray:
    feats = np.ascontiguousarray(feats, np.float64).reshape(-1, 32)
    out = np.zeros(feats.shape[0], np.float64)
    w = flat_weights(weights)
    lib().or_mlp_forward(_ptr(w), feats.shape[0], _ptr(feats), _ptr(out))
    return out


def sh_basis(degree: int, dirs: np.ndarray) -> np.ndarray:
    dirs = np.asarray(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((dirs.shape[0], 16), np.float64)
    y = np.zeros(16, np.float64)
    for i, (a, b, c) in enumerate(dirs):
        lib().or_sh_basis(int(degree), float(a), float(b), float(c), _ptr(y))
        out[i] = y
    return out[:, :(degree + 1) ** 2]


def quat_to_rot(q) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9, np.float64)
    lib().or_quat_to_rot(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def cov3d(log_scale, quat) -> np.ndarray:
    ls = np.ascontiguousarray(log_scale, np.float64)
    q = np.ascontiguousarray(quat, np.float64)
    S = np.zeros(9, np.float64)
    lib().or_cov3d(_ptr(ls), _ptr(q), _ptr(S))
    return S.reshape(3, 3)


def project(osc: OracleScene, cam, o=None, keep=None, keep_amb=None) -> np.ndarray:
    o = o or opts()
    out = np.zeros(osc.n_instanced, SPLAT_DTYPE)
    k = None if keep is None else np.ascontiguousarray(keep, np.uint8)
    ka = None if keep_amb is None else np.ascontiguousarray(keep_amb, np.uint8)
    lib().or_project(osc.assets, osc.instances, osc.n_inst, C.byref(camera(cam)), C.byref(o),
                     _ptr(k), _ptr(ka), _ptr(out))
    return out


def composite(splats: np.ndarray, cam, o=None, rows=None, brute_force=False,
              want_contrib=False):
    o = o or opts()
    splats = np.ascontiguousarray(splats, SPLAT_DTYPE)
    H, W = int(cam.height), int(cam.width)
    r = None if rows is None else np.ascontiguousarray(rows, np.int32)
    nr = H if r is None else r.size
    image = np.zeros((nr, W, 3), np.float64)
    T = np.zeros((nr, W), np.float64)
    amb = np.zeros((nr, W), np.uint8)
    contrib = np.zeros(splats.shape[0], np.int32) if want_contrib else None
    lib().or_composite(_ptr(splats), splats.shape[0], C.byref(camera(cam)), C.byref(o), _ptr(r),
                       nr, _ptr(image), _ptr(T), _ptr(contrib), _ptr(amb), int(bool(brute_force)))
    out = dict(image=image, T=T, ambiguous=amb.astype(bool))
    if want_contrib:
        out["n_contrib"] = contrib
    return out


def render(osc: OracleScene, cam, o=None, keep=None, keep_amb=None, rows=None,
           want_contrib=False):
    """Exact FP64 render: frustum, optional culling decision, projection, compositing."""
    o = o or opts()
    sp = project(osc, cam, o, keep, keep_amb)
    out = composite(sp, cam, o, rows=rows, want_contrib=want_contrib)
    out["splats"] = sp
    return out


def render_rows(osc: OracleScene, cam, rows, o=None, keep=None, keep_amb=None):
    """Exact FP64 render of the given pixel rows only (memory-light: splats that reach no
    requested row are projected and dropped)."""
    o = o or opts()
    r = np.ascontiguousarray(rows, np.int32)
    W = int(cam.width)
    image = np.zeros((r.size, W, 3), np.float64)
    T = np.zeros((r.size, W), np.float64)
    amb = np.zeros((r.size, W), np.uint8)
    k = None if keep is None else np.ascontiguousarray(keep, np.uint8)
    ka = None if keep_amb is None else np.ascontiguousarray(keep_amb, np.uint8)
    n = lib().or_render_rows(osc.assets, osc.instances, osc.n_inst, C.byref(camera(cam)), C.byref(o),
                             _ptr(k), _ptr(ka), _ptr(r), r.size, _ptr(image), _ptr(T), _ptr(amb))
    if n < 0:
        raise MemoryError("oracle row render: allocation failed")
    return dict(image=image, T=T, ambiguous=amb.astype(bool), n_splats=int(n))


def pixel_weights(splats, cam, o, x, y, cap=4096):
    """Contributions alpha_k T_k of the blended fragments at pixel (x, y) and the final T."""
    splats = np.ascontiguousarray(splats, SPLAT_DTYPE)
    w = np.zeros(cap, np.float64)
    T = C.c_double(0.0)
    n = lib().or_pixel_weights(_ptr(splats), splats.shape[0], C.byref(camera(cam)), C.byref(o),
                               int(x), int(y), _ptr(w), cap, C.byref(T))
    return w[:min(n, cap)], T.value


def cull_decision(vis: dict, inside: np.ndarray, threshold=0.0, band=0.0):
    """Keep mask after the MLP (Sec. 3.3): in the frustum and (bypassed or logit > threshold).
    Also returns where |logit - threshold| <= band (ambiguous decision)."""
    keep = inside & (vis["gated"] | (vis["logits"] > threshold))
    amb = (~vis["gated"]) & (np.abs(vis["logits"] - threshold) <= band)
    return keep, amb


def labels(osc: OracleScene, cams, o=None):
    """Sec. 3.1: per view, per instanced Gaussian, whether it is blended at some pixel."""
    o = o or opts()
    out = []
    for cam in cams:
        r = render(osc, cam, o, want_contrib=True)
        out.append(r["n_contrib"] > 0)
    return np.stack(out, 0)


def tile_lists(splats: np.ndarray, cam, tile_size: int, mode: str = "rect", alpha_min=1.0 / 255.0):
    """Per tile (row-major tile index): the valid splats binned to it, in blend order (depth,
    instance, gaussian).  Returns (tile ids, instance ids, gaussian ids) sorted by tile, then
    blend order.

    mode "rect":    every tile of the splat's tile rectangle (the box of its support, R3);
    mode "support": only tiles holding a pixel centre where the splat reaches alpha_min, i.e.
                    q(d) = d^T conic d <= 2 ln(opacity / alpha_min) (Sec. 4.1's 1/255 rule),
                    checked pixel by pixel over the splat's pixel box."""
    tw = (int(cam.width) + tile_size - 1) // tile_size
    v = splats[splats["valid"] != 0]
    tiles, inst, gs, depth = [], [], [], []
    for s in v:
        if mode == "rect":
            cover = [(tx, ty) for ty in range(s["tile_min"][1], s["tile_max"][1] + 1)
                     for tx in range(s["tile_min"][0], s["tile_max"][0] + 1)]
        elif mode == "support":
            xs = np.arange(s["px_min"][0], s["px_max"][0] + 1)
            ys = np.arange(s["px_min"][1], s["px_max"][1] + 1)
            if xs.size == 0 or ys.size == 0:
                continue
            dx = (xs + 0.5 - s["u"])[None, :]
            dy = (ys + 0.5 - s["v"])[:, None]
            a, b, c = s["conic"]
            q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy
            kk = 2.0 * math.log(s["opacity"] / alpha_min)
            yy, xx = np.nonzero(q <= kk)
            cover = sorted(set(zip((xs[xx] // tile_size).tolist(), (ys[yy] // tile_size).tolist())))
        else:
            raise ValueError(mode)
        for tx, ty in cover:
            tiles.append(ty * tw + tx)
            inst.append(s["instance"])
            gs.append(s["gaussian"])
            depth.append(s["depth"])
    tiles, inst, gs, depth = map(np.asarray, (tiles, inst, gs, depth))
    if tiles.size == 0:
        return tiles, inst, gs
    order = np.lexsort((gs, inst, depth, tiles))
    return tiles[order], inst[order], gs[order]


def box_min_quadratic(a, b, c, x0, x1, y0, y1):
    """min over the box [x0, x1] x [y0, y1] (offsets from the splat mean) of the positive-definite
    form q(x, y) = a x^2 + 2 b x y + c y^2, element-wise over arrays.  Zero if the box holds the
    origin; otherwise the minimum lies on an edge, where q is a parabola in the free coordinate
    with its vertex at -b x / c (vertical edges) or -b y / a (horizontal edges), clamped."""
    a, b, c, x0, x1, y0, y1 = np.broadcast_arrays(*(np.asarray(v, np.float64) for v in (a, b, c, x0, x1, y0, y1)))

    def q(x, y):
        return a * x * x + 2.0 * b * x * y + c * y * y

    best = np.full(a.shape, np.inf)
    for xe in (x0, x1):                       # vertical edges x = xe
        y = np.clip(-b * xe / c, y0, y1)
        best = np.minimum(best, q(xe, y))
    for ye in (y0, y1):                       # horizontal edges y = ye
        x = np.clip(-b * ye / a, x0, x1)
        best = np.minimum(best, q(x, ye))
    inside = (x0 <= 0.0) & (0.0 <= x1) & (y0 <= 0.0) & (0.0 <= y1)
    return np.where(inside, 0.0, best)


def tile_lists_ellipse(splats: np.ndarray, cam, tile_size: int, alpha_min=1.0 / 255.0,
                       band_rel=1e-4, band_abs=1e-3, pad_abs=1e-3, pad_rel=1e-5):
    """Tile lists of the pruned binning (R3: exact support, with tiles pruned to the support
    ellipse), in FP64.  A splat of a tile rectangle with more than one tile is listed in tile T
    iff its support ellipse {d : d^T conic d <= kk}, kk = 2 ln(opacity / alpha_min), meets the box
    spanned by T's pixel centres [tx ts + 1/2, tx ts + ts - 1/2] x [ty ts + 1/2, ty ts + ts - 1/2]
    (tiles past the image edge keep their full box); a one-tile rectangle is listed as is.

    A conservative binner in lower precision widens the ellipse: its level by ``band_rel``
    relative plus ``band_abs``, and its horizontal extent by ``pad_abs`` plus ``pad_rel`` of the
    extent.  Pairs whose minimum of q over the tile box lies above kk but within that widening
    (plus an FP32 coordinate allowance) may be listed or not: they are returned as ambiguous.

    Returns (tiles, instances, gaussians, ambiguous): every listed or ambiguous pair, sorted by
    tile, then blend order (depth, instance, gaussian); ``ambiguous`` marks the band pairs."""
    tw = (int(cam.width) + tile_size - 1) // tile_size
    v = splats[splats["valid"] != 0]
    ts = float(tile_size)
    out_t, out_i, out_g, out_d, out_a = [], [], [], [], []
    for s in v:
        tx0, ty0 = int(s["tile_min"][0]), int(s["tile_min"][1])
        tx1, ty1 = int(s["tile_max"][0]), int(s["tile_max"][1])
        if tx0 > tx1 or ty0 > ty1:
            continue
        txs, tys = np.meshgrid(np.arange(tx0, tx1 + 1), np.arange(ty0, ty1 + 1))
        txs, tys = txs.ravel(), tys.ravel()
        if txs.size == 1:
            inn, amb = np.ones(1, bool), np.zeros(1, bool)
        else:
            a, b, c = (float(x) for x in s["conic"])
            kk = 2.0 * math.log(float(s["opacity"]) / alpha_min)
            m = box_min_quadratic(a, b, c, txs * ts + 0.5 - s["u"], txs * ts + ts - 0.5 - s["u"],
                                  tys * ts + 0.5 - s["v"], tys * ts + ts - 0.5 - s["v"])
            k_inf = kk * (1.0 + band_rel) + band_abs
            # horizontal pad (extent <= sqrt(ca k_inf), ca = Sigma_2D[0,0] = c / det(conic)) and an
            # FP32 coordinate allowance, converted to q: |grad q| <= 2 sqrt(max(a, c) q) per unit
            det_c = a * c - b * b
            ext = math.sqrt(max(c / det_c, 0.0) * k_inf)
            p = pad_abs + 2.0 * pad_rel * ext + 1e-6 * (cam.width + cam.height) + 1e-4
            amax = max(a, c)
            k_hi = k_inf * (1.0 + 1e-5) + 2.0 * math.sqrt(amax * k_inf) * p + 2.0 * amax * p * p
            inn = m <= kk
            amb = (m > kk) & (m <= k_hi)
        sel = inn | amb
        n = int(sel.sum())
        out_t.append(tys[sel] * tw + txs[sel])
        out_i.append(np.full(n, s["instance"]))
        out_g.append(np.full(n, s["gaussian"]))
        out_d.append(np.full(n, s["depth"]))
        out_a.append(amb[sel])
    if not out_t:
        e = np.zeros(0, np.int64)
        return e, e, e, np.zeros(0, bool)
    tiles, inst, gs, depth, amb = (np.concatenate(x) for x in (out_t, out_i, out_g, out_d, out_a))
    order = np.lexsort((gs, inst, depth, tiles))
    return tiles[order], inst[order], gs[order], amb[order]


def training_views_table(cams, train_fov_x=None):
    """Per training camera: its centre (asset frame) and normalised focal 2 fx / W."""
    out = np.zeros((len(cams), 4), np.float64)
    for k, c in enumerate(cams):
        R = np.asarray(c.R, np.float64).reshape(3, 3)
        out[k, :3] = -R.T @ np.asarray(c.t, np.float64)
        out[k, 3] = 2.0 * float(c.fx) / int(c.width)
    return out


def train_loss_grad(osc: OracleScene, asset_k: int, views, labels, sv, sg, weights):
    """Sec. 3.2 / 4.1: class-balanced BCE of a batch and its gradient (flat weight layout)."""
    w = flat_weights(weights) if isinstance(weights, dict) else np.ascontiguousarray(weights, np.float64)
    g = np.zeros(10497, np.float64)
    vt = np.ascontiguousarray(views, np.float64)
    lab = np.ascontiguousarray(labels, np.uint8)
    sv = np.ascontiguousarray(sv, np.int32)
    sg = np.ascontiguousarray(sg, np.int32)
    n_gauss = lab.size // vt.shape[0]
    loss = lib().or_train_loss_grad(C.byref(osc.assets[asset_k]), _ptr(vt), _ptr(lab), n_gauss,
                                    _ptr(sv), _ptr(sg), sv.size, _ptr(w), _ptr(g))
    return loss, g


def train_step(osc: OracleScene, asset_k: int, views, labels, sv, sg, w, m, v, lr, beta1, beta2, eps,
               step):
    """One Adam step in FP64; w, m, v (float64 arrays) are updated in place; returns the loss."""
    vt = np.ascontiguousarray(views, np.float64)
    lab = np.ascontiguousarray(labels, np.uint8)
    sv = np.ascontiguousarray(sv, np.int32)
    sg = np.ascontiguousarray(sg, np.int32)
    n_gauss = lab.size // vt.shape[0]
    for x in (w, m, v):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"] and x.size == 10497
    return lib().or_train_step(C.byref(osc.assets[asset_k]), _ptr(vt), _ptr(lab), n_gauss, _ptr(sv),
                               _ptr(sg), sv.size, _ptr(w), _ptr(m), _ptr(v), lr, beta1, beta2, eps,
                               int(step))


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def psnr(a: np.ndarray, b: np.ndarray, peak: float = 1.0) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0.0 else 10.0 * math.log10(peak * peak / mse)
