"""Small scene builders for the tests (no method arithmetic)."""
import math

import numpy as np

import scenes


def one_asset(means, log_scales=None, quats=None, opacity_logits=None, sh=None, sh_degree=0):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    if log_scales is None:
        log_scales = np.full((n, 3), -2.0)
    if quats is None:
        quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    if opacity_logits is None:
        opacity_logits = np.zeros(n)
    K = (sh_degree + 1) ** 2
    if sh is None:
        sh = np.zeros((n, K, 3))
    f = np.float32
    return scenes.Asset(means, np.asarray(log_scales, f).reshape(n, 3), np.asarray(quats, f).reshape(n, 4),
                        np.asarray(opacity_logits, f).reshape(n), np.asarray(sh, f).reshape(n, K, 3),
                        sh_degree)


def identity_instance(asset_id=0):
    return scenes.Instance(asset_id, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 1.0)


def axis_camera(width=32, height=32, fx=40.0, fy=None, cx=None, cy=None):
    """Camera at the origin looking down +z (world = camera frame)."""
    return scenes.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), float(fx),
                         float(fx if fy is None else fy), width / 2.0 if cx is None else cx,
                         height / 2.0 if cy is None else cy, width, height, 0.2)


def logit(p):
    return math.log(p / (1.0 - p))


def rotation_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], np.float64)
