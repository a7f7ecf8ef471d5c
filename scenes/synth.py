"""Seeded synthetic scenes with the shapes and distributions of the paper's workloads.

The paper's assets (RTMV trees, MVHumanNet avatars, a donut; Sec. 4.2) are not available, so
these generators stand in for them.  Every array is float32, the precision the CUDA library
consumes; the oracle widens the same values to float64 exactly.

Conventions (shared by both consumers, stated once here):

* Gaussian parameters per asset: ``means`` (N,3), ``log_scales`` (N,3), ``quats`` (N,4) in
  (w, x, y, z) order and not necessarily normalised, ``opacity_logits`` (N,), ``sh`` (N, K, 3)
  with K = (degree+1)^2, coefficient-major, RGB innermost.
* Instance: world position of a local point mu is ``R @ (s * mu) + t`` (R orthonormal, s > 0).
* Camera: world-to-camera ``x_c = R @ x_w + t``; x right, y down, z forward; pixel
  coordinates ``u = fx * x_c/z_c + cx``, ``v = fy * y_c/z_c + cy``; pixel (i, j) has its centre
  at (i + 0.5, j + 0.5); images are row-major H x W x 3.
* MLP weights: ``W1`` (64,32), ``b1`` (64,), ``W2`` (64,64), ``b2``, ``W3`` (64,64), ``b3``,
  ``W4`` (1,64), ``b4`` (1,), float32, stored as (out, in).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

MLP_LAYERS = ((32, 64), (64, 64), (64, 64), (64, 1))  # (fan_in, fan_out) per layer


@dataclasses.dataclass
class Asset:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    train_fov_x: float = math.radians(50.0)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Asset":
        return Asset(self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity_logits[idx].copy(), self.sh[idx].copy(), self.sh_degree,
                     self.train_fov_x)


@dataclasses.dataclass
class Instance:
    asset_id: int
    R: np.ndarray  # (3,3) float32, orthonormal
    t: np.ndarray  # (3,) float32
    s: float


@dataclasses.dataclass
class Camera:
    R: np.ndarray  # (3,3) float32 world->camera rotation
    t: np.ndarray  # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 0.2

    @property
    def center(self) -> np.ndarray:
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


@dataclasses.dataclass
class Scene:
    assets: List[Asset]
    instances: List[Instance]

    @property
    def n_instanced(self) -> int:
        return sum(self.assets[i.asset_id].n for i in self.instances)


# ----------------------------------------------------------------------------- cameras
def look_at_camera(eye: Sequence[float], target: Sequence[float], width: int, height: int,
                   fov_x_deg: float, up=(0.0, 1.0, 0.0), z_near: float = 0.2) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; horizontal field of view ``fov_x_deg``,
    square pixels, principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:  # looking along the up axis
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], 0)
    t = -R @ eye
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(R.astype(np.float32), t.astype(np.float32), float(np.float32(fx)),
                  float(np.float32(fx)), width / 2.0, height / 2.0, int(width), int(height),
                  z_near)


def fibonacci_directions(n: int) -> np.ndarray:
    """``n`` unit vectors on a golden-angle (Fibonacci) spiral, y_k = 1 - 2(k+0.5)/n."""
    k = np.arange(n, dtype=np.float64)
    y = 1.0 - 2.0 * (k + 0.5) / n
    rad = np.sqrt(np.maximum(0.0, 1.0 - y * y))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rad * np.cos(phi), y, rad * np.sin(phi)], 1)


# ----------------------------------------------------------------------------- surfaces
def _sphere_points(rng, n, radius=1.0):
    p = rng.standard_normal((n, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return p * radius


def _torus_points(rng, n, R=1.0, r=0.4):
    """Area-uniform points on a torus around the y axis (tube angle by rejection)."""
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 64
        u = rng.uniform(0, 2 * math.pi, m)
        v = rng.uniform(0, 2 * math.pi, m)
        keep = rng.uniform(0, R + r, m) < (R + r * np.cos(v))
        u, v = u[keep], v[keep]
        ring = R + r * np.cos(v)
        pts = np.stack([ring * np.cos(u), r * np.sin(v), ring * np.sin(u)], 1)
        out = np.concatenate([out, pts], 0)
    return out[:n]


def _box_points(rng, n, half=0.8):
    """Area-uniform points on the surface of an axis-aligned cube of half-extent ``half``."""
    face = rng.integers(0, 6, n)
    uv = rng.uniform(-half, half, (n, 2))
    p = np.empty((n, 3))
    axis = face // 2
    sign = np.where(face % 2 == 0, 1.0, -1.0)
    for a in range(3):
        sel = axis == a
        others = [b for b in range(3) if b != a]
        p[sel, a] = sign[sel] * half
        p[sel, others[0]] = uv[sel, 0]
        p[sel, others[1]] = uv[sel, 1]
    return p


def _gaussians_on(rng, pts, sh_degree, jitter=0.01, higher_band_std=0.3):
    n = pts.shape[0]
    means = pts + rng.normal(0.0, jitter, (n, 3))
    log_scales = rng.normal(-4.0, 0.5, (n, 3))
    quats = rng.standard_normal((n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    opacity_logits = rng.normal(0.0, 1.5, n)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    # DC coefficient uniform in [-sqrt(pi), sqrt(pi)] so that the DC colour spans [0, 1]
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_band_std, (n, K - 1, 3))
    f = np.float32
    return Asset(means.astype(f), log_scales.astype(f), quats.astype(f),
                 opacity_logits.astype(f), sh.astype(f), sh_degree)


def torus_asset(n=20000, seed=0, sh_degree=0, R=1.0, r=0.4) -> Asset:
    rng = np.random.default_rng(seed)
    return _gaussians_on(rng, _torus_points(rng, n, R, r), sh_degree)


def sphere_asset(n, seed, sh_degree=3, radius=1.0) -> Asset:
    rng = np.random.default_rng(seed)
    return _gaussians_on(rng, _sphere_points(rng, n, radius), sh_degree)


def box_asset(n, seed, sh_degree=3, half=0.8) -> Asset:
    rng = np.random.default_rng(seed)
    return _gaussians_on(rng, _box_points(rng, n, half), sh_degree)


def random_asset(k: int, n: int, sh_degree: int = 3) -> Asset:
    """The k-th asset of the composed scene: sphere, torus or noisy box in turn (seed 1000+k)."""
    seed = 1000 + k
    kind = k % 3
    if kind == 0:
        return sphere_asset(n, seed, sh_degree)
    if kind == 1:
        return torus_asset(n, seed, sh_degree)
    return box_asset(n, seed, sh_degree)


# ----------------------------------------------------------------------------- MLP
def mlp_weights(seed: int = 42) -> dict:
    """Visibility-MLP weights ~ N(0, 1/fan_in), biases zero (32 -> 64 -> 64 -> 64 -> 1)."""
    rng = np.random.default_rng(seed)
    w = {}
    for li, (fi, fo) in enumerate(MLP_LAYERS, start=1):
        w[f"W{li}"] = rng.normal(0.0, 1.0 / math.sqrt(fi), (fo, fi)).astype(np.float32)
        w[f"b{li}"] = np.zeros(fo, np.float32)
    return w


def planar_mlp_weights(seed: int = 7, gain: float = 10.0, noise: float = 0.05,
                       offset: float = 0.0, direction=None) -> dict:
    """Visibility-MLP weights whose logit is close to gain * (u . x) + offset, x the 32 inputs and
    u = ``direction`` (default: a seeded unit vector over the first three inputs, the normalised
    local position): hidden units 0 and 1 carry ReLU(u . x) and ReLU(-u . x) through the three
    layers, the output takes their difference times gain, and every other weight is N(0, 1/fan_in)
    scaled by ``noise``.  Like a trained network, the decisions are coherent in space (or in
    distance) and few logits sit near the threshold."""
    rng = np.random.default_rng(seed)
    w = {}
    for li, (fi, fo) in enumerate(MLP_LAYERS, start=1):
        w[f"W{li}"] = (noise * rng.normal(0.0, 1.0 / math.sqrt(fi), (fo, fi))).astype(np.float32)
        w[f"b{li}"] = np.zeros(fo, np.float32)
    if direction is None:
        n = rng.normal(size=3)
        u = np.zeros(32)
        u[0:3] = n / np.linalg.norm(n)
    else:
        u = np.asarray(direction, np.float64).reshape(32)
    w["W1"][0:2, :] = 0.0
    w["W1"][0, :] = u
    w["W1"][1, :] = -u
    for li in (2, 3):
        w[f"W{li}"][0:2, :] = 0.0
        w[f"W{li}"][0, 0] = 1.0
        w[f"W{li}"][1, 1] = 1.0
    w["W4"][0, 0] = gain
    w["W4"][0, 1] = -gain
    w["b4"][0] = offset
    return w


# ----------------------------------------------------------------------------- configs
def layered_scene(n: int = 20000, spacing: float = 4.0, layers: int = 3) -> Scene:
    """The workload-1 torus as ``layers`` identity-rotation instances spaced ``spacing`` apart
    along -z and shifted sideways, so that each sits in its own range of camera distances (for
    decisions that depend on the distance input); seen by ``layered_camera``."""
    insts = [Instance(0, np.eye(3, dtype=np.float32),
                      np.array([0.9 * ((k % 2) * 2 - 1) * (k > 0), 0.0, -spacing * k], np.float32), 1.0)
             for k in range(layers)]
    return Scene([torus_asset(n, seed=0, sh_degree=0)], insts)


def layered_camera(width: int = 320, height: int = 240) -> Camera:
    return look_at_camera((0.0, 1.5, 3.0), (0.0, 0.0, -4.0), width, height, 60.0)


def _identity_instance(asset_id=0) -> Instance:
    return Instance(asset_id, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 1.0)


def config1_scene(n: int = 20000) -> Scene:
    """Single torus asset (R = 1, r = 0.4) of ``n`` Gaussians, SH degree 0, one identity instance."""
    return Scene([torus_asset(n, seed=0, sh_degree=0)], [_identity_instance()])


def config1_camera(width: int = 256, height: int = 256) -> Camera:
    """256 x 256, 50 degree field of view, distance 3 from the origin, 26.6 degrees above the
    torus plane, looking at the origin."""
    d = np.array([0.0, 0.5, 1.0])
    d = 3.0 * d / np.linalg.norm(d)
    return look_at_camera(d, (0, 0, 0), width, height, 50.0)


def _rotation_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def _random_rotation(rng):
    """Haar-uniform rotation from the QR factorisation of a Gaussian matrix."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def config2_scene(n_assets: int = 16, n_per_asset: int = 500_000, n_instances: int = 64,
                  sh_degree: int = 3, full_rotation: bool = True) -> Scene:
    """Composed scene: ``n_assets`` assets (sphere / torus / box in turn), ``n_instances`` rigid
    instances (random rotation, scale U[0.5, 2]) resting on a 20 x 20 ground plane (seed 7)."""
    assets = [random_asset(k, n_per_asset, sh_degree) for k in range(n_assets)]
    rng = np.random.default_rng(7)
    inst = []
    for i in range(n_instances):
        a = int(rng.integers(0, n_assets))
        R = _random_rotation(rng) if full_rotation else _rotation_y(rng.uniform(0, 2 * math.pi))
        s = rng.uniform(0.5, 2.0)
        xz = rng.uniform(-10.0, 10.0, 2)
        t = np.array([xz[0], s * 1.0, xz[1]])  # unit-size assets rest on y = 0
        inst.append(Instance(a, R.astype(np.float32), t.astype(np.float32), float(np.float32(s))))
    return Scene(assets, inst)


def config2_orbit(n_frames: int = 120, radius: float = 14.0, height: float = 4.0,
                  seed: int = 11) -> np.ndarray:
    """Eye positions of a seeded circular orbit around the origin (random starting phase)."""
    phase = np.random.default_rng(seed).uniform(0, 2 * math.pi)
    a = phase + 2 * math.pi * np.arange(n_frames) / n_frames
    return np.stack([radius * np.cos(a), np.full(n_frames, height), radius * np.sin(a)], 1)


def config2_camera(frame: int = 0, width: int = 1920, height: int = 1080,
                   n_frames: int = 120) -> Camera:
    eye = config2_orbit(n_frames)[frame % n_frames]
    return look_at_camera(eye, (0.0, 0.0, 0.0), width, height, 50.0)


def config5_scene(n_assets: int = 8, n_per_asset: int = 1_000_000, n_instances: int = 200,
                  sh_degree: int = 3) -> Scene:
    """Large composed scene: ``n_assets`` assets of ``n_per_asset`` Gaussians (sphere / torus / box
    in turn), ``n_instances`` rigid instances (random rotation, scale U[0.5, 2]) on a 36 x 36
    ground plane (seed 13): 200M instanced Gaussians by default."""
    assets = [random_asset(k, n_per_asset, sh_degree) for k in range(n_assets)]
    rng = np.random.default_rng(13)
    inst = []
    for i in range(n_instances):
        a = int(rng.integers(0, n_assets))
        R = _random_rotation(rng)
        s = rng.uniform(0.5, 2.0)
        xz = rng.uniform(-18.0, 18.0, 2)
        t = np.array([xz[0], s * 1.0, xz[1]])
        inst.append(Instance(a, R.astype(np.float32), t.astype(np.float32), float(np.float32(s))))
    return Scene(assets, inst)


def config5_camera(frame: int = 0, width: int = 3840, height: int = 2160, n_frames: int = 120) -> Camera:
    eye = config2_orbit(n_frames, radius=26.0, height=6.0, seed=17)[frame % n_frames]
    return look_at_camera(eye, (0.0, 0.0, 0.0), width, height, 50.0)


def tiny_scene(n: int, seed: int, spread: float = 0.6, depth: float = 3.0, sh_degree: int = 0,
               log_scale_mean: float = -2.5, n_instances: int = 1) -> Scene:
    """A handful of Gaussians in front of the default camera (for brute-force checks)."""
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n),
                    rng.uniform(-spread, spread, n)], 1)
    a = _gaussians_on(rng, pts, sh_degree, jitter=0.0)
    a.log_scales = rng.normal(log_scale_mean, 0.4, (n, 3)).astype(np.float32)
    insts = [_identity_instance()]
    for _ in range(1, n_instances):
        R = _random_rotation(rng)
        insts.append(Instance(0, R.astype(np.float32), rng.uniform(-0.3, 0.3, 3).astype(np.float32),
                              float(np.float32(rng.uniform(0.6, 1.2)))))
    return Scene([a], insts)
