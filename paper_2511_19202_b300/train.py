"""Baking an asset's visibility into its MLP (NVGS Sec. 3.1-3.2, 4.1) through the C ABI.

``train_visibility`` = training views (Fibonacci directions x log-spaced distances) -> GPU labels
(nvgs_label_visibility) -> Adam steps on the class-balanced BCE (nvgs_train_visibility_step) ->
the trained FP32 weights, installed with nvgs_set_mlp in the requested precision.  Every step
runs in the library's kernels; this module only sequences the calls.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import nvgs as N


def init_weights(seed: int) -> np.ndarray:
    """N(0, 1/fan_in) weights, zero biases (flat nvgs_set_mlp layout)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ((32, 64), (64, 64), (64, 64), (64, 1)):
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(fi), fo * fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def train_visibility(ctx, asset_id: int, n_dirs: int = 512, n_dist: int = 3, res: int = 512,
                     steps: int = 1500, batch: int = 65536, lr0: float = 2e-3, lr1: float = 2e-4,
                     warmup: float = 0.2, seed: int = 0, precision: int = N.NVGS_PREC_BF16,
                     tile: int = 16, device: int = 0, log_every: int = 0, n_aux: int = 0,
                     aux_angle_deg: float = 2.5, random_offset: bool = False,
                     train_precision: int = N.NVGS_PREC_BF16):
    """Labels, trains and installs the visibility MLP of one asset.  Returns (weights, info).
    train_precision: NVGS_PREC_BF16 runs each step's forward and backward in BF16 on the tensor
    cores (FP32 master weights and Adam), NVGS_PREC_FP32 on the CUDA cores; ``precision`` is the
    arithmetic the installed MLP is queried in.
    n_aux > 0 adds that many auxiliary cone views per main view (a Gaussian is labelled visible
    if any of them blends it; Sec. 3.1); random_offset shifts the asset off the image centre
    (Sec. 3.1, 4.1)."""
    t0 = time.perf_counter()
    info = N.nvgs_get_asset_info(ctx, asset_id)
    group = 1 + int(n_aux)
    all_views = N.nvgs_training_views_ex(ctx, asset_id, n_dirs, n_dist, res, res, n_aux=n_aux,
                                         aux_angle=math.radians(aux_angle_deg), random_offset=random_offset,
                                         seed=seed)
    views = (N.Camera * (len(all_views) // group))(*[all_views[k] for k in range(0, len(all_views), group)])
    n = int(info.n)
    labels = torch.empty(len(views) * n, dtype=torch.uint8, device=f"cuda:{device}")
    flags = N.nvgs_default_flags(use_mlp=0, tile_size=tile)
    N.nvgs_label_visibility(ctx, asset_id, all_views, flags, labels, group=group)
    torch.cuda.synchronize(device)
    t_label = time.perf_counter() - t0
    visible_frac = float(labels.float().mean())
    N.nvgs_train_init(ctx, asset_id, init_weights(seed + 7919 * asset_id), views)
    losses = []
    for step in range(steps):
        lr = N.nvgs_lr_schedule(step, steps, lr0, lr1, warmup)
        want = bool(log_every) and (step % log_every == 0 or step == steps - 1)
        loss = N.nvgs_train_visibility_step(ctx, asset_id, labels, batch, step, lr, seed=seed,
                                            want_loss=want, precision=train_precision)
        if want:
            losses.append((step, loss))
    w = N.nvgs_train_get_weights(ctx, asset_id)
    N.nvgs_set_mlp(ctx, asset_id, w, precision)
    del labels
    torch.cuda.synchronize(device)
    return w, {"label_s": t_label, "train_s": time.perf_counter() - t0 - t_label,
               "total_s": time.perf_counter() - t0, "views": len(views),
               "visible_fraction": visible_frac, "losses": losses}
