"""Differentiable rendering of one asset's parameters through the library (marshalling only).

``render_asset(renderer, asset_id, params, cam, flags)`` uploads ``params`` (device tensors in the
layout of ``nvgs_asset_desc``) with ``nvgs_update_asset``, renders with ``nvgs_render`` (outputs
kept), and on ``backward`` calls ``nvgs_render_backward`` for dL/d(image).  Each forward must be
followed by its backward before the next render on the same renderer: the library differentiates
its most recent frame.
"""
from __future__ import annotations

import torch

from . import nvgs as N

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


class _RenderAsset(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, asset_id, cam, flags, means, log_scales, quats, opacity_logits, sh):
        ps = [t.detach().contiguous() for t in (means, log_scales, quats, opacity_logits, sh)]
        for t in ps:
            if t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError("asset parameters must be float32 CUDA tensors")
        N.nvgs_update_asset(renderer.ctx, asset_id, *ps)
        flags.keep_outputs = 1
        flags.image_memory = N.NVGS_MEM_DEVICE
        image, _ = renderer.render(cam, flags)
        ctx.renderer, ctx.asset_id = renderer, asset_id
        ctx.shapes = [t.shape for t in ps]
        return image

    @staticmethod
    def backward(ctx, g_image):
        r = ctx.renderer
        grads = [torch.zeros(s, dtype=torch.float32, device=r.device) for s in ctx.shapes]
        N.nvgs_render_backward(r.ctx, g_image.contiguous(), ctx.asset_id, *grads)
        return (None, None, None, None, *grads)


def render_asset(renderer, asset_id: int, params: dict, cam, flags: N.RenderFlags | None = None):
    """Image (H x W x 3, CUDA) of the renderer's scene with asset ``asset_id`` set to ``params``
    (dict of the five tensors named in ``PARAM_NAMES``), differentiable in those tensors."""
    flags = flags or renderer.flags()
    return _RenderAsset.apply(renderer, int(asset_id), cam, flags, *(params[k] for k in PARAM_NAMES))
