"""``Renderer``: the NVGS render pass on torch-owned device memory (marshalling only)."""
from __future__ import annotations

import numpy as np
import torch

from . import nvgs as N


class _DeviceArray:
    """Zero-copy view of a library-owned device buffer (CUDA array interface)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None,
                                         "stream": None}


class Renderer:
    """One library context on one CUDA device; enqueues on the given torch stream (or the
    current one)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("the NVGS library needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ctx = N.nvgs_create(device, self.stream.cuda_stream)
        self.n_instanced = 0

    def close(self):
        if self.ctx is not None:
            N.nvgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ scene
    def load_asset(self, asset, **kw) -> int:
        return N.nvgs_load_asset(self.ctx, asset, **kw)

    def set_mlp(self, asset_id: int, weights, precision: int = N.NVGS_PREC_FP32):
        N.nvgs_set_mlp(self.ctx, asset_id, weights, precision)

    def set_instances(self, instances):
        N.nvgs_set_instances(self.ctx, instances)
        self.n_instanced = N.nvgs_scene_info(self.ctx)[0]

    def load_scene(self, scene, weights=None, precision: int = N.NVGS_PREC_FP32, **kw):
        ids = [self.load_asset(a, **kw) for a in scene.assets]
        if weights is not None:
            for k, i in enumerate(ids):
                w = weights[k] if isinstance(weights, (list, tuple)) else weights
                if w is not None:
                    self.set_mlp(i, w, precision)
        self.set_instances(scene.instances)
        return ids

    # ------------------------------------------------------------------ frames
    @staticmethod
    def flags(**kw) -> N.RenderFlags:
        return N.nvgs_default_flags(**kw)

    def render(self, cam, flags: N.RenderFlags | None = None, out: torch.Tensor | None = None):
        flags = flags or self.flags()
        if out is None:
            out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=self.device)
        st = N.nvgs_render(self.ctx, cam, flags, out)
        return out, st.as_dict()

    def render_views(self, cams, instance_sets=None, flags: N.RenderFlags | None = None, out=None,
                     max_pairs: int = 0, use_graph: bool = False, want_stats: bool = True):
        """Views with their own instance subsets (lists of indices into the scene's instances;
        None: all), one launch per stage for the whole batch (optionally replayed as a CUDA
        graph).  Returns (images, batch totals)."""
        flags = flags or self.flags()
        if out is None:
            out = [torch.empty((c.height, c.width, 3), dtype=torch.float32, device=self.device) for c in cams]
        st = N.nvgs_render_views(self.ctx, cams, instance_sets, flags, out, max_pairs, use_graph, want_stats)
        return out, st

    def render_batch(self, cams, flags: N.RenderFlags | None = None, out=None, max_pairs: int = 0,
                     use_graph: bool = False, want_stats: bool = True):
        """Several views in one sync-free call (optionally replayed as a CUDA graph)."""
        flags = flags or self.flags()
        if out is None:
            out = [torch.empty((c.height, c.width, 3), dtype=torch.float32, device=self.device) for c in cams]
        st = N.nvgs_render_batch(self.ctx, cams, flags, out, max_pairs, use_graph, want_stats)
        return out, st

    def render_host(self, cam, flags: N.RenderFlags, out: np.ndarray | torch.Tensor):
        """Render into HOST memory (the device-to-host copy happens inside the call)."""
        flags.image_memory = N.NVGS_MEM_HOST
        st = N.nvgs_render(self.ctx, cam, flags, out)
        return out, st.as_dict()

    def query_visibility(self, cam, flags: N.RenderFlags | None = None):
        flags = flags or self.flags()
        n = self.n_instanced
        logits = torch.empty(n, dtype=torch.float32, device=self.device)
        keep = torch.empty(n, dtype=torch.uint8, device=self.device)
        st = N.nvgs_query_visibility(self.ctx, cam, flags, logits, keep)
        return logits, keep, st.as_dict()

    def last_frame(self):
        """Copies of the last frame's internal buffers (survivors, records, sorted pairs, tile
        ranges) as CUDA tensors."""
        v = N.nvgs_last_frame(self.ctx)
        ns, npairs = int(v.n_survivors), int(v.n_pairs)
        n_tiles = int(v.tiles_x * v.tiles_y)

        def grab(ptr, count, dtype):
            if not count or not ptr:
                return torch.empty(count, dtype=dtype, device=self.device)
            typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.int64: "<i8", torch.int16: "<i2"}[dtype]
            view = _DeviceArray(ptr, count, typestr)
            self.stream.synchronize()
            return torch.as_tensor(view, device=self.device).clone()

        rec = grab(v.records, 16 * ns, torch.float32).view(-1, 16)
        out = dict(
            survivors=grab(v.survivors, 2 * ns, torch.int32).view(-1, 2),
            records=rec,
            tile_rects=rec[:, 12:].contiguous().view(torch.int32),   # stored inside the records
            pair_values=grab(v.pair_values, npairs, torch.int32),
            # 16-bit tile ids come back as int32 (ids below 65536: read as unsigned)
            pair_keys=(grab(v.pair_keys, npairs, torch.int16).to(torch.int32) & 0xffff
                       if v.pair_key_bytes == 2 else grab(v.pair_keys, npairs, torch.int32)),
            tile_ranges=grab(v.tile_ranges, 2 * n_tiles, torch.int32).view(-1, 2),
            tiles_x=int(v.tiles_x), tiles_y=int(v.tiles_y), tile_size=int(v.tile_size),
            depth_bits=int(v.depth_bits))
        return out

    def sort_pairs(self, keys: torch.Tensor, values: torch.Tensor, key_bits: int):
        N.nvgs_sort_pairs(self.ctx, keys, values, keys.numel(), key_bits)
