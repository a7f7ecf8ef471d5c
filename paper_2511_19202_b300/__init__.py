"""NVGS render pass for one NVIDIA B300: a C-ABI CUDA library (``libnvgs.so``, include/nvgs.h)
plus this thin Python binding.

``nvgs``      ctypes binding, one function per C entry point (argument marshalling only)
``render``    ``Renderer``: scene upload and per-frame calls on torch-owned device memory
``build``     in-tree nvcc build of ``libnvgs.so`` for sm_103a

Submodules load on first use so that ``python -m paper_2511_19202_b300.build`` works before the
library exists.  Using ``nvgs`` or ``render`` without a built library raises ImportError.
"""
import importlib

__all__ = ["nvgs", "render", "build", "Renderer"]


def __getattr__(name):
    if name in ("nvgs", "render", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    if name == "Renderer":
        return importlib.import_module(f"{__name__}.render").Renderer
    raise AttributeError(name)
