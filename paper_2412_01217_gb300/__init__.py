"""GB300 (sm_103a) multi-level-pyramid Gaussian splatting: the differentiable rendering
hot path of RGBDS-SLAM's mapping step (Sec. III-B..D) behind the C ABI of include/sg.h.

The CUDA library (libsg.so, built in-tree from csrc/) is mandatory: there is no CPU or
eager-PyTorch fallback.  PyTorch supplies device memory and streams only.
"""
from ._lib import SgError, load as load_library, lib_path  # noqa: F401
from .splat import (LossConfig, MappingStep, PyramidRasterizer, PyramidSplat, RenderConfig,  # noqa: F401
                    build_pyramid, make_views, pyramid_splat, to_device_params)

__all__ = ["RenderConfig", "LossConfig", "PyramidRasterizer", "PyramidSplat", "pyramid_splat",
           "MappingStep", "build_pyramid", "make_views", "to_device_params", "load_library",
           "lib_path", "SgError"]
