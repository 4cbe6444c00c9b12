"""ctypes view of the C ABI in include/sg.h (argument marshalling only).

Loading fails loudly when libsg.so is missing or cannot be loaded: there is no CPU or
eager fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

c_f = C.c_float
c_i = C.c_int32
c_p = C.c_void_p


class SgCamera(C.Structure):
    _fields_ = [("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f), ("W", c_i), ("H", c_i),
                ("R_cw", c_f * 9), ("t_cw", c_f * 3)]


class SgView(C.Structure):
    _fields_ = [("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f), ("R", c_f * 9), ("t", c_f * 3),
                ("W", c_i), ("H", c_i), ("tiles_x", c_i), ("tiles_y", c_i), ("tile_offset", c_i),
                ("pixel_offset", c_i), ("level", c_i), ("camera", c_i)]


class SgGaussians(C.Structure):
    _fields_ = [("mean", c_p), ("log_scale", c_p), ("quat", c_p), ("opacity_logit", c_p),
                ("rgb", c_p), ("sem", c_p), ("N", c_i), ("C", c_i), ("sh", c_p), ("sh_degree", c_i),
                ("sem_sh", c_p)]


SgGaussianGrads = SgGaussians  # same layout (non-const pointers)


class SgConfig(C.Structure):
    _fields_ = [("alpha_max", c_f), ("alpha_min", c_f), ("T_min", c_f), ("z_near", c_f),
                ("dilation", c_f), ("fov_clamp", c_f), ("bg", c_f * 3), ("tile_w", c_i),
                ("tile_h", c_i), ("batch", c_i), ("persistent", c_i), ("pixels_per_thread", c_i),
                ("pixels_per_thread_bwd", c_i), ("batch_bwd", c_i), ("isotropic", c_i), ("check_numeric", c_i),
                ("half_tile_fwd", c_i)]


class SgProjected(C.Structure):
    _fields_ = [("geo", c_p), ("rect", c_p), ("ext", c_p), ("rgb", c_p), ("sem", c_p)]


class SgTileLists(C.Structure):
    _fields_ = [("capacity", c_i), ("tile", c_p), ("record", c_p), ("ranges", c_p), ("count", c_p), ("order", c_p),
                ("half_masks", c_i)]


class SgImages(C.Structure):
    _fields_ = [("rgb", c_p), ("depth", c_p), ("sem", c_p)]


class SgSaved(C.Structure):
    _fields_ = [("T_final", c_p), ("last", c_p), ("n_contrib", c_p)]


class SgTargets(C.Structure):
    _fields_ = [("rgb", c_p), ("depth", c_p), ("label", c_p), ("sem", c_p)]


class SgLossConfig(C.Structure):
    _fields_ = [("lambda_r", c_f), ("lambda_s", c_f), ("w_depth", c_f), ("w_sem", c_f),
                ("sem_mode", c_i), ("n_classes", c_i), ("decoder", c_p), ("decoder_grad", c_p),
                ("check_numeric", c_i)]


class SgAdamGroup(C.Structure):
    _fields_ = [("param", c_p), ("grad", c_p), ("m", c_p), ("v", c_p), ("n", C.c_int64), ("lr", c_f)]


class SgMlp(C.Structure):
    _fields_ = [("W1", c_p), ("W2", c_p), ("W3", c_p), ("W2t", c_p), ("W3t", c_p), ("b1", c_p), ("b2", c_p),
                ("b3", c_p)]


class SgMlpActs(C.Structure):
    _fields_ = [(k, c_p) for k in ("H1", "H1t", "H2", "H2t", "Y", "dY", "dYt", "dH2", "dH2t", "dH1t")]


class SgMlpGrads(C.Structure):
    _fields_ = [(k, c_p) for k in ("W1", "W2", "W3", "b1", "b2", "b3")]


STATUS = {0: "SG_OK", 1: "SG_ERR_INVALID_ARG", 2: "SG_ERR_CAPACITY", 3: "SG_ERR_TIMEOUT",
          4: "SG_ERR_NUMERIC", 5: "SG_ERR_CUDA"}
STATUS_CAPACITY = 1
STATUS_NUMERIC = 2
STATUS_TIMEOUT = 4
MAX_VIEWS = 64

# every entry point declared in include/sg.h: name -> (restype, argtypes)
P = C.POINTER
SIGNATURES = {
    "sg_last_error": (C.c_char_p, []),
    "sg_version": (C.c_char_p, []),
    "sg_read_status": (c_i, [c_p, c_p, P(C.c_uint32)]),
    "sg_kernel_launch_count": (C.c_uint64, []),
    "sg_default_config": (None, [P(SgConfig)]),
    "sg_default_loss_config": (None, [P(SgLossConfig)]),
    "sg_make_views": (c_i, [P(SgCamera), c_i, c_i, c_i, c_i, P(SgView), P(C.c_int64), P(c_i)]),
    "sg_project_gaussians": (c_i, [P(SgGaussians), c_p, c_i, P(SgConfig), P(SgProjected), c_p, c_p]),
    "sg_tile_lists_workspace_size": (C.c_size_t, [C.c_int64, c_i]),
    "sg_build_tile_lists": (c_i, [P(SgProjected), c_i, c_i, c_p, c_i, P(SgConfig), P(SgTileLists),
                                  c_p, C.c_size_t, c_p, c_p]),
    "sg_render_pyramid": (c_i, [P(SgGaussians), P(SgProjected), P(SgTileLists), c_p, c_i, c_i,
                                P(SgConfig), P(SgImages), P(SgSaved), c_p, c_p]),
    "sg_loss_workspace_size": (C.c_size_t, [P(SgView), c_i, c_i, c_i]),
    "sg_pyramid_loss": (c_i, [P(SgImages), P(SgTargets), c_p, P(SgView), c_i, c_i,
                              P(SgLossConfig), c_p, P(SgImages), c_p, C.c_size_t, c_p, c_p]),
    "sg_pyramid_loss_noalloc": (c_i, [P(SgImages), P(SgTargets), c_p, P(SgView), c_i, c_i,
                                      P(SgLossConfig), c_p, P(SgImages), c_p, c_p]),
    "sg_backward_workspace_size": (C.c_size_t, [C.c_int64, c_i]),
    "sg_render_pyramid_backward": (c_i, [P(SgGaussians), P(SgProjected), P(SgTileLists), c_p, c_i,
                                         c_i, P(SgConfig), P(SgSaved), P(SgImages),
                                         P(SgGaussianGrads), c_p, C.c_size_t, c_p, c_p]),
    "sg_render_pyramid_backward_raster": (c_i, [P(SgGaussians), P(SgProjected), P(SgTileLists), c_p, c_i,
                                                c_i, P(SgConfig), P(SgSaved), P(SgImages),
                                                P(SgGaussianGrads), c_p, C.c_size_t, c_p, c_p]),
    "sg_project_gaussians_backward": (c_i, [P(SgGaussians), P(SgProjected), c_p, c_i, P(SgConfig), c_p,
                                            C.c_size_t, P(SgGaussianGrads), c_p]),
    "sg_build_pyramid": (c_i, [c_p, c_p, c_p, c_p, c_i, P(SgView), c_i, c_p]),
    "sg_adam_step": (c_i, [c_p, c_p, c_p, c_p, C.c_int64, c_f, c_f, c_f, c_f, c_i, c_p]),
    "sg_adam_multi": (c_i, [P(SgAdamGroup), c_i, c_f, c_f, c_f, c_i, c_i, c_p, c_p]),
    "sg_gemm_bf16": (c_i, [c_p, C.c_int64, c_p, C.c_int64, c_i, c_i, c_i, c_p, C.c_int64, c_i, c_p, c_p]),
    "sg_gemm_bf16_timeout_probe": (c_i, [c_p, C.c_int64, c_p, C.c_int64, c_i, c_i, c_i, c_p, C.c_int64, C.c_uint32,
                                         c_p, c_p]),
    "sg_mlp_pack_weights": (c_i, [c_p] * 8 + [c_p]),
    "sg_mlp_forward": (c_i, [P(SgMlp), c_p, c_i, P(SgMlpActs), c_p, c_p]),
    "sg_mlp_backward": (c_i, [P(SgMlp), c_p, c_p, c_p, c_i, P(SgMlpActs), P(SgMlpGrads), c_p, c_p, c_p]),
    "sg_extract_patches": (c_i, [c_p, c_p, c_p, P(SgCamera), c_p, c_i, c_i, c_p, c_p, c_p]),
    "sg_init_gaussians": (c_i, [c_p, c_p, c_p, P(SgCamera), c_p, c_i, c_p, c_i, c_f, P(SgGaussians), c_p]),
    "sg_apply_mlp_init": (c_i, [c_p, c_i, c_p, c_p, P(SgGaussians), c_p]),
}

_lib = None


class SgError(RuntimeError):
    def __init__(self, name, code, msg):
        super().__init__(f"{name} -> {STATUS.get(code, code)}: {msg}")
        self.code = code


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libsg.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libsg.so not found at {_build.LIB}; run __graft_entry__.build()")
    lib = C.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def call(name, *args):
    """Call an sg_* function and raise SgError on a non-zero status."""
    lib = load()
    code = getattr(lib, name)(*args)
    if code != 0:
        raise SgError(name, code, lib.sg_last_error().decode())
    return code
