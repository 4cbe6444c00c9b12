"""Python side of the pyramid splatting library: buffers, the autograd Function and the
CUDA-graph-captured mapping step.  Every computation runs in the sm_103a kernels behind
the C ABI (include/sg.h); this module only allocates device memory with PyTorch, fills the
C structs and passes the current stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (SgCamera, SgConfig, SgGaussians, SgImages, SgLossConfig, SgProjected, SgSaved,
                   SgTargets, SgTileLists, SgView, call)

PARAM_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "rgb", "sem")


SH_KEYS = ("sh", "sem_sh")


def sh_degree(g):
    """Degree D of the spherical-harmonic features of a parameter dict: g["sh"] is
    N x ((D+1)^2 - 1) x 3 (colour), g["sem_sh"] N x ((D+1)^2 - 1) x C (semantic feature);
    one D for both, 0 without them."""
    Ks = {g[k].shape[1] for k in SH_KEYS if g.get(k) is not None and g[k].shape[1]}
    if not Ks:
        return 0
    if len(Ks) > 1:
        raise ValueError("sh and sem_sh must have the same degree")
    K = Ks.pop()
    D = {3: 1, 8: 2, 15: 3}.get(K)
    if D is None:
        raise ValueError(f"{K} SH coefficients per channel; expected 3, 8 or 15")
    return D


def param_keys(g):
    """PARAM_KEYS, plus "sh" / "sem_sh" when the parameters carry them."""
    return PARAM_KEYS + tuple(k for k in SH_KEYS if g.get(k) is not None and g[k].shape[1])


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("pyramid splatting needs a CUDA device (GB300, sm_103a); no CPU path exists")


@dataclass
class RenderConfig:
    """Rendering constants (Sec. III-C conventions) and the launch shape."""
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    T_min: float = 1e-4
    z_near: float = 0.2
    dilation: float = 0.3
    fov_clamp: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    tile_w: int = 16
    tile_h: int = 16
    batch: int = 256
    persistent: bool = True
    pixels_per_thread: int = 1
    pixels_per_thread_bwd: int = 2
    batch_bwd: int = 0  # 0: same as batch
    isotropic: bool = False  # Eq. 2 projection (radius f r / d) instead of EWA
    check_numeric: bool = False  # flag non-finite Gaussian parameters in the status word
    # per-instance half masks in the tile lists: the adjoint of 8x8 tiles at one pixel per
    # thread then runs one warp per half tile (faster on long lists, lists slower to build)
    half_masks: bool = False
    # with half masks: the forward also one warp per half tile (faster on long lists)
    half_tile_fwd: bool = False

    def to_c(self):
        c = SgConfig()
        c.alpha_max, c.alpha_min, c.T_min = self.alpha_max, self.alpha_min, self.T_min
        c.z_near, c.dilation, c.fov_clamp = self.z_near, self.dilation, self.fov_clamp
        for i in range(3):
            c.bg[i] = self.bg[i]
        c.tile_w, c.tile_h, c.batch, c.persistent = self.tile_w, self.tile_h, self.batch, int(self.persistent)
        c.pixels_per_thread = int(self.pixels_per_thread)
        c.pixels_per_thread_bwd = int(self.pixels_per_thread_bwd)
        c.batch_bwd = int(self.batch_bwd)
        c.isotropic = int(self.isotropic)
        c.check_numeric = int(self.check_numeric)
        c.half_tile_fwd = int(self.half_tile_fwd)
        return c


@dataclass
class LossConfig:
    """Eq. 10-13 weights.  sem_mode "ce": cross-entropy of softmax(decoder @ S) against labels;
    "paper": (1 - lambda_s) L1 + lambda_s (1 - SSIM) against a semantic colour image."""
    lambda_r: float = 0.2
    lambda_s: float = 0.2
    w_depth: float = 1.0
    w_sem: float = 1.0
    sem_mode: str = "ce"
    n_classes: int = 0
    check_numeric: bool = False  # flag non-finite loss terms in the status word

    def to_c(self, decoder=None, decoder_grad=None):
        c = SgLossConfig()
        c.lambda_r, c.lambda_s, c.w_depth, c.w_sem = self.lambda_r, self.lambda_s, self.w_depth, self.w_sem
        c.sem_mode = 0 if self.sem_mode == "ce" else 1
        c.n_classes = self.n_classes
        c.decoder = decoder.data_ptr() if decoder is not None else None
        c.decoder_grad = decoder_grad.data_ptr() if decoder_grad is not None else None
        c.check_numeric = int(self.check_numeric)
        return c


def camera_struct(cam):
    c = SgCamera()
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.W, c.H = int(cam["W"]), int(cam["H"])
    R = np.asarray(cam["R_cw"], np.float64).reshape(9)
    t = np.asarray(cam["t_cw"], np.float64).reshape(3)
    for i in range(9):
        c.R_cw[i] = float(R[i])
    for i in range(3):
        c.t_cw[i] = float(t[i])
    return c


def make_views(cams, levels, tile_w=16, tile_h=16):
    """Host view table (sg_make_views): camera-major, level-minor."""
    n = len(cams)
    arr = (SgCamera * n)(*[camera_struct(c) for c in cams])
    out = (SgView * (n * levels))()
    tp = C.c_int64(0)
    tt = C.c_int32(0)
    call("sg_make_views", arr, n, levels, tile_w, tile_h, out, C.byref(tp), C.byref(tt))
    return out, int(tp.value), int(tt.value)


def views_to_device(views, device):
    raw = bytes(C.string_at(C.addressof(views), C.sizeof(views)))
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def gaussians_struct(g, N=None, C_=None):
    s = SgGaussians()
    s.mean, s.log_scale, s.quat = g["mean"].data_ptr(), g["log_scale"].data_ptr(), g["quat"].data_ptr()
    s.opacity_logit, s.rgb, s.sem = g["opacity_logit"].data_ptr(), g["rgb"].data_ptr(), g["sem"].data_ptr()
    s.N = g["mean"].shape[0] if N is None else N
    s.C = g["sem"].shape[1] if C_ is None else C_
    D = sh_degree(g)
    if D:
        s.sh_degree = D
        keys = param_keys(g)
        if "sh" in keys:
            s.sh = g["sh"].data_ptr()
        if "sem_sh" in keys:
            s.sem_sh = g["sem_sh"].data_ptr()
    return s


def to_device_params(g, device="cuda"):
    """dict of arrays -> dict of contiguous float32 CUDA tensors (quat/sem 16-B aligned);
    "sh" (N x K x 3) and "sem_sh" (N x K x C) are carried when present."""
    out = {}
    for k in PARAM_KEYS + tuple(k for k in SH_KEYS if g.get(k) is not None):
        out[k] = torch.as_tensor(np.ascontiguousarray(g[k], dtype=np.float32)).to(device).contiguous()
    return out


class PyramidRasterizer:
    """Buffers and calls for rendering n_cams keyframes x `levels` pyramid levels of N
    Gaussians with C semantic channels in one batched pass.

    Only one forward may be in flight per rasterizer: the tile lists and the saved
    per-pixel state of the last forward are what the backward uses.
    """

    def __init__(self, N, C, cams, levels=1, cfg: RenderConfig | None = None, capacity=None,
                 loss_cfg: LossConfig | None = None, device="cuda", sh_degree=0, sem_sh=False):
        require_cuda()
        _lib.load()
        self.N, self.C, self.levels = int(N), int(C), int(levels)
        self.cfg = cfg or RenderConfig()
        self.loss_cfg = loss_cfg or LossConfig(n_classes=C)
        self.device = torch.device(device)
        self.n_cams = len(cams)
        self.views_host, self.P, self.n_tiles = make_views(cams, levels, self.cfg.tile_w, self.cfg.tile_h)
        self.V = self.n_cams * self.levels
        self.views = views_to_device(self.views_host, self.device)
        self.N_max = self.N
        self.R = self.N * self.V
        dev = self.device
        f32 = dict(dtype=torch.float32, device=dev)
        i32 = dict(dtype=torch.int32, device=dev)
        self.geo = torch.zeros(max(1, self.R) * 8, **f32)
        self.rect = torch.zeros(max(1, self.R) * 2, **i32)
        self.ext = torch.zeros(max(1, self.R) * 2, **f32)
        if capacity is None:
            capacity = max(1 << 16, 16 * self.R)
        self.capacity = int(capacity)
        self.tile = torch.zeros(self.capacity, **i32)
        self.record = torch.zeros(self.capacity, **i32)
        self.ranges = torch.zeros(self.n_tiles * 2, **i32)
        self.order = torch.zeros(self.n_tiles, **i32)
        self.count = torch.zeros(1, **i32)
        self.status = torch.zeros(1, **i32)
        self.work_counter = torch.zeros(2, **i32)
        lib = _lib.load()
        self.tile_ws = torch.zeros(lib.sg_tile_lists_workspace_size(self.R, self.capacity), dtype=torch.uint8, device=dev)
        P = self.P
        self.img_rgb = torch.zeros(3 * P, **f32)
        self.img_depth = torch.zeros(P, **f32)
        self.img_sem = torch.zeros(self.C * P, **f32)
        self.T_final = torch.zeros(P, **f32)
        self.last = torch.zeros(P, **i32)
        self.n_contrib = torch.zeros(P, **i32)
        self.dL_rgb = torch.zeros(3 * P, **f32)
        self.dL_depth = torch.zeros(P, **f32)
        self.dL_sem = torch.zeros(self.C * P, **f32)
        self.terms = torch.zeros(4 * self.V, **f32)
        self.loss_ws = torch.zeros(lib.sg_loss_workspace_size(self.views_host, self.V, self.C,
                                                              max(self.C, self.loss_cfg.n_classes)),
                                   dtype=torch.uint8, device=dev)
        self.bwd_ws = torch.zeros(lib.sg_backward_workspace_size(max(1, self.R), 0), dtype=torch.uint8, device=dev)
        self._ccfg = self.cfg.to_c()
        # per-record view-dependent colour / semantic feature (spherical-harmonic features only)
        self.rec_rgb = self.rec_sem = None
        self._proj = SgProjected(self.geo.data_ptr(), self.rect.data_ptr(), self.ext.data_ptr(), 0, 0)
        if sh_degree:
            self._alloc_record_colour()
        if sem_sh:
            self._alloc_record_semantics()
        self._lists = SgTileLists(self.capacity, self.tile.data_ptr(), self.record.data_ptr(),
                                  self.ranges.data_ptr(), self.count.data_ptr(), self.order.data_ptr(), 0)
        self._saved = SgSaved(self.T_final.data_ptr(), self.last.data_ptr(), self.n_contrib.data_ptr())

    def _alloc_record_colour(self):
        self.rec_rgb = torch.zeros(max(1, self.N_max * self.V) * 3, dtype=torch.float32, device=self.device)
        self._proj.rgb = self.rec_rgb.data_ptr()

    def _alloc_record_semantics(self):
        R = max(1, self.N_max * self.V)
        self.rec_sem = torch.zeros(R * self.C, dtype=torch.float32, device=self.device)
        self._proj.sem = self.rec_sem.data_ptr()
        # the backward workspace gains its block of C semantic gradients per record
        self.bwd_ws = torch.zeros(_lib.load().sg_backward_workspace_size(R, self.C), dtype=torch.uint8,
                                  device=self.device)

    def _check_colour(self, g):
        keys = param_keys(g)
        need = [("sh" in keys and self.rec_rgb is None, self._alloc_record_colour),
                ("sem_sh" in keys and self.rec_sem is None, self._alloc_record_semantics)]
        for missing, alloc in need:
            if missing:
                if torch.cuda.is_current_stream_capturing():
                    raise RuntimeError("spherical-harmonic features: build the rasterizer with sh_degree > 0 "
                                       "(and sem_sh=True) before capturing a graph")
                alloc()

    def set_count(self, N):
        """Use the first N <= capacity Gaussians (buffers keep their maximum size)."""
        if N > self.N_max:
            raise ValueError(f"N = {N} exceeds the rasterizer's capacity {self.N_max}")
        self.N = int(N)
        self.R = self.N * self.V

    # ---- view table ------------------------------------------------------------------
    def set_cameras(self, cams):
        """Replace the keyframe poses/intrinsics (image sizes must stay the same).  The
        device table is updated with an async copy on the current stream, so a captured
        graph replayed afterwards sees the new cameras."""
        views, P, nt = make_views(cams, self.levels, self.cfg.tile_w, self.cfg.tile_h)
        if P != self.P or nt != self.n_tiles:
            raise ValueError("image sizes changed; build a new rasterizer")
        self.views_host = views
        host = torch.frombuffer(bytearray(C.string_at(C.addressof(views), C.sizeof(views))), dtype=torch.uint8)
        self.views.copy_(host.pin_memory(), non_blocking=True)

    def view_slice(self, packed, v, nch):
        """(nch, H, W) view into a packed planar buffer for view-level v."""
        vw = self.views_host[v]
        p0, H, W = vw.pixel_offset, vw.H, vw.W
        return packed[nch * p0: nch * (p0 + H * W)].view(nch, H, W)

    # ---- forward -----------------------------------------------------------------------
    def project(self, g):
        self._check_colour(g)
        gs = gaussians_struct(g)
        call("sg_project_gaussians", C.byref(gs), _ptr(self.views), self.V, C.byref(self._ccfg),
             C.byref(self._proj), _ptr(self.status), _stream())

    def build_lists(self):
        # the compositing kernels read the lists through the same struct, so they follow
        # this choice
        self._lists.half_masks = int(self.cfg.half_masks)
        call("sg_build_tile_lists", C.byref(self._proj), self.N, self.V, _ptr(self.views), self.n_tiles,
             C.byref(self._ccfg), C.byref(self._lists), _ptr(self.tile_ws), self.tile_ws.numel(),
             _ptr(self.status), _stream())

    def rasterize(self, g, out_rgb=None, out_depth=None, out_sem=None):
        gs = gaussians_struct(g)
        imgs = SgImages((out_rgb if out_rgb is not None else self.img_rgb).data_ptr(),
                        (out_depth if out_depth is not None else self.img_depth).data_ptr(),
                        (out_sem if out_sem is not None else self.img_sem).data_ptr())
        call("sg_render_pyramid", C.byref(gs), C.byref(self._proj), C.byref(self._lists), _ptr(self.views),
             self.V, self.n_tiles, C.byref(self._ccfg), C.byref(imgs), C.byref(self._saved),
             _ptr(self.work_counter), _stream())

    def forward(self, g, **out):
        self.project(g)
        self.build_lists()
        self.rasterize(g, **out)

    # ---- loss ----------------------------------------------------------------------------
    def loss(self, gt, rendered=None, decoder=None, decoder_grad=None, loss_cfg=None):
        """Eq. 10-13 for every view-level; gt: dict(rgb, depth, label[, sem]) packed like the
        images.  Fills self.terms (V x 4: L_r, L_d, L_s, total) and self.dL_*."""
        lcfg = loss_cfg or self.loss_cfg
        lc = lcfg.to_c(decoder, decoder_grad)
        need = _lib.load().sg_loss_workspace_size(self.views_host, self.V, self.C, max(self.C, lcfg.n_classes))
        if need > self.loss_ws.numel():
            self.loss_ws = torch.zeros(need, dtype=torch.uint8, device=self.device)
        r = rendered or (self.img_rgb, self.img_depth, self.img_sem)
        ri = SgImages(r[0].data_ptr(), r[1].data_ptr(), r[2].data_ptr())
        ti = SgTargets(gt["rgb"].data_ptr(), gt["depth"].data_ptr(),
                       gt["label"].data_ptr() if gt.get("label") is not None else None,
                       gt["sem"].data_ptr() if gt.get("sem") is not None else None)
        di = SgImages(self.dL_rgb.data_ptr(), self.dL_depth.data_ptr(), self.dL_sem.data_ptr())
        call("sg_pyramid_loss", C.byref(ri), C.byref(ti), _ptr(self.views), self.views_host, self.V, self.C,
             C.byref(lc), _ptr(self.terms), C.byref(di), _ptr(self.loss_ws), self.loss_ws.numel(),
             _ptr(self.status), _stream())

    # ---- backward ------------------------------------------------------------------------
    def backward(self, g, grads, dL=None, between=None):
        """ADDS dL/dparams into grads (dict like g); dL defaults to self.dL_* (from loss).
        The compositing adjoint and the projection adjoint are two library calls;
        `between` (optional) is called on the host between them (e.g. to record an event)."""
        gs = gaussians_struct(g)
        gr = gaussians_struct(grads)
        d = dL or (self.dL_rgb, self.dL_depth, self.dL_sem)
        di = SgImages(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr())
        call("sg_render_pyramid_backward_raster", C.byref(gs), C.byref(self._proj), C.byref(self._lists),
             _ptr(self.views), self.V, self.n_tiles, C.byref(self._ccfg), C.byref(self._saved),
             C.byref(di), C.byref(gr), _ptr(self.bwd_ws), self.bwd_ws.numel(), _ptr(self.work_counter),
             _stream())
        if between is not None:
            between()
        call("sg_project_gaussians_backward", C.byref(gs), C.byref(self._proj), _ptr(self.views), self.V,
             C.byref(self._ccfg), _ptr(self.bwd_ws), self.bwd_ws.numel(), C.byref(gr), _stream())

    # ---- diagnostics --------------------------------------------------------------------
    def instance_count(self):
        return int(self.count.item())

    def check_status(self):
        """Reads the device status word (sg_read_status; synchronises the stream) and raises
        SgError for a capacity overflow, a timeout or a non-finite value (checks on)."""
        bits = C.c_uint32(0)
        lib = _lib.load()
        code = lib.sg_read_status(_ptr(self.status), _stream(), C.byref(bits))
        if code == 2:
            raise _lib.SgError("sg_build_tile_lists", 2,
                               f"{self.instance_count()} tile instances exceed capacity {self.capacity}")
        if code != 0:
            raise _lib.SgError("sg_read_status", code, lib.sg_last_error().decode())
        return int(bits.value)


def build_pyramid(rast: PyramidRasterizer, rgb0, depth0, label0=None, sem0=None):
    """GT pyramid of every keyframe (Eq. 4-6) from level-0 frames, packed like the images.
    rgb0: list of (3,H,W), depth0: list of (H,W), label0: list of (H,W) int or None."""
    dev = rast.device
    P = rast.P
    rgb = torch.zeros(3 * P, dtype=torch.float32, device=dev)
    depth = torch.zeros(P, dtype=torch.float32, device=dev)
    label = torch.full((P,), -1, dtype=torch.int32, device=dev) if label0 is not None else None
    n_sem = sem0[0].shape[0] if sem0 is not None else 0
    sem = torch.zeros(max(1, n_sem) * P, dtype=torch.float32, device=dev) if sem0 is not None else None
    for c in range(rast.n_cams):
        v = c * rast.levels
        rast.view_slice(rgb, v, 3).copy_(torch.as_tensor(np.asarray(rgb0[c], np.float32)))
        rast.view_slice(depth, v, 1).copy_(torch.as_tensor(np.asarray(depth0[c], np.float32))[None])
        if label is not None:
            rast.view_slice(label, v, 1).copy_(torch.as_tensor(np.asarray(label0[c], np.int32))[None])
        if sem is not None:
            rast.view_slice(sem, v, n_sem).copy_(torch.as_tensor(np.asarray(sem0[c], np.float32)))
    if rast.levels > 1:
        call("sg_build_pyramid", _ptr(rgb), _ptr(depth), _ptr(label), _ptr(sem), n_sem, rast.views_host,
             rast.V, _stream())
    return dict(rgb=rgb, depth=depth, label=label, sem=sem)


class PyramidSplat(torch.autograd.Function):
    """Differentiable render of all pyramid levels of all keyframes (Eq. 7-9).

    forward(rast, mean, log_scale, quat, opacity_logit, rgb, sem) -> (rgb, depth, sem)
    packed planar images; backward runs the hand-written adjoint (sg_render_pyramid_backward),
    which uses only the per-pixel T_final / last / n_contrib saved by the forward.
    """

    @staticmethod
    def forward(ctx, rast, mean, log_scale, quat, opacity_logit, rgb, sem, sh=None, sem_sh=None):
        g = dict(mean=mean.contiguous(), log_scale=log_scale.contiguous(), quat=quat.contiguous(),
                 opacity_logit=opacity_logit.contiguous(), rgb=rgb.contiguous(), sem=sem.contiguous())
        if sh is not None:
            g["sh"] = sh.contiguous()
        if sem_sh is not None:
            g["sem_sh"] = sem_sh.contiguous()
        out_rgb = torch.empty(3 * rast.P, dtype=torch.float32, device=rast.device)
        out_depth = torch.empty(rast.P, dtype=torch.float32, device=rast.device)
        out_sem = torch.empty(rast.C * rast.P, dtype=torch.float32, device=rast.device)
        rast.forward(g, out_rgb=out_rgb, out_depth=out_depth, out_sem=out_sem)
        ctx.rast = rast
        ctx.keys = param_keys(g)
        ctx.save_for_backward(*[g[k] for k in ctx.keys])
        return out_rgb, out_depth, out_sem

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_sem):
        rast = ctx.rast
        params = dict(zip(ctx.keys, ctx.saved_tensors))
        grads = {k: torch.zeros_like(v) for k, v in params.items()}
        z = lambda t, n: t.contiguous() if t is not None else torch.zeros(n, dtype=torch.float32, device=rast.device)
        rast.backward(params, grads, dL=(z(d_rgb, 3 * rast.P), z(d_depth, rast.P), z(d_sem, rast.C * rast.P)))
        return (None, *[grads[k] for k in PARAM_KEYS], grads.get("sh"), grads.get("sem_sh"))


def pyramid_splat(rast, g):
    return PyramidSplat.apply(rast, *[g[k] for k in PARAM_KEYS], g.get("sh"), g.get("sem_sh"))


# ------------------------------------------------------------------------------------------
# One mapping iteration (project -> lists -> render -> loss -> adjoint -> Adam), capturable
# ------------------------------------------------------------------------------------------

DEFAULT_LR = dict(mean=1e-4, log_scale=5e-3, quat=1e-3, opacity_logit=5e-2, rgb=2.5e-3, sem=2.5e-3,
                  sh=1.25e-4, sem_sh=1.25e-4)


class MappingStep:
    """Owns Gaussian parameters, their gradients and Adam moments, a rasterizer and the GT
    pyramid; `step()` runs one forward+backward+Adam iteration over every view-level, and
    `capture()` records the same sequence into a CUDA graph replayed by `replay()`."""

    def __init__(self, rast: PyramidRasterizer, params: dict, gt: dict, lr=None, decoder=None,
                 scene_scale=1.0):
        self.rast = rast
        self.p = params
        self.gt = gt
        self.lr = dict(DEFAULT_LR)
        self.lr["mean"] *= scene_scale
        if lr:
            self.lr.update(lr)
        self.grads = {k: torch.zeros_like(v) for k, v in params.items()}
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.decoder = decoder
        self.decoder_grad = torch.zeros_like(decoder) if decoder is not None else None
        self.t = 0
        self.graph = None

    def _adam_groups(self):
        from ._lib import SgAdamGroup
        groups = [SgAdamGroup(self.p[k].data_ptr(), self.grads[k].data_ptr(), self.m[k].data_ptr(),
                              self.v[k].data_ptr(), self.p[k].numel(), self.lr[k]) for k in param_keys(self.p)]
        return (SgAdamGroup * len(groups))(*groups), len(groups)

    def _step_kernels(self, t):
        """One iteration.  Gradients are zero on entry (allocated zeroed; the fused Adam
        zeroes each one after reading it)."""
        r = self.rast
        if self.decoder_grad is not None:
            self.decoder_grad.zero_()
        r.forward(self.p)
        r.loss(self.gt, decoder=self.decoder, decoder_grad=self.decoder_grad)
        r.backward(self.p, self.grads)
        groups, n = self._adam_groups()
        check = r.cfg.check_numeric or r.loss_cfg.check_numeric
        call("sg_adam_multi", groups, n, 0.9, 0.999, 1e-15, t, 1, _ptr(r.status) if check else None, _stream())

    def step(self):
        self.t += 1
        self._step_kernels(self.t)

    def capture(self, warmup=1):
        """Record one iteration into a CUDA graph (Adam bias correction frozen at the
        captured step count; replays after that use it)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._step_kernels(max(1, self.t))
        return self.graph

    def replay(self):
        self.graph.replay()
        self.t += 1

    def total_loss(self):
        return float(self.rast.terms.view(-1, 4)[:, 3].sum().item())
