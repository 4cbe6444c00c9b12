"""Mapping loop of the GaussianMapping thread (Sec. III-A): keyframes arrive, new Gaussians
are inserted from each keyframe, and every iteration renders all pyramid levels of one
keyframe (Eq. 7-9), evaluates the tightly coupled loss (Eq. 10-13) and back-propagates to
the Gaussians (Sec. III-D), followed by Adam.

Each iteration is one CUDA-graph replay (captured again after every insertion, when the
Gaussian count changes); before a replay the keyframe's camera table and ground-truth
pyramid are copied into the buffers the graph reads.  Insertion uses either the heuristic
initializer (sg_init_gaussians) or the learned one (patches -> MLP -> sg_apply_mlp_init).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from ._lib import call
from .splat import (LossConfig, MappingStep, PyramidRasterizer, RenderConfig, build_pyramid,
                    camera_struct, gaussians_struct)


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _s():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Mapper:
    """Gaussian map of capacity n_max with C semantic features, decoded to n_classes.

    frames: list of level-0 ground-truth frames (dict rgb (3,H,W), depth (H,W), label (H,W))
    cams:   their cameras (same image size).
    """

    def __init__(self, frames, cams, n_max, C=16, n_classes=32, levels=3, cfg=None, decoder=None,
                 lr=None, device="cuda", seed=0, loss_cfg=None):
        self.dev = torch.device(device)
        self.frames, self.cams = frames, cams
        self.levels, self.C, self.n_classes = levels, C, n_classes
        self.rast = PyramidRasterizer(n_max, C, [cams[0]], levels, cfg or RenderConfig(),
                                      capacity=24 * n_max,
                                      loss_cfg=loss_cfg or LossConfig(n_classes=n_classes),
                                      device=self.dev)
        self.n_max = n_max
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=self.dev)
        self.P = dict(mean=z(n_max, 3), log_scale=z(n_max, 3), quat=z(n_max, 4), opacity_logit=z(n_max),
                      rgb=z(n_max, 3), sem=z(n_max, C))
        self.P["quat"][:, 0] = 1.0
        self.N = 0
        self.gts = [build_pyramid(self.rast, [f["rgb"]], [f["depth"]], [f["label"]]) for f in frames]
        self.gt = {k: (v.clone() if v is not None else None) for k, v in self.gts[0].items()}
        if decoder is None:
            g = torch.Generator().manual_seed(seed)
            decoder = torch.randn(n_classes, C, generator=g) * 0.3
        self.decoder = decoder.to(self.dev).contiguous()
        self.lr = lr
        self.rng = np.random.default_rng(seed)
        self.step = None
        self.graph = None
        self.iters = 0
        self._frame_dev = {}
        self.mlp_seconds = 0.0

    # ---- device copies of the level-0 frames ---------------------------------------------
    def frame_dev(self, k):
        if k not in self._frame_dev:
            f = self.frames[k]
            self._frame_dev[k] = (torch.as_tensor(f["rgb"]).to(self.dev).contiguous(),
                                  torch.as_tensor(f["depth"]).to(self.dev).contiguous(),
                                  torch.as_tensor(f["label"]).to(self.dev).contiguous())
        return self._frame_dev[k]

    def params(self):
        return {k: v[: self.N] for k, v in self.P.items()}

    # ---- insertion ---------------------------------------------------------------------------
    def choose_pixels(self, k, n_new, cover_thresh=0.5):
        """Pixels of keyframe k with valid depth that the current map leaves uncovered
        (level-0 T_final > cover_thresh); a seeded random subset of at most n_new."""
        f = self.frames[k]
        valid = f["depth"] > 0
        if self.N > 0:
            self.rast.set_cameras([self.cams[k]])
            self.rast.set_count(self.N)
            self.rast.forward(self.params())
            T = self.rast.view_slice(self.rast.T_final, 0, 1)[0].cpu().numpy()
            valid &= T > cover_thresh
        ys, xs = np.nonzero(valid)
        if len(xs) > n_new:
            sel = self.rng.choice(len(xs), n_new, replace=False)
            xs, ys = xs[sel], ys[sel]
        return np.stack([xs, ys], 1).astype(np.int32)

    def insert(self, k, n_new, init="heuristic", mlp=None, kappa=1.0):
        pix = self.choose_pixels(k, n_new)
        B = min(len(pix), self.n_max - self.N)
        if B <= 0:
            return 0, pix[:0]
        pix = pix[:B]
        pix_d = torch.as_tensor(pix).to(self.dev).contiguous()
        rgb, depth, label = self.frame_dev(k)
        cam = camera_struct(self.cams[k])
        out = gaussians_struct({kk: v[self.N:self.N + B] for kk, v in self.P.items()})
        call("sg_init_gaussians", _p(rgb), _p(depth), _p(label), C.byref(cam), _p(pix_d), B, _p(self.decoder),
             self.n_classes, kappa, C.byref(out), _s())
        if init == "learned":
            Bp = ((B + 127) // 128) * 128
            X = torch.empty(Bp, 2048, dtype=torch.bfloat16, device=self.dev)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            call("sg_extract_patches", _p(rgb), _p(depth), _p(label), C.byref(cam), _p(pix_d), B, Bp, _p(X), None,
                 _s())
            Y = mlp.forward(X, Bp)
            call("sg_apply_mlp_init", _p(Y), B, _p(mlp.y_mean), _p(mlp.y_std), C.byref(out), _s())
            t1.record()
            t1.synchronize()
            self.mlp_seconds += t0.elapsed_time(t1) / 1e3
        self.N += B
        self.rast.set_count(self.N)
        self.graph = None
        return B, pix

    # ---- optimisation ---------------------------------------------------------------------
    def _ensure_step(self):
        if self.step is None:
            self.step = MappingStep(self.rast, {k: v for k, v in self.P.items()}, self.gt, lr=self.lr,
                                    decoder=self.decoder)
        self.step.p = self.params()
        self.step.grads = {k: v[: self.N] for k, v in self._full_grads().items()}
        self.step.m = {k: v[: self.N] for k, v in self._full("m").items()}
        self.step.v = {k: v[: self.N] for k, v in self._full("v").items()}

    def _full(self, name):
        if not hasattr(self, "_buf_" + name):
            setattr(self, "_buf_" + name, {k: torch.zeros_like(v) for k, v in self.P.items()})
        return getattr(self, "_buf_" + name)

    def _full_grads(self):
        return self._full("g")

    def _select(self, k):
        self.rast.set_cameras([self.cams[k]])
        for key, v in self.gts[k].items():
            if v is not None:
                self.gt[key].copy_(v, non_blocking=True)

    def iterate(self, k, use_graph=True):
        """One mapping iteration on keyframe k (all pyramid levels)."""
        self._select(k)
        if self.graph is None:
            self._ensure_step()
            self.step.t = self.iters
            self.step.step()  # eager warm-up of this Gaussian count (also sizes workspaces)
            self.iters += 1
            if use_graph:
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self.step._step_kernels(max(1, self.iters))
            return
        if use_graph:
            self.graph.replay()
        else:
            self.step._step_kernels(max(1, self.iters))
        self.iters += 1

    # ---- evaluation ---------------------------------------------------------------------
    def psnr(self, cams, frames):
        """Mean level-0 RGB PSNR over held-out views."""
        vals = []
        for cam, f in zip(cams, frames):
            self.rast.set_cameras([cam])
            self.rast.forward(self.params())
            img = self.rast.view_slice(self.rast.img_rgb, 0, 3)
            gt = torch.as_tensor(f["rgb"]).to(self.dev)
            mse = float(((img.clamp(0, 1) - gt) ** 2).mean().item())
            vals.append(-10.0 * math.log10(max(mse, 1e-12)))
        return float(np.mean(vals))

    def evaluate(self, cams, frames):
        """Level-0 quality on held-out views: RGB PSNR, depth L1 (over valid target depth) and
        semantic mIoU (argmax of the decoded features against the labels, over the classes
        present in prediction or target).  Evaluation only, not part of the optimised path."""
        psnr, l1, inter, union = [], [], None, None
        K = self.decoder.shape[0]
        for cam, f in zip(cams, frames):
            self.rast.set_cameras([cam])
            self.rast.forward(self.params())
            img = self.rast.view_slice(self.rast.img_rgb, 0, 3)
            gt = torch.as_tensor(f["rgb"]).to(self.dev)
            mse = float(((img.clamp(0, 1) - gt) ** 2).mean().item())
            psnr.append(-10.0 * math.log10(max(mse, 1e-12)))
            d = self.rast.view_slice(self.rast.img_depth, 0, 1)[0]
            gd = torch.as_tensor(f["depth"]).to(self.dev)
            m = gd > 0
            l1.append(float((d[m] - gd[m]).abs().mean().item()))
            S = self.rast.view_slice(self.rast.img_sem, 0, self.C).reshape(self.C, -1)
            pred = (self.decoder @ S).argmax(0)
            lab = torch.as_tensor(f["label"]).to(self.dev).reshape(-1).long()
            ok = lab >= 0
            pi = torch.bincount(pred[ok] * K + lab[ok], minlength=K * K).reshape(K, K)
            i_ = pi.diag().double()
            u_ = pi.sum(0).double() + pi.sum(1).double() - i_
            inter = i_ if inter is None else inter + i_
            union = u_ if union is None else union + u_
        present = union > 0
        miou = float((inter[present] / union[present]).mean().item())
        return dict(psnr=float(np.mean(psnr)), depth_l1=float(np.mean(l1)), miou=miou)

    def converged(self, start, count):
        """[count][32] targets of the learned initializer: log-scale (3), opacity logit (1),
        semantic feature (C) of Gaussians start..start+count-1, zero-padded."""
        T = torch.zeros(count, 32, device=self.dev)
        T[:, 0:3] = self.P["log_scale"][start:start + count]
        T[:, 3] = self.P["opacity_logit"][start:start + count]
        T[:, 4:4 + self.C] = self.P["sem"][start:start + count]
        return T
