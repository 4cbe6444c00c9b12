"""Ablation analogues on seeded synthetic rooms (the paper's MLP-GS and TCMF-RO studies,
Fig. 6 and Table IV, on stand-in data):

* pyramid: the mapper trained on all pyramid levels of each keyframe per iteration
  (coarse-to-fine, Eq. 4-6) against the same mapper trained on level 0 only; held-out level-0
  PSNR over GPU-seconds, and the GPU-seconds the pyramid form needs to reach the single-level
  form's final PSNR.
* loss terms: the tightly coupled loss (Eq. 13) against the same run without the depth term,
  without the semantic term, and with RGB only; held-out PSNR, depth L1 and semantic mIoU.
  New Gaussians start with a zero semantic feature here (the heuristic initializer would
  otherwise copy the keyframe's label into it), so the semantics come from the loss alone.

Run: python -m paper_2412_01217_gb300.ablation [--quick] [--out FILE]
"""
from __future__ import annotations

import argparse
import json

import torch

from .experiments import room_views, run_mapper
from .mapping import Mapper
from .splat import LossConfig


def _setup(quick):
    import synthetic
    if quick:
        return dict(W=320, H=180, fx=160.0, fy=160.0, cx=159.5, cy=89.5), 40_000, 5_000
    return dict(synthetic.REPLICA_LIKE), 300_000, 37_500


def _decoder():
    g = torch.Generator().manual_seed(5)
    return torch.randn(32, 16, generator=g) * 0.3


def pyramid_ablation(quick=True, keyframes=6, iters_per_kf=90, room_seed=777):
    intr, n_max, new_per_kf = _setup(quick)
    kf, frames, ev, ev_frames = room_views(room_seed, intr, keyframes, 4)
    decoder = _decoder()
    curves = {}
    for levels in (1, 3):
        def make(frames_, kf_, n_max_, decoder=None, seed=0, levels=levels):
            return Mapper(frames_, kf_, n_max_, decoder=decoder, seed=seed, levels=levels)
        _, _, curve = run_mapper(kf, frames, n_max, iters_per_kf, new_per_kf, ev=ev, ev_frames=ev_frames,
                                 eval_every=max(10, iters_per_kf // 3), seed=room_seed, decoder=decoder,
                                 mapper_factory=make)
        curves[levels] = curve
        torch.cuda.empty_cache()
    p_star = curves[1][-1][2]
    reach = next((c for c in curves[3] if c[2] >= p_star), None)
    return {"experiment": "coarse-to-fine pyramid (3 levels) vs level 0 only",
            "images": f"{intr['W']}x{intr['H']}", "gaussians": n_max, "keyframes": keyframes,
            "iters_per_keyframe": iters_per_kf,
            "single_level_final_psnr": p_star, "single_level_gpu_seconds": curves[1][-1][0],
            "pyramid_final_psnr": curves[3][-1][2], "pyramid_gpu_seconds": curves[3][-1][0],
            "pyramid_gpu_seconds_to_single_level_final_psnr": reach[0] if reach else None,
            "single_level_curve": curves[1], "pyramid_curve": curves[3]}


def loss_ablation(quick=True, keyframes=6, iters_per_kf=90, room_seed=778):
    intr, n_max, new_per_kf = _setup(quick)
    kf, frames, ev, ev_frames = room_views(room_seed, intr, keyframes, 4)
    decoder = _decoder()
    out = {"experiment": "loss-term ablation (Eq. 13)", "images": f"{intr['W']}x{intr['H']} x 3 levels",
           "gaussians": n_max, "keyframes": keyframes, "iters_per_keyframe": iters_per_kf, "runs": {}}
    for name, wd, ws in (("full", 1.0, 1.0), ("no_depth", 0.0, 1.0), ("no_semantic", 1.0, 0.0),
                         ("rgb_only", 0.0, 0.0)):
        lc = LossConfig(n_classes=32, w_depth=wd, w_sem=ws)

        def make(frames_, kf_, n_max_, decoder=None, seed=0, lc=lc):
            return Mapper(frames_, kf_, n_max_, decoder=decoder, seed=seed, loss_cfg=lc)
        m, _, _ = run_mapper(kf, frames, n_max, iters_per_kf, new_per_kf, seed=room_seed, decoder=decoder,
                             mapper_factory=make, kappa=0.0)
        out["runs"][name] = m.evaluate(ev, ev_frames)
        del m
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="320x180 images, 40k Gaussians")
    ap.add_argument("--keyframes", type=int, default=8)
    ap.add_argument("--iters-per-kf", type=int, default=150)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    res = {"pyramid": pyramid_ablation(args.quick, args.keyframes, args.iters_per_kf),
           "loss_terms": loss_ablation(args.quick, args.keyframes, args.iters_per_kf)}
    s = json.dumps(res)
    print(s)
    if args.out:
        with open(args.out, "w") as f:
            f.write(s + "\n")


if __name__ == "__main__":
    main()
