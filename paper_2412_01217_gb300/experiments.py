"""Learned-initializer experiment: does the MLP reach the plain mapper's final PSNR in fewer
GPU-seconds on the same GB300?

1. Training pairs: the plain mapper (heuristic initializer) maps seeded synthetic rooms;
   each inserted Gaussian gives one pair (7x7x41 patch at its insertion pixel, the
   log-scale / opacity logit / semantic feature it holds at the end of the run).
2. The MLP is trained on those pairs by the tcgen05 kernels (learned_init.MLPInit).
3. On a held-out room both mappers run the same schedule; PSNR on held-out views is
   sampled every `eval_every` iterations.  GPU-seconds are CUDA-event times of the
   iterations plus the insertion work (for the learned form: patch extraction and MLP
   inference included), evaluation excluded.

Run: python -m paper_2412_01217_gb300.experiments [--quick] [--out FILE]
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import multiprocessing as mp
import time

import numpy as np
import torch

from ._lib import call
from .learned_init import MLPInit
from .mapping import Mapper
from .splat import camera_struct


def _raycast(args):
    import synthetic
    room_seed, cams = args
    room = synthetic.Room(n_classes=32, seed=room_seed)
    return [room.raycast(c) for c in cams]


def room_views(room_seed, intr, n_kf, n_eval, pool=None):
    """Keyframe and held-out cameras on the room's trajectory, with ray-cast frames."""
    import synthetic
    room = synthetic.Room(n_classes=32, seed=room_seed)
    if n_eval:
        # keyframes on even trajectory samples, held-out views between them
        cams = room.trajectory(2 * max(n_kf, n_eval), intr, seed=room_seed + 1)
        kf, ev = cams[0::2][:n_kf], cams[1::2][:n_eval]
    else:
        kf, ev = room.trajectory(n_kf, intr, seed=room_seed + 1), []
    jobs = [(room_seed, [c]) for c in kf + ev]
    res = pool.map(_raycast, jobs) if pool else [_raycast(j) for j in jobs]
    frames = [r[0] for r in res]
    return kf, frames[:n_kf], ev, frames[n_kf:]


def run_mapper(kf, frames, n_max, iters_per_kf, new_per_kf, init="heuristic", mlp=None, ev=None, ev_frames=None,
               eval_every=0, seed=0, decoder=None, mapper_factory=None, kappa=1.0):
    """Insert from every keyframe in turn and optimise; returns the mapper, insertion
    records and the PSNR curve [(gpu_seconds, iteration, psnr)].  mapper_factory(frames, kf,
    n_max, decoder=, seed=) builds the Mapper (default: Mapper with its defaults); kappa scales
    the label one-hot the heuristic initializer writes into new semantic features."""
    m = (mapper_factory or Mapper)(frames, kf, n_max, decoder=decoder, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    inserted = []
    curve = []
    gpu_s = 0.0
    it = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(len(kf)):
        e0.record()
        mlp_before = m.mlp_seconds
        start = m.N
        B, pix = m.insert(k, new_per_kf, init=init, mlp=mlp, kappa=kappa)
        e1.record()
        e1.synchronize()
        # the learned form's patch + MLP time is inside this interval already
        gpu_s += e0.elapsed_time(e1) / 1e3
        inserted.append((k, start, B, pix))
        for _ in range(iters_per_kf):
            kk = int(rng.integers(0, k + 1))
            e0.record()
            m.iterate(kk)
            e1.record()
            e1.synchronize()
            gpu_s += e0.elapsed_time(e1) / 1e3
            it += 1
            if eval_every and it % eval_every == 0:
                curve.append((gpu_s, it, m.psnr(ev, ev_frames)))
    return m, inserted, curve


def training_pairs(m, inserted, frames_dev_fn):
    """Patches (X, Xt) and converged targets T for every Gaussian the mapper inserted."""
    Xs, Ts = [], []
    for k, start, B, pix in inserted:
        if B == 0:
            continue
        Bp = ((B + 127) // 128) * 128
        rgb, depth, label = frames_dev_fn(k)
        cam = camera_struct(m.cams[k])
        pix_d = torch.as_tensor(pix).to(m.dev).contiguous()
        X = torch.empty(Bp, 2048, dtype=torch.bfloat16, device=m.dev)
        call("sg_extract_patches", C.c_void_p(rgb.data_ptr()), C.c_void_p(depth.data_ptr()),
             C.c_void_p(label.data_ptr()), C.byref(cam), C.c_void_p(pix_d.data_ptr()), B, Bp,
             C.c_void_p(X.data_ptr()), None, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        Xs.append(X[:B].clone())
        Ts.append(m.converged(start, B))
    return torch.cat(Xs), torch.cat(Ts)


def run(quick=False, train_rooms=3, iters_per_kf=150, keyframes=8, epochs=16, workers=16, max_pairs=None, log=None):
    """The whole experiment; returns the result dict (see module docstring)."""
    import synthetic
    pool = None
    if workers > 1:
        ctx = mp.get_context("spawn")
        pool = ctx.Pool(min(workers, mp.cpu_count()))
    if quick:
        intr = dict(W=320, H=180, fx=160.0, fy=160.0, cx=159.5, cy=89.5)
        n_max, new_per_kf = 40_000, 5_000
    else:
        intr = dict(synthetic.REPLICA_LIKE)
        n_max, new_per_kf = 300_000, 37_500
    n_kf = keyframes
    t0 = time.time()
    # ---- 1. training pairs ----
    Xs, Ts = [], []
    g = torch.Generator().manual_seed(5)
    decoder = torch.randn(32, 16, generator=g) * 0.3
    for r in range(train_rooms):
        kf, frames, _, _ = room_views(100 + r, intr, n_kf, 0, pool)
        m, ins, _ = run_mapper(kf, frames, n_max, iters_per_kf, new_per_kf, seed=100 + r, decoder=decoder)
        X, T = training_pairs(m, ins, m.frame_dev)
        Xs.append(X)
        Ts.append(T)
        del m
        torch.cuda.empty_cache()
        if log:
            log(f"room {100 + r}: {X.shape[0]} pairs")
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    n = min(X.shape[0], max_pairs or X.shape[0])
    n = (n // 4096) * 4096
    X, T = X[:n].contiguous(), T[:n].contiguous()
    t_data = time.time() - t0
    # ---- 2. training ----
    mlp = MLPInit(seed=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = mlp.fit(X, T, epochs=epochs)
    e1.record()
    e1.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    # ---- 3. time-to-PSNR on the held-out room ----
    kf, frames, ev, ev_frames = room_views(999, intr, n_kf, 4, pool)
    if pool is not None:
        pool.close()
    eval_every = max(10, iters_per_kf // 3)
    _, _, plain = run_mapper(kf, frames, n_max, iters_per_kf, new_per_kf, init="heuristic", ev=ev,
                             ev_frames=ev_frames, eval_every=eval_every, seed=999, decoder=decoder)
    _, _, learned = run_mapper(kf, frames, n_max, iters_per_kf, new_per_kf, init="learned", mlp=mlp, ev=ev,
                               ev_frames=ev_frames, eval_every=eval_every, seed=999, decoder=decoder)
    p_star = plain[-1][2]
    reach = next((c for c in learned if c[2] >= p_star), None)
    return {
        "experiment": "learned vs heuristic initializer, time-to-PSNR",
        "images": f"{intr['W']}x{intr['H']} x 3 levels", "gaussians": n_max, "keyframes": n_kf,
        "iters_per_keyframe": iters_per_kf, "train_pairs": int(n), "train_epochs": epochs,
        "train_loss_per_epoch": hist, "train_gpu_seconds": train_s, "data_wall_seconds": t_data,
        "plain_final_psnr": p_star, "plain_gpu_seconds": plain[-1][0],
        "learned_final_psnr": learned[-1][2], "learned_gpu_seconds_total": learned[-1][0],
        "learned_gpu_seconds_to_plain_final_psnr": reach[0] if reach else None,
        "speedup_to_plain_final_psnr": (plain[-1][0] / reach[0]) if reach else None,
        "plain_curve": plain, "learned_curve": learned,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="small images and Gaussian counts")
    ap.add_argument("--out", default=None)
    ap.add_argument("--train-rooms", type=int, default=3)
    ap.add_argument("--iters-per-kf", type=int, default=150)
    ap.add_argument("--keyframes", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=16)
    ap.add_argument("--max-pairs", type=int, default=None, help="train on at most this many pairs")
    args = ap.parse_args()
    out = run(quick=args.quick, train_rooms=args.train_rooms, iters_per_kf=args.iters_per_kf,
              keyframes=args.keyframes, epochs=args.epochs, max_pairs=args.max_pairs)
    s = json.dumps(out)
    print(s)
    if args.out:
        with open(args.out, "w") as f:
            f.write(s + "\n")


if __name__ == "__main__":
    main()
