"""Launch-shape autotuner of the compositing kernels.

For each screen-tile shape (8x8, 16x8, 16x16, 32x8) one rasterizer is built (the tile
lists depend on the tile shape); then the shared-memory batch depth (16, 32, 64, 128, 256) and
the pixels per thread are varied in place, for the forward (1, 2 pixels per thread) and, with
its own batch depth, for the backward (1, 2, 4).  For 8x8 tiles the lists are also built
with per-instance half masks, which run the adjoint at one pixel per thread one warp per
half tile, and the forward is timed both with shared batches and one warp per half tile.  Every candidate is timed with CUDA events over a few repetitions of the tile-list
build, the forward (render) and the backward on the caller's own Gaussians, cameras and
targets; the configuration with the smallest lists + forward + backward time wins.  The
forward output does not depend on any of these choices (bit-identical across them, which
the tests check), so the tuner changes speed only.  Results are cached in a JSON file keyed by GPU name and a
workload signature.
"""
from __future__ import annotations

import json
import os
from dataclasses import replace

import torch

from .splat import PyramidRasterizer, RenderConfig

TILES = ((16, 16), (8, 8), (32, 8), (16, 8))
BATCHES = (16, 32, 64, 128, 256)
PPT_FWD = (1, 2)
PPT_BWD = (1, 2, 4)
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pyramid_splat_gb300_autotune.json")


def _valid(tw, th, ppt):
    return th % (4 * ppt) == 0 and tw * th // ppt >= 32


def signature(N, C, cams, levels):
    return f"N{N}-C{C}-L{levels}-" + "-".join(f"{c['W']}x{c['H']}" for c in cams)


def _time(fn, reps):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / reps


def autotune(params, cams, levels, gt, loss_cfg, base: RenderConfig | None = None, decoder=None, reps=3,
             use_cache=True, log=None):
    """Returns (best RenderConfig, table of timings in ms)."""
    base = base or RenderConfig()
    N, C = params["mean"].shape[0], params["sem"].shape[1]
    key = f"{torch.cuda.get_device_name()}|{signature(N, C, cams, levels)}"
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
            if key in cache:
                return replace(base, **cache[key]["config"]), cache[key]["table"]
        except Exception:
            pass
    table = []
    best = None
    for tw, th in TILES:
        cfg0 = replace(base, tile_w=tw, tile_h=th, pixels_per_thread=1, pixels_per_thread_bwd=1, batch_bwd=0)
        r = PyramidRasterizer(N, C, cams, levels, cfg0, loss_cfg=loss_cfg)
        grads = {k: torch.zeros_like(v) for k, v in params.items()}
        r.project(params)
        r.build_lists()
        r.rasterize(params)
        dec_grad = torch.zeros_like(decoder) if decoder is not None else None
        r.loss(gt, decoder=decoder, decoder_grad=dec_grad)
        torch.cuda.synchronize()
        r.check_status()
        t_lists = _time(r.build_lists, reps)
        table.append(dict(tile=f"{tw}x{th}", batch=0, kernel="lists", ppt=0, ms=t_lists))
        # forward: batch x pixels per thread
        fwd_best = None
        for batch in BATCHES:
            for ppt in PPT_FWD:
                if not _valid(tw, th, ppt):
                    continue
                r.cfg = replace(cfg0, batch=batch, pixels_per_thread=ppt)
                r._ccfg = r.cfg.to_c()
                t = _time(lambda: r.rasterize(params), reps)
                table.append(dict(tile=f"{tw}x{th}", batch=batch, kernel="fwd", ppt=ppt, ms=t))
                if fwd_best is None or t < fwd_best[0]:
                    fwd_best = (t, batch, ppt)
        # backward (its own batch and pixels per thread; the saved state does not depend on them)
        r.cfg = replace(cfg0, batch=fwd_best[1], pixels_per_thread=fwd_best[2])
        r._ccfg = r.cfg.to_c()
        r.rasterize(params)
        bwd_best = None
        for batch in BATCHES:
            for ppt in PPT_BWD:
                if not _valid(tw, th, ppt):
                    continue
                r.cfg = replace(cfg0, batch=fwd_best[1], pixels_per_thread=fwd_best[2], batch_bwd=batch,
                                pixels_per_thread_bwd=ppt)
                r._ccfg = r.cfg.to_c()
                t = _time(lambda: r.backward(params, grads), reps)
                table.append(dict(tile=f"{tw}x{th}", batch=batch, kernel="bwd", ppt=ppt, ms=t))
                if bwd_best is None or t < bwd_best[0]:
                    bwd_best = (t, batch, ppt)
        total = t_lists + fwd_best[0] + bwd_best[0]
        if log:
            log(f"tile {tw}x{th}: lists {t_lists:.3f} ms, fwd {fwd_best[0]:.3f} ms (batch {fwd_best[1]}, "
                f"ppt {fwd_best[2]}), bwd {bwd_best[0]:.3f} ms (batch {bwd_best[1]}, ppt {bwd_best[2]})")
        chosen_fwd = dict(tile_w=tw, tile_h=th, batch=fwd_best[1], pixels_per_thread=fwd_best[2])
        if best is None or total < best[0]:
            best = (total, dict(chosen_fwd, batch_bwd=bwd_best[1], pixels_per_thread_bwd=bwd_best[2],
                                half_masks=False, half_tile_fwd=False))
        if (tw, th) == (8, 8):
            # lists with half masks, and the adjoint's one-warp-per-half mode they enable
            r.cfg = replace(cfg0, half_masks=True, batch=fwd_best[1], pixels_per_thread=fwd_best[2],
                            pixels_per_thread_bwd=1)
            r._ccfg = r.cfg.to_c()
            t_lists_h = _time(r.build_lists, reps)
            t_fwd_h = _time(lambda: r.rasterize(params), reps)  # (on the lists kept by the half rule)
            # the forward one warp per half tile too (at one pixel per thread)
            r.cfg = replace(r.cfg, pixels_per_thread=1, half_tile_fwd=True)
            r._ccfg = r.cfg.to_c()
            t_fwd_hh = _time(lambda: r.rasterize(params), reps)
            fwd_half = t_fwd_hh < t_fwd_h
            if not fwd_half:
                r.cfg = replace(r.cfg, pixels_per_thread=fwd_best[2], half_tile_fwd=False)
                r._ccfg = r.cfg.to_c()
                r.rasterize(params)
            t_bwd_h = _time(lambda: r.backward(params, grads), reps)
            table.append(dict(tile="8x8", batch=0, kernel="lists_half", ppt=0, ms=t_lists_h))
            table.append(dict(tile="8x8", batch=fwd_best[1], kernel="fwd_half", ppt=fwd_best[2], ms=t_fwd_h))
            table.append(dict(tile="8x8", batch=0, kernel="fwd_half_tile", ppt=1, ms=t_fwd_hh))
            table.append(dict(tile="8x8", batch=0, kernel="bwd_half", ppt=1, ms=t_bwd_h))
            total_h = t_lists_h + min(t_fwd_h, t_fwd_hh) + t_bwd_h
            if log:
                log(f"tile 8x8 with half masks: lists {t_lists_h:.3f} ms, fwd {t_fwd_h:.3f} ms "
                    f"(one warp per half tile: {t_fwd_hh:.3f} ms), bwd {t_bwd_h:.3f} ms")
            if total_h < best[0]:
                cfg_h = dict(chosen_fwd, batch_bwd=bwd_best[1], pixels_per_thread_bwd=1, half_masks=True,
                             half_tile_fwd=fwd_half)
                if fwd_half:
                    cfg_h["pixels_per_thread"] = 1
                best = (total_h, cfg_h)
        del r, grads
        torch.cuda.empty_cache()
    chosen = replace(base, **best[1])
    if use_cache:
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            cache = json.load(open(CACHE)) if os.path.exists(CACHE) else {}
            cache[key] = dict(config=best[1], table=table)
            json.dump(cache, open(CACHE, "w"))
        except Exception:
            pass
    return chosen, table
