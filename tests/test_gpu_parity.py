"""GPU parity of the CUDA path (called through the C ABI) against the FP64 oracle.

Forward: |gpu - oracle| <= 1e-4 |oracle| + 1e-5 per pixel and channel.  Gradients:
|gpu - oracle| <= 2e-3 |oracle| + 1e-6 max|oracle| per element.  Tile lists: against the
FP64 definition of the set N per tile (every Gaussian whose alpha reaches 1/255 at a pixel of
the tile is listed; every listed one comes close to the tile; inside each tile the order is
(float32 key of the FP64 camera depth, index)).  Pixels where a decision of the method is not
fixed for a float32 evaluation -- alpha within the measured float32 alpha error of the skip
threshold, the transmittance within its propagated error of T_min, an undecided depth key
next to a neighbouring key -- are excluded; their share is asserted to be below 0.1 %.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from helpers import (ALPHA_TOL, T_TOL, AMBIGUOUS, AMBIGUOUS_GRAD, FWD_ABS, FWD_REL, MAX_MASKED, check_close, check_grads,
                     ref_render, unambiguous)
from kernel_rules import kept_and_masks, tile_halves_reach, tile_reaches_alpha_min

pytestmark = pytest.mark.gpu

KEYS = ("mean", "log_scale", "quat", "opacity_logit", "rgb", "sem")


def f32_camera(cam):
    c = dict(cam)
    c["R_cw"] = np.asarray(cam["R_cw"], np.float32).astype(np.float64)
    c["t_cw"] = np.asarray(cam["t_cw"], np.float32).astype(np.float64)
    for k in ("fx", "fy", "cx", "cy"):
        c[k] = float(np.float32(cam[k]))
    return c


def make(g, cams, levels=1, capacity=None, **kw):
    from paper_2412_01217_gb300 import PyramidRasterizer, RenderConfig, to_device_params
    C = g["sem"].shape[1]
    r = PyramidRasterizer(g["mean"].shape[0], C, cams, levels, RenderConfig(**kw), capacity=capacity)
    return r, to_device_params(g)


def view_images(r, v, C):
    return dict(rgb=r.view_slice(r.img_rgb, v, 3).cpu().numpy(),
                depth=r.view_slice(r.img_depth, v, 1)[0].cpu().numpy(),
                sem=r.view_slice(r.img_sem, v, C).cpu().numpy(),
                T=r.view_slice(r.T_final, v, 1)[0].cpu().numpy(),
                n_contrib=r.view_slice(r.n_contrib, v, 1)[0].cpu().numpy())


def oracle_cams(cams, levels):
    out = []
    for c in cams:
        out.extend(oracle.level_cameras(c, levels))
    return out


@pytest.fixture(scope="module")
def cloud():
    g = synthetic.cloud_scene(2000, 8, seed=1)
    cam = f32_camera(synthetic.cloud_camera())
    return g, cam


def test_projection_matches_oracle(cloud):
    g, cam = cloud
    r, p = make(g, [cam])
    r.project(p)
    torch.cuda.synchronize()
    geo = r.geo.view(-1, 8).cpu().numpy().astype(np.float64)
    rect = r.rect.view(-1, 2).cpu().numpy().view(np.uint32)
    pr = oracle.project(g, cam)
    P = oracle.P
    vg = rect[:, 0] != rect[:, 1]
    vo = pr[:, P["VALID"]] == 1
    assert vg.sum() > 1000
    assert not (vg & ~vo).any(), "GPU keeps a Gaussian the oracle culls"
    m = vg
    # the 2D mean is stored as int16 integer part + float fraction
    packed = r.geo.view(-1, 8)[:, 7].cpu().numpy().view(np.uint32)
    ui = (packed & 0xFFFF).astype(np.uint16).view(np.int16).astype(np.float64)
    vi = (packed >> 16).astype(np.uint16).view(np.int16).astype(np.float64)
    check_close("u", ui[m] + geo[m, 0], pr[m, P["U"]], 0, 2e-6)
    check_close("v", vi[m] + geo[m, 1], pr[m, P["V"]], 0, 2e-6)
    check_close("depth", geo[m, 2], pr[m, P["DEPTH"]], 1e-6, 0)
    check_close("opacity", geo[m, 3], pr[m, P["OPAC"]], 1e-6, 1e-7)
    # the record stores the conditional factors: conic = 2 [[m00^2 + m10^2, m10 m11], [., m11^2]]
    m00, m10, m11 = geo[m, 4], geo[m, 5], geo[m, 6]
    conic = {"CA": 2 * (m00 ** 2 + m10 ** 2), "CB": 2 * m10 * m11, "CC": 2 * m11 ** 2}
    scale = np.maximum(np.abs(pr[m, P["CA"]]), np.abs(pr[m, P["CC"]]))
    for k, val in conic.items():
        check_close(f"conic {k}", val / scale, pr[m, P[k]] / scale, 0, 2e-5)
    # every pixel where alpha can reach 1/255 lies inside the GPU tile rectangle
    tx0, ty0 = rect[:, 0] & 0xFFFF, rect[:, 0] >> 16
    tx1, ty1 = rect[:, 1] & 0xFFFF, rect[:, 1] >> 16
    for i in np.where(vo)[0]:
        x0 = max(0, int(np.ceil(pr[i, P["U"]] - pr[i, P["EXTX"]])))
        x1 = min(cam["W"] - 1, int(np.floor(pr[i, P["U"]] + pr[i, P["EXTX"]])))
        y0 = max(0, int(np.ceil(pr[i, P["V"]] - pr[i, P["EXTY"]])))
        y1 = min(cam["H"] - 1, int(np.floor(pr[i, P["V"]] + pr[i, P["EXTY"]])))
        if x0 > x1 or y0 > y1:
            continue
        assert vg[i], i
        assert tx0[i] <= x0 // 16 and tx1[i] >= x1 // 16 + 1 and ty0[i] <= y0 // 16 and ty1[i] >= y1 // 16 + 1, i
        assert tx1[i] - tx0[i] <= (x1 // 16 + 1 - x0 // 16) + 1 and ty1[i] - ty0[i] <= (y1 // 16 + 1 - y0 // 16) + 1


def _gpu_lists(r):
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    K = r.instance_count()
    tiles = r.tile[:K].cpu().numpy().view(np.uint32).astype(np.int64)
    recs = r.record[:K].cpu().numpy().view(np.uint32).astype(np.int64)
    if r.cfg.half_masks:  # records in bits 0-29, half masks in bits 30-31
        recs &= (1 << 30) - 1
    ranges = r.ranges.view(-1, 2).cpu().numpy().astype(np.int64)
    return K, tiles, recs, ranges


def _gpu_half_masks(r, K):
    """Each listed instance's half mask (bit 0: top half of the tile, bit 1: bottom)."""
    return (r.record[:K].cpu().numpy().view(np.uint32) >> 30).astype(np.int64)


def _check_ranges_and_order(r, tiles, ranges):
    """Ranges hold each tile's [start, end) ((0, 0) when empty); the work order lists every
    tile once, by descending half-octave bucket of its instance count, ascending id within a
    bucket."""
    assert np.all(np.diff(tiles) >= 0)
    t = np.arange(r.n_tiles)
    starts, ends = np.searchsorted(tiles, t, "left"), np.searchsorted(tiles, t, "right")
    expect = np.stack([np.where(starts == ends, 0, starts), np.where(starts == ends, 0, ends)], 1)
    assert np.array_equal(ranges, expect)
    n = ranges[:, 1] - ranges[:, 0]
    lz = np.floor(np.log2(np.maximum(n, 1))).astype(np.int64)
    sub = np.where(lz >= 1, (n >> np.maximum(lz - 1, 0)) & 1, 0)
    bucket = np.where(n > 0, 1 + 2 * lz + sub, 0)
    assert np.array_equal(r.order.cpu().numpy().astype(np.int64), np.argsort(-bucket, kind="stable"))


def lists_match_definition(r, g, ocams):
    """PRIMARY tile-list parity, against the FP64 definition of the set N of Eq. 7-9 per tile
    (oracle.tile_pairs / tile_reach / the projection's depth key), independent of every float32
    rule of the kernels:
      * every (Gaussian, tile) whose alpha reaches 1/255 at a pixel centre of the tile is listed
        (pairs within the float32 alpha error of the threshold may go either way);
      * every listed pair comes close to its tile: the least exponent of the footprint over the
        tile's pixel-centre rectangle is at most ln(o / alpha_min) + 2e-3 (the lists' margin);
      * inside each tile the records follow (float32 key of the FP64 depth, record index),
        except next to an undecided key.
    Returns (instances, pairs that must be listed, listed pairs that reach no pixel)."""
    K, tiles, recs, ranges = _gpu_lists(r)
    _check_ranges_and_order(r, tiles, ranges)
    tw, th, N = r.cfg.tile_w, r.cfg.tile_h, r.N
    amin = 1.0 / 255.0
    key = np.zeros(r.V * N, np.float32)
    damb = np.zeros(r.V * N, bool)
    n_must = n_extra = 0
    for v, oc in enumerate(ocams):
        vh = r.views_host[v]
        pr = oracle.project(g, oc)
        key[v * N:(v + 1) * N] = pr[:, oracle.P["DKEY"]]
        damb[v * N:(v + 1) * N] = pr[:, oracle.P["DAMB"]] > 0
        sel = (recs // N) == v
        gi = recs[sel] % N
        loc = tiles[sel] - vh.tile_offset
        assert np.all((loc >= 0) & (loc < vh.tiles_x * vh.tiles_y))
        gtx, gty = loc % vh.tiles_x, loc // vh.tiles_x
        listed = set(zip(gi.tolist(), gtx.tolist(), gty.tolist()))
        assert len(listed) == int(sel.sum()), "a (Gaussian, tile) pair is listed twice"
        fg, ftx, fty = oracle.tile_pairs(pr, oc, tw, th)
        reach = oracle.tile_reach(pr, oc, fg, ftx, fty, tw, th)
        must = reach["alpha"] >= amin * (1 + ALPHA_TOL)
        missing = [p for p in zip(fg[must].tolist(), ftx[must].tolist(), fty[must].tolist()) if p not in listed]
        assert not missing, f"view {v}: {len(missing)} (Gaussian, tile) pairs reach alpha_min but are not listed: {missing[:5]}"
        got = oracle.tile_reach(pr, oc, gi, gtx, gty, tw, th)
        far = ~(got["sigma_min"] <= got["thr"] + 2e-3 + 1e-4 * np.abs(got["thr"]))
        assert not far.any(), f"view {v}: {int(far.sum())} listed pairs the footprint does not reach"
        # half masks: a half of the tile holding a pixel centre where alpha reaches alpha_min
        # (FP64) is marked
        hm = _gpu_half_masks(r, K)[sel] if r.cfg.half_masks else np.full(len(gi), 3, np.int64)
        for h in (0, 1):
            hty = 2 * gty + h
            inside = hty * (th // 2) < oc["H"]
            if not inside.any():
                continue
            hr = oracle.tile_reach(pr, oc, gi[inside], gtx[inside], hty[inside], tw, th // 2)
            need = hr["alpha"] >= amin * (1 + ALPHA_TOL)
            bit = ((hm[inside] >> h) & 1) == 1
            assert np.all(bit | ~need), f"view {v}: {int((need & ~bit).sum())} reached halves unmarked"
        n_must += int(must.sum())
        n_extra += int((got["alpha"] < amin).sum())
    same = tiles[1:] == tiles[:-1]
    a, b = recs[:-1][same], recs[1:][same]
    ka, kb = key[a].view(np.int32).astype(np.int64), key[b].view(np.int32).astype(np.int64)
    in_order = (ka < kb) | ((ka == kb) & (a < b))
    undecided = (damb[a] | damb[b]) & (np.abs(ka - kb) <= 1)
    assert np.all(in_order | undecided), f"{int((~in_order & ~undecided).sum())} adjacent pairs out of depth order"
    assert undecided.mean() < 1e-3 if len(undecided) else True
    return K, n_must, n_extra


def lists_match_kernel_rule(r):
    """KERNEL UNIT TEST (not parity with the paper's definition): given the kernels' own
    float32 records and their float32 culling rule (kernel_rules.py), the emitted lists are
    bit-exactly the (tile, depth bits, record) order that oracle.tile_lists defines -- this
    isolates the sort and emission kernels from the projection's rounding."""
    K, tiles, recs, ranges = _gpu_lists(r)
    rect = r.rect.view(-1, 2).cpu().numpy().view(np.uint32)
    rects = np.stack([rect[:, 0] & 0xFFFF, rect[:, 0] >> 16, rect[:, 1] & 0xFFFF, rect[:, 1] >> 16], 1)
    depth = r.geo.view(-1, 8)[:, 2].cpu().numpy()
    tx = [r.views_host[v].tiles_x for v in range(r.V)]
    to = [r.views_host[v].tile_offset for v in range(r.V)]
    geo = r.geo.view(-1, 8).cpu().numpy()
    ext = r.ext.view(-1, 2).cpu().numpy()
    tw, th = r.cfg.tile_w, r.cfg.tile_h
    Wv = np.array([r.views_host[v].W for v in range(r.V)])
    Hv = np.array([r.views_host[v].H for v in range(r.V)])

    half = r.cfg.half_masks

    def band(recs_, tx_, ty_):
        v = recs_ // r.N
        X0, Y0 = tx_ * tw, ty_ * th
        return (geo[recs_], ext[recs_], X0, np.minimum(X0 + tw - 1, Wv[v] - 1), Y0,
                np.minimum(Y0 + th - 1, Hv[v] - 1))

    def halves(recs_, tx_, ty_):
        return tile_halves_reach(*band(recs_, tx_, ty_), th)

    def keep(recs_, tx_, ty_):
        # without half masks the rule runs on the tile row's whole band; with them, a tile
        # is kept when either half's rule keeps it
        if not half:
            return tile_reaches_alpha_min(*band(recs_, tx_, ty_))
        return kept_and_masks(recs_, tx_, ty_, *halves(recs_, tx_, ty_))[0]

    rt, rr, rg = oracle.tile_lists(rects, depth, tx, to, r.n_tiles, r.N, keep=keep)
    assert K == len(rt)
    assert np.array_equal(tiles, rt)
    assert np.array_equal(recs, rr)
    assert np.array_equal(ranges, rg)
    if not half:
        return K
    # each instance's half mask, from the same rule (a run's length is its kept tiles' count)
    v = rr // r.N
    local = rt - np.asarray(to, np.int64)[v]
    ltx, lty = local % np.asarray(tx, np.int64)[v], local // np.asarray(tx, np.int64)[v]
    _, want = kept_and_masks(rr, ltx, lty, *halves(rr, ltx, lty))
    got = _gpu_half_masks(r, K)
    assert np.array_equal(got, want), f"{int((got != want).sum())} of {K} half masks differ"
    return K


def test_tile_lists_match_definition_single_view(cloud):
    g, cam = cloud
    for tw, th, half in ((16, 16, False), (8, 8, False), (32, 8, False), (8, 8, True), (16, 16, True)):
        r, p = make(g, [cam], tile_w=tw, tile_h=th, half_masks=half)
        r.project(p)
        r.build_lists()
        K, n_must, n_extra = lists_match_definition(r, g, [cam])
        assert K > 2000 and n_must > 0.5 * K
        assert lists_match_kernel_rule(r) == K


@pytest.mark.parametrize("half", [False, True])
def test_tile_lists_with_17_bit_tile_ids(half):
    """8 x 8 tiles of a 2400 x 1800 view: 67,500 tiles need 17-bit tile ids, so the tile sort
    runs three radix passes of 6, 6 and 5 bits (the width the batched workload's 92k tiles
    take); with half masks the last pass splits them from the records."""
    g = synthetic.cloud_scene(1500, 8, seed=3)
    cam = f32_camera(synthetic.make_camera(2400, 1800, 2250.0, 2250.0, 1199.5, 899.5))
    r, p = make(g, [cam], tile_w=8, tile_h=8, capacity=1 << 20, half_masks=half)
    assert r.n_tiles == 300 * 225 and r.n_tiles > 1 << 16
    r.project(p)
    r.build_lists()
    K, n_must, n_extra = lists_match_definition(r, g, [cam])
    assert K > 100000 and n_must > 0.5 * K
    assert lists_match_kernel_rule(r) == K


@pytest.mark.parametrize("half", [False, True])
def test_tile_lists_overflow_without_the_slot_cache(half):
    """The emission pass reads each (record, tile row) slot's kept run from a cache that the
    count pass fills when the slots fit the instance capacity, and recomputes the run
    otherwise.  Each slot keeps one or more tiles, so the slots fit whenever the instances do;
    with a capacity below the slot count the recomputing path runs, the overflow is reported
    (SG_STATUS_CAPACITY) and the instance count is still the exact K."""
    room, g, cams = room_small()
    r, p = make(g, cams, levels=3, tile_w=8, tile_h=8, half_masks=half)
    r.project(p)
    r.build_lists()
    K = _gpu_lists(r)[0]
    rows = r.rect.view(-1, 2).cpu().numpy().view(np.uint32)
    ty0, ty1 = rows[:, 0] >> 16, rows[:, 1] >> 16
    tx0, tx1 = rows[:, 0] & 0xFFFF, rows[:, 1] & 0xFFFF
    slots = int(np.where((tx1 > tx0) & (ty1 > ty0), ty1.astype(np.int64) - ty0, 0).sum())
    assert 0 < slots < K
    r2, p2 = make(g, cams, levels=3, capacity=slots - 1, tile_w=8, tile_h=8, half_masks=half)
    r2.project(p2)
    r2.build_lists()
    torch.cuda.synchronize()
    assert int(r2.status.item()) & 1  # SG_STATUS_CAPACITY
    assert r2.instance_count() == K


def room_small(n=20000, C=16, seed=4, ncam=2, W=320, H=180):
    room = synthetic.Room(n_classes=32, seed=3)
    intr = dict(W=W, H=H, fx=W / 2.0, fy=W / 2.0, cx=W / 2 - 0.5, cy=H / 2 - 0.5)
    cams = [f32_camera(c) for c in room.trajectory(ncam, intr, seed=7)]
    g = room.sample_gaussians(n, C, seed=seed, sem_mode="random")
    return room, g, cams


@pytest.mark.parametrize("tile, half", [((16, 16), False), ((8, 8), True)])
def test_tile_lists_match_definition_pyramid_multi_view(tile, half):
    room, g, cams = room_small()
    r, p = make(g, cams, levels=3, tile_w=tile[0], tile_h=tile[1], half_masks=half)
    r.project(p)
    r.build_lists()
    K, n_must, n_extra = lists_match_definition(r, g, oracle_cams(cams, 3))
    assert K > 10000 and n_must > 0.5 * K
    assert lists_match_kernel_rule(r) == K


@pytest.mark.parametrize("isotropic", [False, True])
def test_forward_matches_oracle_cloud(cloud, isotropic):
    g, cam = cloud
    r, p = make(g, [cam], isotropic=isotropic)
    r.forward(p)
    got = view_images(r, 0, 8)
    ref = ref_render(g, cam, dict(isotropic=int(isotropic)))
    ok = unambiguous(ref["flags"])
    for k in ("rgb", "depth", "sem", "T"):
        check_close(k, got[k], ref[k], FWD_REL, FWD_ABS, mask=ok)
    assert np.array_equal(got["n_contrib"][ok], ref["n_contrib"][ok])


def test_forward_bitwise_identical_across_tiles_batches_and_runs(cloud):
    g, cam = cloud
    base = None
    # (the 8x8 cases with half masks: persistent ones run the forward one warp per half tile)
    for tw, th, batch, pers, ppt, half in ((16, 16, 128, True, 1, False), (8, 8, 32, True, 1, False),
                                           (32, 8, 256, False, 2, False), (16, 8, 64, True, 2, False),
                                           (16, 16, 128, True, 4, False), (8, 8, 64, False, 2, False),
                                           (8, 8, 64, True, 1, True), (8, 8, 64, False, 1, True),
                                           (16, 16, 128, True, 1, False)):
        r, p = make(g, [cam], tile_w=tw, tile_h=th, batch=batch, persistent=pers, pixels_per_thread=ppt,
                    half_masks=half, half_tile_fwd=half and pers)
        r.forward(p)
        im = view_images(r, 0, 8)
        if base is None:
            base = im
            continue
        for k in ("rgb", "depth", "sem", "T", "n_contrib"):
            assert np.array_equal(im[k], base[k]), (k, tw, th, batch, pers, ppt, half)


@pytest.mark.parametrize("ppt, batch_bwd, isotropic, tile", [(1, 0, False, "16x16"), (2, 0, False, "16x16"),
                                                           (4, 0, False, "16x16"), (1, 16, False, "16x16"),
                                                           (2, 64, False, "16x16"), (1, 0, True, "16x16"),
                                                           (1, 16, False, "8x8"), (1, 16, False, "8x8-half"),
                                                           (1, 0, True, "8x8-half")])
def test_backward_matches_oracle_cloud(cloud, ppt, batch_bwd, isotropic, tile):
    """8x8-half: lists with half masks, so the adjoint (and, in the isotropic case, the forward)
    runs one warp per half tile."""
    g, cam = cloud
    tw, th = (int(x) for x in tile.split("-")[0].split("x"))
    half = tile.endswith("half")
    r, p = make(g, [cam], pixels_per_thread_bwd=ppt, batch_bwd=batch_bwd, isotropic=isotropic, tile_w=tw,
                tile_h=th, half_masks=half, half_tile_fwd=half and isotropic)
    r.forward(p)
    ocfg = dict(isotropic=int(isotropic))
    ref_f = ref_render(g, cam, ocfg)
    keep = unambiguous(ref_f["flags"], AMBIGUOUS_GRAD).astype(np.float64)
    rng = np.random.default_rng(11)
    H, W, C = cam["H"], cam["W"], 8
    up_rgb = rng.normal(size=(3, H, W)) * keep
    up_d = rng.normal(size=(H, W)) * keep
    up_s = rng.normal(size=(C, H, W)) * keep
    dl = (torch.tensor(up_rgb.reshape(-1), dtype=torch.float32, device="cuda"),
          torch.tensor(up_d.reshape(-1), dtype=torch.float32, device="cuda"),
          torch.tensor(up_s.reshape(-1), dtype=torch.float32, device="cuda"))
    grads = {k: torch.zeros_like(v) for k, v in p.items()}
    r.backward(p, grads, dL=dl)
    got = {k: v.cpu().numpy() for k, v in grads.items()}
    # the float32 inputs the GPU saw are exactly what the oracle gets
    up_rgb32 = dl[0].cpu().numpy().astype(np.float64).reshape(3, H, W)
    up_d32 = dl[1].cpu().numpy().astype(np.float64).reshape(H, W)
    up_s32 = dl[2].cpu().numpy().astype(np.float64).reshape(C, H, W)
    ref = oracle.render_backward(g, cam, up_rgb32, up_d32, up_s32, cfg=ocfg)
    check_grads(got, ref, KEYS)
    if isotropic:  # Eq. 2 uses only log_scale[0]: rotation and the other scales get zero
        assert not got["quat"].any() and not got["log_scale"][:, 1:].any()
    # the persistent work queue and the per-record gradient workspace are left zero, so the
    # next launch needs no memset; a second backward adds exactly the same gradients
    assert not r.work_counter.any() and not r.bwd_ws.any()
    again = {k: torch.zeros_like(v) for k, v in p.items()}
    r.backward(p, again, dL=dl)
    for k in KEYS:
        a, b = again[k].cpu().numpy(), got[k]
        assert np.allclose(a, b, rtol=1e-4, atol=1e-6 * (np.abs(b).max() + 1e-12)), k


def test_pyramid_build_matches_oracle():
    room, g, cams = room_small(ncam=2, W=322, H=183)
    from paper_2412_01217_gb300 import build_pyramid
    r, p = make(g, cams, levels=3)
    frames = [room.raycast(c) for c in cams]
    for f in frames:
        f["label"][:3, :5] = -1
        f["depth"][10:14, 20:30] = 0.0
    gt = build_pyramid(r, [f["rgb"] for f in frames], [f["depth"] for f in frames],
                       [f["label"] for f in frames])
    torch.cuda.synchronize()
    for c, f in enumerate(frames):
        ref = oracle.build_pyramid(f["rgb"], f["depth"], f["label"], 3)
        for l in range(3):
            v = c * 3 + l
            check_close(f"rgb c{c} l{l}", r.view_slice(gt["rgb"], v, 3).cpu().numpy(), ref[l][0], 1e-6, 1e-6)
            check_close(f"depth c{c} l{l}", r.view_slice(gt["depth"], v, 1)[0].cpu().numpy(), ref[l][1], 1e-6, 1e-6)
            assert np.array_equal(r.view_slice(gt["label"], v, 1)[0].cpu().numpy(), ref[l][2])


# (semantic channels, classes, W, H, keyframes, levels) per case; the tensor-core decoder
# kernel is persistent, so the larger images give its blocks many 256-pixel items each
LOSS_CASES = {"ce": (8, 8, 100, 70, 2, 2), "ce_decoder": (8, 8, 100, 70, 2, 2),
              "ce_decoder32": (16, 32, 100, 70, 2, 2), "ce_decoder16_640x480": (16, 16, 640, 480, 1, 2),
              "ce_decoder32_1200x680": (16, 32, 1200, 680, 1, 3), "ce_decoder32x32_320x240": (32, 32, 320, 240, 2, 2),
              "paper": (8, 8, 100, 70, 2, 2)}


@pytest.mark.parametrize("mode", list(LOSS_CASES))
def test_loss_matches_oracle(mode):
    from paper_2412_01217_gb300 import LossConfig
    rng = np.random.default_rng(5)
    Cs, K, W, H, ncam, levels = LOSS_CASES[mode]
    room, g, cams = room_small(n=2000, ncam=ncam, W=W, H=H, C=Cs)
    r, p = make(g, cams, levels=levels)
    P = r.P
    rend = (torch.tensor(rng.uniform(size=3 * P), dtype=torch.float32, device="cuda"),
            torch.tensor(rng.uniform(1, 3, size=P), dtype=torch.float32, device="cuda"),
            torch.tensor(rng.normal(size=Cs * P), dtype=torch.float32, device="cuda"))
    gdepth = rng.uniform(1, 3, size=P)
    gdepth[rng.uniform(size=P) < 0.2] = 0.0
    gt = dict(rgb=torch.tensor(rng.uniform(size=3 * P), dtype=torch.float32, device="cuda"),
              depth=torch.tensor(gdepth, dtype=torch.float32, device="cuda"),
              label=torch.tensor(rng.integers(-1, K, size=P), dtype=torch.int32, device="cuda"),
              sem=torch.tensor(rng.uniform(size=Cs * P), dtype=torch.float32, device="cuda"))
    dec = dgrad = None
    if mode.startswith("ce_decoder"):
        dec = torch.tensor(rng.normal(size=(K, Cs)) * 0.5, dtype=torch.float32, device="cuda")
        dgrad = torch.zeros_like(dec)
    lc = LossConfig(sem_mode="paper" if mode == "paper" else "ce", n_classes=K)
    r.loss(gt, rendered=rend, decoder=dec, decoder_grad=dgrad, loss_cfg=lc)
    torch.cuda.synchronize()
    terms = r.terms.view(-1, 4).cpu().numpy()
    dec_ref_total = np.zeros((K, Cs))
    for v in range(r.V):
        sl = lambda t, n: r.view_slice(t, v, n).cpu().numpy().astype(np.float64)
        tot, tm, gr = oracle.level_loss(sl(rend[0], 3), sl(rend[1], 1)[0], sl(rend[2], Cs), sl(gt["rgb"], 3),
                                        sl(gt["depth"], 1)[0],
                                        sl(gt["sem"], Cs) if mode == "paper" else r.view_slice(gt["label"], v, 1)[0].cpu().numpy(),
                                        sem_mode="paper" if mode == "paper" else "ce",
                                        decoder=dec.cpu().numpy() if dec is not None else None)
        assert terms[v, 0] == pytest.approx(tm["L_r"], rel=1e-5)
        assert terms[v, 1] == pytest.approx(tm["L_d"], rel=1e-5)
        assert terms[v, 2] == pytest.approx(tm["L_s"], rel=1e-5)
        assert terms[v, 3] == pytest.approx(tot, rel=1e-5)
        for name, buf, n in (("rgb", r.dL_rgb, 3), ("depth", r.dL_depth, 1), ("sem", r.dL_sem, Cs)):
            got = r.view_slice(buf, v, n).cpu().numpy()
            ref = gr[name].reshape(got.shape)
            check_close(f"dL/d{name} v{v}", got, ref, 1e-4, 1e-4 * np.abs(ref).max())
        if dec is not None:
            dec_ref_total += gr["decoder"]
    if dec is not None:
        check_close("dL/ddecoder", dgrad.cpu().numpy(), dec_ref_total, 1e-4, 1e-6)


@pytest.mark.parametrize("isotropic, half", [(False, False), (True, False), (False, True)])
def test_multiview_pyramid_forward_backward_matches_oracle(isotropic, half):
    """Two keyframes x three levels rendered in ONE persistent launch: every pixel of
    every view-level against the oracle, and all parameter gradients; also with the Eq. 2
    isotropic projection, whose radius f r / d takes each level's own focal length, and with
    8x8 tiles carrying half masks (the adjoint one warp per half tile)."""
    room, g, cams = room_small(n=6000, ncam=2, W=160, H=96)
    kw = dict(tile_w=8, tile_h=8, pixels_per_thread_bwd=1, half_masks=True) if half else {}
    r, p = make(g, cams, levels=3, isotropic=isotropic, **kw)
    r.forward(p)
    ocams = oracle_cams(cams, 3)
    ocfg = dict(isotropic=int(isotropic))
    rng = np.random.default_rng(2)
    ups = []
    for v, oc in enumerate(ocams):
        got = view_images(r, v, 16)
        ref = ref_render(g, oc, ocfg)
        ok = unambiguous(ref["flags"], limit=max(MAX_MASKED, 1.0 / ref["flags"].size))
        for k in ("rgb", "depth", "sem", "T"):
            check_close(f"v{v} {k}", got[k], ref[k], FWD_REL, FWD_ABS, mask=ok)
        assert np.array_equal(got["n_contrib"][ok], ref["n_contrib"][ok])
        keep = unambiguous(ref["flags"], AMBIGUOUS_GRAD, limit=max(MAX_MASKED, 1.0 / ref["flags"].size)).astype(np.float64)
        H, W = oc["H"], oc["W"]
        ups.append((rng.normal(size=(3, H, W)) * keep, rng.normal(size=(H, W)) * keep,
                    rng.normal(size=(16, H, W)) * keep))
    dl = [torch.zeros(3 * r.P, device="cuda"), torch.zeros(r.P, device="cuda"), torch.zeros(16 * r.P, device="cuda")]
    for v, (a, b, c) in enumerate(ups):
        r.view_slice(dl[0], v, 3).copy_(torch.tensor(a, dtype=torch.float32))
        r.view_slice(dl[1], v, 1).copy_(torch.tensor(b[None], dtype=torch.float32))
        r.view_slice(dl[2], v, 16).copy_(torch.tensor(c, dtype=torch.float32))
    grads = {k: torch.zeros_like(t) for k, t in p.items()}
    r.backward(p, grads, dL=tuple(dl))
    got = {k: t.cpu().numpy() for k, t in grads.items()}
    ref = {k: 0.0 for k in KEYS}
    for v, oc in enumerate(ocams):
        a = r.view_slice(dl[0], v, 3).cpu().numpy().astype(np.float64)
        b = r.view_slice(dl[1], v, 1)[0].cpu().numpy().astype(np.float64)
        c = r.view_slice(dl[2], v, 16).cpu().numpy().astype(np.float64)
        rv = oracle.render_backward(g, oc, a, b, c, cfg=ocfg)
        for k in KEYS:
            ref[k] = ref[k] + rv[k]
    check_grads(got, ref, KEYS)
    if isotropic:
        assert not got["quat"].any() and not got["log_scale"][:, 1:].any()


def test_capacity_overflow_sets_status_and_reports_need(cloud):
    g, cam = cloud
    r, p = make(g, [cam], capacity=500)
    r.forward(p)
    torch.cuda.synchronize()
    assert int(r.status.item()) & 1
    full, _ = make(g, [cam])
    full.project(p)
    full.build_lists()
    torch.cuda.synchronize()
    assert r.instance_count() == full.instance_count() > 500
    from paper_2412_01217_gb300 import SgError
    with pytest.raises(SgError):
        r.check_status()


def test_adam_step_matches_numpy():
    import ctypes as C
    from paper_2412_01217_gb300._lib import call
    rng = np.random.default_rng(0)
    n = 10007
    p0, g0 = rng.normal(size=n), rng.normal(size=n)
    m0, v0 = rng.normal(size=n) * 0.1, rng.uniform(size=n) * 0.1
    t = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in (p0, g0, m0, v0)]
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    call("sg_adam_step", *[C.c_void_p(x.data_ptr()) for x in t], n, 1e-2, 0.9, 0.999, 1e-8, 3, s)
    torch.cuda.synchronize()
    m = 0.9 * m0 + 0.1 * g0
    v = 0.999 * v0 + 0.001 * g0 ** 2
    p = p0 - 1e-2 * (m / (1 - 0.9 ** 3)) / (np.sqrt(v / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(t[0].cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    assert np.allclose(t[2].cpu().numpy(), m, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("sizes, offset", [((4000, 1200, 16), 0), ((4001, 7, 33), 1)])
def test_adam_multi_matches_numpy(sizes, offset):
    """Fused multi-group Adam: the 16-byte path (every group a multiple of 4 elements, aligned)
    and the scalar path (odd sizes, one group starting 4 bytes into its buffer); gradients zeroed."""
    import ctypes as C
    from paper_2412_01217_gb300._lib import SgAdamGroup, call
    rng = np.random.default_rng(1)
    groups, ref, keep = [], [], []
    for k, n in enumerate(sizes):
        p0, g0 = rng.normal(size=n), rng.normal(size=n)
        g0[::17] = 0.0
        m0, v0 = rng.normal(size=n) * 0.1, rng.uniform(size=n) * 0.1
        v0[::17] = 0.0
        m0[::17] = 0.0
        bufs = []
        for a in (p0, g0, m0, v0):
            o = offset if k == 1 else 0
            t = torch.zeros(n + o, dtype=torch.float32, device="cuda")
            t[o:] = torch.tensor(a, dtype=torch.float32)
            bufs.append(t[o:])
        keep.append(bufs)
        lr = 1e-2 * (k + 1)
        groups.append(SgAdamGroup(*[b.data_ptr() for b in bufs], n, lr))
        # the kernel receives the betas as float32: the reference uses the same values
        b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
        p0, g0, m0, v0 = (np.float32(a).astype(np.float64) for a in (p0, g0, m0, v0))
        m = b1 * m0 + (1 - b1) * g0
        v = b2 * v0 + (1 - b2) * g0 ** 2
        p = p0 - lr * (m / (1 - b1 ** 3)) / (np.sqrt(v / (1 - b2 ** 3)) + 1e-15)
        ref.append((p, m, v))
    arr = (SgAdamGroup * len(groups))(*groups)
    call("sg_adam_multi", arr, len(groups), 0.9, 0.999, 1e-15, 3, 1, None,
         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    for (p, m, v), bufs in zip(ref, keep):
        assert np.allclose(bufs[0].cpu().numpy(), p, rtol=1e-5, atol=1e-6)
        assert np.allclose(bufs[2].cpu().numpy(), m, rtol=1e-5, atol=1e-7)
        assert np.allclose(bufs[3].cpu().numpy(), v, rtol=1e-5, atol=1e-9)
        assert not bufs[1].any()


def test_float32_alpha_and_transmittance_errors_are_within_the_bands():
    """The ambiguity bands of every parity test bound the kernels' float32 errors.
    Alpha (helpers.ALPHA_TOL): isolated Gaussians (rotated, elongated, opacities 0.05-0.98, a
    general camera pose) with colour (1, 0, 0) render rgb[0] = alpha at every pixel they reach,
    which the oracle gives in FP64; pixels the oracle skips outside the band are skipped.
    Transmittance (helpers.T_TOL): T at 8000 sampled pixels of a dense room level."""
    rng = np.random.default_rng(31)
    W, H, cell = 320, 240, 20
    cam = synthetic.make_camera(W, H, 300.0, 300.0, 159.5, 119.5)
    a = 0.2
    R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    cam = f32_camera(dict(cam, R_cw=R, t_cw=np.array([0.05, -0.02, 0.1])))
    nx, ny = W // cell, H // cell
    n = nx * ny
    z = rng.uniform(2.0, 4.0, n)
    cx, cy = (np.arange(n) % nx) * cell + cell / 2, (np.arange(n) // nx) * cell + cell / 2
    u = (cx + rng.uniform(-2, 2, n) - cam["cx"]) / cam["fx"] * z
    v = (cy + rng.uniform(-2, 2, n) - cam["cy"]) / cam["fy"] * z
    pc = np.stack([u, v, z], 1)
    Rc, tc = np.asarray(cam["R_cw"]).reshape(3, 3), np.asarray(cam["t_cw"])
    mean = (pc - tc) @ Rc          # world point with R mean + t = pc
    q = rng.normal(size=(n, 4))
    s = np.stack([rng.uniform(0.004, 0.012, n), rng.uniform(0.0015, 0.006, n), rng.uniform(0.002, 0.008, n)], 1)
    o = rng.uniform(0.05, 0.98, n)
    f32 = lambda x: np.ascontiguousarray(x, np.float32)
    g = dict(mean=f32(mean), log_scale=f32(np.log(s)), quat=f32(q / np.linalg.norm(q, axis=1, keepdims=True)),
             opacity_logit=f32(np.log(o / (1 - o))), rgb=f32(np.tile([1.0, 0.0, 0.0], (n, 1))),
             sem=f32(np.zeros((n, 4))))
    r, p = make(g, [cam])
    r.forward(p)
    got = view_images(r, 0, 4)
    ref = ref_render(g, cam)
    assert ref["n_contrib"].max() == 1  # isolated footprints
    al = ref["rgb"][0]
    amin, amax = 1 / 255, 0.99
    sel = (al >= amin * (1 + ALPHA_TOL)) & (al <= amax * (1 - ALPHA_TOL))
    rel = np.abs(got["rgb"][0][sel] - al[sel]) / al[sel]
    print(f"float32 alpha relative error: max {rel.max():.3e}, p99.9 {np.quantile(rel, 0.999):.3e} "
          f"over {sel.sum()} pixels")
    assert sel.sum() > 3000
    assert rel.max() <= ALPHA_TOL, rel.max()
    below = (al == 0) & ((ref["flags"] & oracle.FLAG_SKIP) == 0)
    assert np.all(got["rgb"][0][below] == 0)
    # transmittance in a dense scene (35-40 contributors per pixel)
    room = synthetic.Room(n_classes=32, seed=3)
    cam = f32_camera(room.trajectory(4, synthetic.REPLICA_LIKE, seed=7)[1])
    g = room.sample_gaussians(300_000, 16, seed=4, sem_mode="random")
    r, p = make(g, [cam], levels=3)
    r.forward(p)
    oc = oracle.level_cameras(cam, 3)[2]
    pix = np.stack([rng.integers(0, oc["W"], 8000), rng.integers(0, oc["H"], 8000)], 1)
    ref = ref_render(g, oc, pixels=pix)
    ok = unambiguous(ref["flags"])
    Tg = r.view_slice(r.T_final, 2, 1).cpu().numpy()[0, pix[:, 1], pix[:, 0]]
    relT = np.abs(Tg - ref["T"])[ok] / ref["T"][ok]
    print(f"float32 transmittance relative error: max {relT.max():.3e}, p99.9 {np.quantile(relT, 0.999):.3e} "
          f"over {ok.sum()} pixels, mean contributors {ref['n_contrib'].mean():.1f}")
    assert ref["n_contrib"].mean() > 20
    assert relT.max() <= T_TOL, relT.max()
