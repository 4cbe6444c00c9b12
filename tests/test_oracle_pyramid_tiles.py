"""Pins of the oracle's pyramid (Eq. 4-6) and of its integer tile-list reference."""
import numpy as np
import pytest

import oracle
import synthetic


def test_level_cameras_keep_pixel_centres_consistent():
    """A level-(l+1) pixel is the box mean of level-l pixels 2x, 2x+1.  Downsampling the
    level-0 'x coordinate' image must therefore give, at the level-1 projection of any
    3D point, the level-0 projection of that point."""
    cam = synthetic.make_camera(64, 48, 70.0, 65.0, 31.5, 23.5)
    cams = oracle.level_cameras(cam, 3)
    H, W = 48, 64
    X = np.broadcast_to(np.arange(W, dtype=float)[None, None], (3, H, W)).copy()
    Y = np.broadcast_to(np.arange(H, dtype=float)[None, :, None], (3, H, W)).copy()
    pyr_x = oracle.build_pyramid(X, np.ones((H, W)), np.zeros((H, W), np.int32), 3)
    pyr_y = oracle.build_pyramid(Y, np.ones((H, W)), np.zeros((H, W), np.int32), 3)
    rng = np.random.default_rng(0)
    for _ in range(20):
        p = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(1, 3)])
        u0 = cam["fx"] * p[0] / p[2] + cam["cx"]
        v0 = cam["fy"] * p[1] / p[2] + cam["cy"]
        for l in (1, 2):
            c = cams[l]
            ul = c["fx"] * p[0] / p[2] + c["cx"]
            vl = c["fy"] * p[1] / p[2] + c["cy"]
            xi, yi = int(np.floor(ul)), int(np.floor(vl))
            if not (0 <= xi < c["W"] - 1 and 0 <= yi < c["H"] - 1):
                continue
            # the pyramid coordinate images are affine in the pixel index: interpolate
            xs = pyr_x[l][0][0]
            ys = pyr_y[l][0][0]
            interp_u = xs[yi, xi] + (ul - xi) * (xs[yi, xi + 1] - xs[yi, xi])
            interp_v = ys[yi, xi] + (vl - yi) * (ys[yi + 1, xi] - ys[yi, xi])
            assert interp_u == pytest.approx(u0, abs=1e-9)
            assert interp_v == pytest.approx(v0, abs=1e-9)
    assert [c["W"] for c in cams] == [64, 32, 16] and [c["H"] for c in cams] == [48, 24, 12]


def test_level_camera_sizes_match_the_downsampled_images_for_odd_sizes():
    """157 x 91 -> 78 x 45 -> 39 x 22 (floor at every level, worked by hand), and every
    level's camera has exactly the size of its image in the target pyramid."""
    cam = synthetic.make_camera(157, 91, 140.0, 140.0, 77.7, 44.6)
    cams = oracle.level_cameras(cam, 3)
    assert [(c["W"], c["H"]) for c in cams] == [(157, 91), (78, 45), (39, 22)]
    pyr = oracle.build_pyramid(np.zeros((3, 91, 157)), np.ones((91, 157)), np.zeros((91, 157), np.int32), 3)
    for c, (rgb, depth, label) in zip(cams, pyr):
        assert rgb.shape == (3, c["H"], c["W"]) and depth.shape == label.shape == (c["H"], c["W"])


def test_downsample_rules():
    rgb = np.arange(3 * 4 * 6, dtype=float).reshape(3, 4, 6)
    depth = np.array([[1, 0, 2, 2, 0, 0], [3, 0, 2, 2, 0, 0], [0, 0, 1, 5, 4, 4], [0, 0, 1, 1, 4, 4]], float)
    label = np.array([[1, 2, 3, 3, -1, -1], [2, 1, 3, 4, -1, -1], [0, 0, 7, 7, 2, 2], [9, 9, 6, 6, 3, 1]])
    r2, d2, l2 = oracle.downsample(rgb, depth, label)
    assert r2.shape == (3, 2, 3)
    assert r2[0, 0, 0] == pytest.approx((0 + 1 + 6 + 7) / 4)
    assert np.allclose(d2, [[2.0, 2.0, 0.0], [0.0, 2.0, 4.0]])
    # ties break to the lowest id; -1 entries are ignored; all -1 stays -1
    assert l2.tolist() == [[1, 3, -1], [0, 6, 2]]
    # odd sizes floor
    r3, d3, l3 = oracle.downsample(np.zeros((3, 5, 7)), np.zeros((5, 7)), np.zeros((5, 7), int))
    assert r3.shape == (3, 2, 3) and d3.shape == (2, 3)


def test_tile_lists_reference_brute_force():
    """Tiny example: each record's instances are exactly the tiles of its rectangle,
    instances are sorted by (tile, depth, record) and ranges delimit each tile."""
    rng = np.random.default_rng(0)
    n_per_view, V = 30, 2
    tiles_x, tiles_y = [5, 3], [4, 2]
    off = [0, 20]
    total = 26
    rects, depth = [], []
    for v in range(V):
        for _ in range(n_per_view):
            x0 = rng.integers(0, tiles_x[v]); x1 = rng.integers(x0, tiles_x[v] + 1)
            y0 = rng.integers(0, tiles_y[v]); y1 = rng.integers(y0, tiles_y[v] + 1)
            rects.append([x0, y0, x1, y1])
            depth.append(rng.choice([1.5, 2.0, 2.0, 3.25]) if rng.uniform() < 0.5 else rng.uniform(0.5, 5))
    rects = np.array(rects)
    depth = np.array(depth, np.float32)
    tiles, recs, ranges = oracle.tile_lists(rects, depth, tiles_x, off, total, n_per_view)
    # membership
    expect = set()
    for r, (x0, y0, x1, y1) in enumerate(rects):
        v = r // n_per_view
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                expect.add((off[v] + ty * tiles_x[v] + tx, r))
    assert set(zip(tiles.tolist(), recs.tolist())) == expect and len(tiles) == len(expect)
    # order
    keys = [(t, float(depth[r]), r) for t, r in zip(tiles, recs)]
    assert keys == sorted(keys)
    # ranges; a tile without instances has the range (0, 0) (the format of the lists' ranges)
    for t in range(total):
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t)
        assert (e - s) == np.sum(tiles == t)
        if e == s:
            assert s == 0, (t, s)


def test_tile_lists_empty_tiles_have_range_zero():
    """A 4 x 1 grid where tiles 1 and 3 hold nothing: their ranges are (0, 0), the others
    [start, end) of their instances."""
    rects = np.array([[0, 0, 1, 1], [2, 0, 3, 1], [0, 0, 1, 1]])
    depth = np.array([2.0, 1.0, 1.0], np.float32)
    tiles, recs, ranges = oracle.tile_lists(rects, depth, [4], [0], 4, 3)
    assert tiles.tolist() == [0, 0, 2] and recs.tolist() == [2, 0, 1]
    assert ranges.tolist() == [[0, 2], [0, 0], [2, 3], [0, 0]]


def _records_f32(pr, cam, T):
    """Float32 records (u_frac, v_frac, depth, opacity, m00, m10, m11, packed int16 mean),
    half extents and tile rectangles in the projection's format, from the FP64 projection."""
    P = oracle.P
    v = pr[:, P["VALID"]] > 0
    u, vv = pr[:, P["U"]], pr[:, P["V"]]
    s00, s01, s11 = pr[:, P["S00"]], pr[:, P["S01"]], pr[:, P["S11"]]
    o = pr[:, P["OPAC"]]
    det = s00 * s11 - s01 * s01
    with np.errstate(all="ignore"):
        thr = np.log(o * 255.0) + 1e-3
        ex = np.sqrt(2 * thr * s00) * 1.002 + 0.01
        ey = np.sqrt(2 * thr * s11) * 1.002 + 0.01
        ui, vi = np.rint(u), np.rint(vv)
        geo = np.zeros((len(u), 8), np.float32)
        geo[:, 0], geo[:, 1], geo[:, 2], geo[:, 3] = u - ui, vv - vi, pr[:, P["TZ"]], o
        geo[:, 4] = 1 / np.sqrt(2 * s00)
        geo[:, 5] = -s01 / np.sqrt(2 * s00 * det)
        geo[:, 6] = np.sqrt(s00 / (2 * det))
        packed = (ui.astype(np.int64) & 0xFFFF) | ((vi.astype(np.int64) & 0xFFFF) << 16)
        geo[:, 7] = packed.astype(np.uint32).view(np.float32)
        x0 = np.maximum(np.ceil(u - ex), 0); x1 = np.minimum(np.floor(u + ex), cam["W"] - 1)
        y0 = np.maximum(np.ceil(vv - ey), 0); y1 = np.minimum(np.floor(vv + ey), cam["H"] - 1)
    ok = v & (x0 <= x1) & (y0 <= y1)
    rects = np.zeros((len(u), 4), np.int64)
    rects[ok] = np.stack([x0[ok] // T, y0[ok] // T, x1[ok] // T + 1, y1[ok] // T + 1], 1)
    return geo, np.stack([ex, ey], 1).astype(np.float32), rects


def test_tile_culling_rule_keeps_every_tile_a_pixel_reaches():
    """The float32 culling rule is conservative: every tile holding a pixel centre where the
    Gaussian (FP64, from the oracle's projection) reaches alpha >= 1/255 is kept; and it is
    not vacuous: it drops a sizeable share of the rectangle tiles (elongated footprints)."""
    import synthetic
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(800, 4, seed=9).items()}
    g["log_scale"][:, 0] += 1.0       # elongated, so that rectangles over-cover
    cam = synthetic.cloud_camera()
    T = 8
    pr = oracle.project(g, cam)
    geo, ext, rects = _records_f32(pr, cam, T)
    P = oracle.P
    n_tiles = n_kept = 0
    for r in np.nonzero(rects[:, 2] > rects[:, 0])[0]:
        tx0, ty0, tx1, ty1 = rects[r]
        S = np.array([[pr[r, P["S00"]], pr[r, P["S01"]]], [pr[r, P["S01"]], pr[r, P["S11"]]]])
        Q = np.linalg.inv(S)
        txs, tys = np.meshgrid(np.arange(tx0, tx1), np.arange(ty0, ty1))
        txs, tys = txs.ravel(), tys.ravel()
        X0, Y0 = txs * T, tys * T
        X1, Y1 = np.minimum(X0 + T - 1, cam["W"] - 1), np.minimum(Y0 + T - 1, cam["H"] - 1)
        kept = oracle.tile_reaches_alpha_min(np.repeat(geo[r:r + 1], len(txs), 0), np.repeat(ext[r:r + 1], len(txs), 0),
                                             X0, X1, Y0, Y1)
        for k in range(len(txs)):
            xs, ys = np.meshgrid(np.arange(X0[k], X1[k] + 1) - pr[r, P["U"]], np.arange(Y0[k], Y1[k] + 1) - pr[r, P["V"]])
            sig = 0.5 * (Q[0, 0] * xs * xs + 2 * Q[0, 1] * xs * ys + Q[1, 1] * ys * ys)
            reaches = (pr[r, P["OPAC"]] * np.exp(-sig) >= 1 / 255).any()
            assert kept[k] or not reaches, (r, txs[k], tys[k])
        n_tiles += len(txs)
        n_kept += int(kept.sum())
    assert n_tiles > 2000 and n_kept < 0.9 * n_tiles, (n_kept, n_tiles)


def _min_quadratic_over_rect(A, B, C, x0, x1, y0, y1):
    """min of A x^2 + 2 B x y + C y^2 (positive definite) over [x0, x1] x [y0, y1], FP64:
    0 if the rectangle holds the origin, else the least of the four edges' clamped 1-D minima."""
    if x0 <= 0 <= x1 and y0 <= 0 <= y1:
        return 0.0
    q = lambda x, y: A * x * x + 2 * B * x * y + C * y * y
    best = np.inf
    for x in (x0, x1):
        best = min(best, q(x, min(y1, max(y0, -B * x / C))))
    for y in (y0, y1):
        best = min(best, q(min(x1, max(x0, -B * y / A)), y))
    return best


def test_tile_culling_rule_keeps_only_tiles_the_footprint_reaches():
    """The other direction of the rule: a kept tile's pixel-centre rectangle meets the
    footprint sigma <= thr' (thr' recovered from the stored extent), evaluated in FP64 from
    the same float32 records, up to float32 rounding -- so the rule drops the tiles of a
    rectangle row that the ellipse's vertical extent misses, and every tile left or right of
    its span."""
    import synthetic
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(500, 4, seed=10).items()}
    g["log_scale"][:, 0] += 1.0
    cam = synthetic.cloud_camera()
    T = 8
    pr = oracle.project(g, cam)
    geo, ext, rects = _records_f32(pr, cam, T)
    n_kept = 0
    for r in np.nonzero(rects[:, 2] > rects[:, 0])[0]:
        tx0, ty0, tx1, ty1 = rects[r]
        txs, tys = np.meshgrid(np.arange(tx0, tx1), np.arange(ty0, ty1))
        txs, tys = txs.ravel(), tys.ravel()
        X0, Y0 = txs * T, tys * T
        X1, Y1 = np.minimum(X0 + T - 1, cam["W"] - 1), np.minimum(Y0 + T - 1, cam["H"] - 1)
        kept = oracle.tile_reaches_alpha_min(np.repeat(geo[r:r + 1], len(txs), 0), np.repeat(ext[r:r + 1], len(txs), 0),
                                             X0, X1, Y0, Y1)
        uf, vf, m00, m10, m11 = (float(v) for v in geo[r, [0, 1, 4, 5, 6]])
        packed = int(geo[r:r + 1, 7].view(np.uint32)[0])
        ui = float(np.int16(np.uint16(packed & 0xFFFF)))
        vi = float(np.int16(np.uint16(packed >> 16)))
        thr = ((float(ext[r, 0]) - 0.01) / 1.002 * m00) ** 2
        A, B, C = m00 * m00 + m10 * m10, m10 * m11, m11 * m11
        for k in np.nonzero(kept)[0]:
            smin = _min_quadratic_over_rect(A, B, C, X0[k] - ui - uf, X1[k] - ui - uf, Y0[k] - vi - vf, Y1[k] - vi - vf)
            assert smin <= thr * (1 + 1e-4) + 1e-4, (r, txs[k], tys[k], smin, thr)
            n_kept += 1
    assert n_kept > 1000


def test_tile_lists_with_culling_lists_only_kept_pairs():
    """With a keep rule the reference lists exactly the kept (record, tile) pairs, in the
    same (tile, depth, record) order."""
    rects = np.array([[0, 0, 3, 2], [1, 0, 2, 2], [0, 1, 3, 2]])
    depth = np.array([2.0, 1.0, 3.0], np.float32)
    keep = lambda recs, tx, ty: (tx + ty + recs) % 2 == 0
    tiles, recs, ranges = oracle.tile_lists(rects, depth, [3], [0], 6, 3, keep=keep)
    full_t, full_r, _ = oracle.tile_lists(rects, depth, [3], [0], 6, 3)
    sel = [(t, r) for t, r in zip(full_t, full_r) if ((t % 3) + (t // 3) + r) % 2 == 0]
    assert list(zip(tiles.tolist(), recs.tolist())) == sel
    for t in range(6):
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t) and (e - s) == np.sum(tiles == t)
