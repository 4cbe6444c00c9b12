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
    # ranges
    for t in range(total):
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t)
        assert (e - s) == np.sum(tiles == t)
