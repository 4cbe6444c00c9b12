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


def _alpha_axis_aligned(cam, mean, s, o, px, py, b=0.3):
    """alpha of an axis-aligned Gaussian seen by a camera with identity pose, from the
    closed-form Sigma2D = J diag(exp(2 s)) J^T + b I (matrix inverse by numpy)."""
    z = mean[2]
    u, v = cam["fx"] * mean[0] / z + cam["cx"], cam["fy"] * mean[1] / z + cam["cy"]
    J = np.array([[cam["fx"] / z, 0, -cam["fx"] * mean[0] / z ** 2], [0, cam["fy"] / z, -cam["fy"] * mean[1] / z ** 2]])
    Q = np.linalg.inv(J @ np.diag(np.exp(2 * np.asarray(s))) @ J.T + b * np.eye(2))
    d = np.stack([np.asarray(px, float) - u, np.asarray(py, float) - v])
    return o * np.exp(-0.5 * np.einsum("in,ij,jn->n", d, Q, d))


def _axis_aligned_scene(n=60, seed=12):
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.45, 0.45, n), rng.uniform(1.5, 3.0, n)], 1)
    s = np.log(rng.uniform(0.01, 0.08, (n, 3)))
    logit = rng.normal(0.5, 1.0, n)
    g = dict(mean=mean, log_scale=s, quat=np.tile([1.0, 0, 0, 0], (n, 1)), opacity_logit=logit,
             rgb=np.ones((n, 3)), sem=np.zeros((n, 4)))
    return g, 1 / (1 + np.exp(-logit))


@pytest.mark.parametrize("T", [(8, 8), (16, 16), (32, 8)])
def test_tile_membership_matches_closed_form_alpha(T):
    """The set N of a tile holds a Gaussian iff its alpha reaches 1/255 at one of the tile's
    pixel centres: tile_pairs covers every tile with such a pixel, and tile_reach's largest
    alpha over each tile equals the closed-form alpha maximised over that tile's pixels."""
    tw, th = T
    cam = synthetic.cloud_camera()
    g, o = _axis_aligned_scene()
    pr = oracle.project(g, cam)
    gs, tx, ty = oracle.tile_pairs(pr, cam, tw, th)
    listed = set(zip(gs.tolist(), tx.tolist(), ty.tolist()))
    reach = oracle.tile_reach(pr, cam, gs, tx, ty, tw, th)
    ys, xs = np.mgrid[0:cam["H"], 0:cam["W"]]
    n_in = 0
    for i in range(len(o)):
        a = _alpha_axis_aligned(cam, g["mean"][i], g["log_scale"][i], o[i], xs.ravel(), ys.ravel())
        hit = a >= 1 / 255
        for x, y in zip(xs.ravel()[hit], ys.ravel()[hit]):
            assert (i, x // tw, y // th) in listed, (i, x, y)
        sel = np.nonzero(gs == i)[0]
        for k in sel:
            m = (xs.ravel() // tw == tx[k]) & (ys.ravel() // th == ty[k])
            assert reach["alpha"][k] == pytest.approx(a[m].max(), rel=1e-9, abs=1e-15)
            n_in += bool(a[m].max() >= 1 / 255)
        assert np.all(reach["thr"][sel] == pytest.approx(np.log(o[i] * 255.0), rel=1e-12))
    assert n_in > 100 and len(gs) > n_in  # the rectangles over-cover: some listed tiles are missed


def test_tile_reach_sigma_min_is_the_minimum_over_the_pixel_centre_rectangle():
    """sigma_min against a dense sampling of the tile's continuous pixel-centre rectangle (an
    upper bound, approached within the grid spacing) for rotated, elongated footprints, and 0
    on the tile holding the 2D mean."""
    cam = synthetic.cloud_camera()
    rng = np.random.default_rng(3)
    n = 12
    q = rng.normal(size=(n, 4))
    g = dict(mean=np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1.5, 3, n)], 1),
             log_scale=np.log(np.stack([rng.uniform(0.05, 0.15, n), rng.uniform(0.005, 0.01, n),
                                        rng.uniform(0.005, 0.01, n)], 1)),
             quat=q / np.linalg.norm(q, axis=1, keepdims=True), opacity_logit=np.full(n, 2.0),
             rgb=np.ones((n, 3)), sem=np.zeros((n, 4)))
    pr = oracle.project(g, cam)
    P = oracle.P
    tw = th = 8
    gs, tx, ty = oracle.tile_pairs(pr, cam, tw, th)
    reach = oracle.tile_reach(pr, cam, gs, tx, ty, tw, th)
    fine = np.linspace(0, 1, 161)
    for k in range(0, len(gs), 7):
        i = gs[k]
        X0, Y0 = tx[k] * tw, ty[k] * th
        X1, Y1 = min(X0 + tw - 1, cam["W"] - 1), min(Y0 + th - 1, cam["H"] - 1)
        xs, ys = np.meshgrid(X0 + fine * (X1 - X0), Y0 + fine * (Y1 - Y0))
        dx, dy = xs - pr[i, P["U"]], ys - pr[i, P["V"]]
        sig = 0.5 * (pr[i, P["CA"]] * dx * dx + pr[i, P["CC"]] * dy * dy) + pr[i, P["CB"]] * dx * dy
        smin = reach["sigma_min"][k]
        assert smin <= sig.min() * (1 + 1e-12) + 1e-12
        assert smin >= sig.min() - 0.02 * (1 + sig.min())
        holds = X0 <= pr[i, P["U"]] <= X1 and Y0 <= pr[i, P["V"]] <= Y1
        assert (smin == 0.0) == holds
