"""CPU checks of the kernels' float32 tile-culling rule (``kernel_rules``) against the FP64
definition of the set N per tile: the rule is conservative (keeps every tile a pixel of the
footprint reaches) and tight (keeps only tiles whose pixel-centre rectangle the footprint
reaches).  These are unit tests of a kernel rule, not pins of the oracle."""
import numpy as np

import oracle
from kernel_rules import records_f32, tile_reaches_alpha_min


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
    geo, ext, rects = records_f32(pr, cam, T)
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
        kept = tile_reaches_alpha_min(np.repeat(geo[r:r + 1], len(txs), 0), np.repeat(ext[r:r + 1], len(txs), 0),
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
    geo, ext, rects = records_f32(pr, cam, T)
    n_kept = 0
    for r in np.nonzero(rects[:, 2] > rects[:, 0])[0]:
        tx0, ty0, tx1, ty1 = rects[r]
        txs, tys = np.meshgrid(np.arange(tx0, tx1), np.arange(ty0, ty1))
        txs, tys = txs.ravel(), tys.ravel()
        X0, Y0 = txs * T, tys * T
        X1, Y1 = np.minimum(X0 + T - 1, cam["W"] - 1), np.minimum(Y0 + T - 1, cam["H"] - 1)
        kept = tile_reaches_alpha_min(np.repeat(geo[r:r + 1], len(txs), 0), np.repeat(ext[r:r + 1], len(txs), 0),
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


def test_half_mask_rule_is_conservative_and_splits_tile_rows():
    """The culling rule applied to each half of a tile row (the half masks of the tile lists):
    every half holding a pixel centre where the FP64 footprint reaches alpha >= 1/255 is
    marked (conservative); a sizeable share of kept tiles is marked for one half only (the
    masks are not vacuous); and the tiles kept by the hull of the two halves' runs are those
    the rule keeps on the whole row, up to float32 rounding at a run's ends."""
    import synthetic
    from kernel_rules import kept_and_masks, tile_halves_reach
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(800, 4, seed=11).items()}
    g["log_scale"][:, 0] += 1.0
    cam = synthetic.cloud_camera()
    T = 8
    pr = oracle.project(g, cam)
    geo, ext, rects = records_f32(pr, cam, T)
    P = oracle.P
    n_kept = n_single = n_diff = 0
    for r in np.nonzero(rects[:, 2] > rects[:, 0])[0]:
        tx0, ty0, tx1, ty1 = rects[r]
        txs, tys = np.meshgrid(np.arange(tx0, tx1), np.arange(ty0, ty1))
        txs, tys = txs.ravel(), tys.ravel()
        X0, Y0 = txs * T, tys * T
        X1, Y1 = np.minimum(X0 + T - 1, cam["W"] - 1), np.minimum(Y0 + T - 1, cam["H"] - 1)
        g_r, e_r = np.repeat(geo[r:r + 1], len(txs), 0), np.repeat(ext[r:r + 1], len(txs), 0)
        top, bottom = tile_halves_reach(g_r, e_r, X0, X1, Y0, Y1, T)
        keep, mask = kept_and_masks(np.full(len(txs), r), txs, tys, top, bottom)
        whole = tile_reaches_alpha_min(g_r, e_r, X0, X1, Y0, Y1)
        n_diff += int((keep != whole).sum())
        S = np.array([[pr[r, P["S00"]], pr[r, P["S01"]]], [pr[r, P["S01"]], pr[r, P["S11"]]]])
        Q = np.linalg.inv(S)
        for k in range(len(txs)):
            for h, (ya, yb) in enumerate(((Y0[k], min(Y0[k] + T // 2 - 1, Y1[k])), (Y0[k] + T // 2, Y1[k]))):
                if ya > yb:
                    continue
                xs, ys = np.meshgrid(np.arange(X0[k], X1[k] + 1) - pr[r, P["U"]], np.arange(ya, yb + 1) - pr[r, P["V"]])
                sig = 0.5 * (Q[0, 0] * xs * xs + 2 * Q[0, 1] * xs * ys + Q[1, 1] * ys * ys)
                if (pr[r, P["OPAC"]] * np.exp(-sig) >= (1 / 255) * (1 + 1e-5)).any():
                    assert keep[k] and (mask[k] >> h) & 1, (r, txs[k], tys[k], h)
        n_kept += int(keep.sum())
        n_single += int((keep & ((mask == 1) | (mask == 2))).sum())
    assert n_kept > 1000 and n_single > 0.1 * n_kept, (n_single, n_kept)
    assert n_diff <= 0.002 * n_kept, (n_diff, n_kept)


def test_kept_and_masks_matches_a_direct_loop():
    """kept_and_masks against a loop over (record, tile row) runs: the kept tiles are every
    tile between the leftmost and rightmost reached one, and each carries its halves' bits
    (3 on every tile of a run longer than 255 tiles)."""
    from kernel_rules import kept_and_masks
    rng = np.random.default_rng(3)
    n = 4000
    recs = rng.integers(0, 40, n)
    ty = rng.integers(0, 6, n)
    tx = rng.integers(0, 300, n)
    top = rng.random(n) < 0.3
    bottom = rng.random(n) < 0.3
    keep, mask = kept_and_masks(recs, tx, ty, top, bottom)
    for i in range(n):
        same = (recs == recs[i]) & (ty == ty[i])
        reached = tx[same & (top | bottom)]
        if len(reached) == 0:
            assert not keep[i]
            continue
        lo, hi = reached.min(), reached.max()
        assert keep[i] == (lo <= tx[i] <= hi)
        want = 3 if hi - lo + 1 > 255 else int(top[i]) | (int(bottom[i]) << 1)
        assert mask[i] == want
