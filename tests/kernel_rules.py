"""The tile-list kernels' own float32 culling rule, restated for kernel unit tests.

NOT the oracle.  Which tiles a Gaussian is listed in is not fixed by the paper: any superset
of the tiles holding a pixel where its alpha reaches alpha_min gives the same images (Eq.
7-9).  The oracle defines that set in FP64 (``oracle.tile_reach``) and the primary tile-list
parity tests compare the kernels with it.  The kernels list a conservative superset chosen
by a float32 rule; this module repeats that rule step by step so that a unit test can check
the sort and emission kernels bit for bit on the kernels' own float32 records.  Its CPU
tests (``test_kernel_rules.py``) check the rule against the FP64 definition in both
directions.
"""
import numpy as np

import oracle


def tile_reaches_alpha_min(geo, ext, X0, X1, Y0, Y1):
    """Float32 tile culling rule of the tile lists, for arrays of (record, tile) pairs.

    geo: (n, 8) float32 records (u_frac, v_frac, depth, opacity, m00, m10, m11, packed
    int16 (u_int, v_int)); ext: (n, 2) float32 half extents; X0..X1, Y0..Y1: the tile's
    pixel-centre rectangle (int).  The record's alpha >= alpha_min region is the ellipse
    sigma = (m00 dx)^2 + (m10 dx + m11 dy)^2 <= thr, and the projection wrote
    ex = sqrt(2 thr s00) 1.002 + 0.01 with m00 = 1 / sqrt(2 s00), so
    thr' = ((ex - 0.01) (1 / 1.002) m00)^2.  Within the band dy in [y0, y1] of the tile's row
    the ellipse spans dx in [xl, xr]: with A = m00^2 + m10^2, B = m10 m11, C = m11^2 and
    p = m00 m11 (A C - B^2 = p^2), the band is cut to |dy| <= sqrt(A thr') / p, the right
    edge (s(dy) - B dy) / A with s = sqrt(A thr' - (p dy)^2) is largest at
    dy = -B (sqrt(thr' C) / p) / C and the left edge (-B dy - s) / A smallest at the opposite
    dy, each clamped to the band.  The tile is kept when its pixel-centre columns meet
    [xl, xr]: ((X1 - u_int) - u_frac) >= xl and ((X0 - u_int) - u_frac) <= xr.  Every step is
    one correctly rounded float32 operation (square roots and divisions included) in a fixed
    order, so the decision is reproducible bit for bit from the same float32 records; the
    kept tiles of a tile row are contiguous.  Returns a bool array.
    """
    f = np.float32
    geo = np.asarray(geo, np.float32)
    ext = np.asarray(ext, np.float32)
    packed = geo[:, 7].view(np.uint32)
    ui = (packed & 0xFFFF).astype(np.uint16).view(np.int16).astype(np.int64)
    vi = (packed >> 16).astype(np.uint16).view(np.int16).astype(np.int64)
    uf, vf = geo[:, 0], geo[:, 1]
    X0, X1 = np.asarray(X0, np.int64), np.asarray(X1, np.int64)
    Y0, Y1 = np.asarray(Y0, np.int64), np.asarray(Y1, np.int64)
    m00, m10, m11 = geo[:, 4], geo[:, 5], geo[:, 6]
    with np.errstate(all="ignore"):
        t = ((ext[:, 0] - f(0.01)) * f(1.0 / 1.002)) * m00
        thr = t * t
        A = m00 * m00 + m10 * m10
        B = m10 * m11
        Cq = m11 * m11
        p = m00 * m11
        y0 = (Y0 - vi).astype(np.float32) - vf
        y1 = (Y1 - vi).astype(np.float32) - vf
        dymax = np.sqrt(A * thr) / p
        yb0 = np.fmax(y0, -dymax)
        yb1 = np.fmin(y1, dymax)
        dxmax = np.sqrt(thr * Cq) / p
        dyr = -((B * dxmax) / Cq)

        def s_of(dy):
            q = p * dy
            return np.sqrt(np.fmax(A * thr - q * q, f(0)))

        dr = np.fmin(yb1, np.fmax(yb0, dyr))
        dl = np.fmin(yb1, np.fmax(yb0, -dyr))
        xr = (s_of(dr) - B * dr) / A
        xl = (-(B * dl) - s_of(dl)) / A
        keep = (yb0 <= yb1) & (((X1 - ui).astype(np.float32) - uf) >= xl) & (((X0 - ui).astype(np.float32) - uf) <= xr)
    return keep


def records_f32(pr, cam, T):
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


def tile_halves_reach(geo, ext, X0, X1, Y0, Y1, tile_h):
    """The kernels' rule applied to the two halves of each tile: the pixel-centre rows
    [Y0, Y0 + tile_h / 2) and [Y0 + tile_h / 2, Y1] (the second empty when the image ends
    first).  Returns (top, bottom) bool arrays."""
    Y0, Y1 = np.asarray(Y0, np.int64), np.asarray(Y1, np.int64)
    Yh = Y0 + tile_h // 2
    top = tile_reaches_alpha_min(geo, ext, X0, X1, Y0, np.minimum(Yh - 1, Y1))
    has_bottom = Yh <= Y1
    bottom = has_bottom & tile_reaches_alpha_min(geo, ext, X0, X1, np.minimum(Yh, Y1), Y1)
    return top, bottom


def kept_and_masks(recs, tx, ty, top, bottom):
    """Per (record, tile row) the kernels keep the hull of the tiles either half reaches
    (the two halves' runs overlap for one convex footprint, so this is their union) and mark
    each kept tile's halves: top | bottom << 1, or 3 on every tile of a run longer than 255
    tiles.  Returns (keep, mask) over the given (record, tile) pairs."""
    recs, tx, ty = (np.asarray(a, np.int64) for a in (recs, tx, ty))
    reach = np.asarray(top, bool) | np.asarray(bottom, bool)
    key = recs * (1 << 20) + ty
    groups, inv = np.unique(key, return_inverse=True)
    lo = np.full(len(groups), np.iinfo(np.int64).max)
    hi = np.full(len(groups), np.iinfo(np.int64).min)
    np.minimum.at(lo, inv[reach], tx[reach])
    np.maximum.at(hi, inv[reach], tx[reach])
    keep = (tx >= lo[inv]) & (tx <= hi[inv])
    mask = np.asarray(top, np.int64) | (np.asarray(bottom, np.int64) << 1)
    mask = np.where(hi[inv] - lo[inv] + 1 > 255, 3, mask)
    return keep, mask
