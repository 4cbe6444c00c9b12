"""Pins of the oracle's insertion step (oracle/init.py) to facts that do not restate it: the
back-projected mean projects back onto its pixel at its depth, the heuristic scale has a
one-pixel Eq. 2 footprint, the patch rows carry the pixel's own values at the centre, unit
rays through the neighbours' pixel centres, zeros outside the image and beyond 2009
features, and standardising a target then applying the outputs gives the target back."""
import math

import numpy as np
import pytest

import synthetic
from oracle import init as oi


def _frame(seed=0, W=12, H=9, K=32):
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(size=(3, H, W))
    depth = rng.uniform(0.5, 4.0, size=(H, W))
    depth[rng.uniform(size=(H, W)) < 0.2] = 0.0
    label = rng.integers(-1, K + 3, size=(H, W))   # some labels outside [0, 32)
    a = 0.4
    R = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]]) @ \
        np.array([[1, 0, 0], [0, math.cos(0.2), -math.sin(0.2)], [0, math.sin(0.2), math.cos(0.2)]])
    cam = synthetic.make_camera(W, H, 10.0, 11.5, 5.5, 4.0, R_cw=R, t_cw=[0.3, -0.1, 0.7])
    return rgb, depth, label, cam


def test_heuristic_mean_projects_back_onto_its_pixel():
    rgb, depth, label, cam = _frame()
    ys, xs = np.nonzero(depth > 0)
    pix = np.stack([xs, ys], 1)
    g = oi.heuristic_init(rgb, depth, label, cam, pix)
    R, t = np.asarray(cam["R_cw"]), np.asarray(cam["t_cw"])
    pc = g["mean"] @ R.T + t                      # camera-frame points
    np.testing.assert_allclose(pc[:, 2], depth[ys, xs], rtol=1e-13)
    np.testing.assert_allclose(cam["fx"] * pc[:, 0] / pc[:, 2] + cam["cx"], xs, atol=1e-12)
    np.testing.assert_allclose(cam["fy"] * pc[:, 1] / pc[:, 2] + cam["cy"], ys, atol=1e-12)
    # Eq. 2: an isotropic Gaussian of radius r at depth d spans f r / d pixels -- one pixel here
    np.testing.assert_allclose(cam["fx"] * np.exp(g["log_scale"]) / depth[ys, xs][:, None], 1.0, rtol=1e-13)
    assert np.array_equal(g["quat"], np.tile([1.0, 0, 0, 0], (len(xs), 1)))
    assert not g["opacity_logit"].any()
    np.testing.assert_array_equal(g["rgb"], rgb[:, ys, xs].T)


def test_heuristic_semantic_feature_is_the_scaled_code_row():
    rgb, depth, label, cam = _frame(seed=1)
    code = np.random.default_rng(2).normal(size=(32, 16))
    ys, xs = np.nonzero(depth > 0)
    g = oi.heuristic_init(rgb, depth, label, cam, np.stack([xs, ys], 1), code=code, kappa=2.5)
    for i, (x, y) in enumerate(zip(xs, ys)):
        lab = label[y, x]
        want = 2.5 * code[lab] if 0 <= lab < 32 else np.zeros(16)
        np.testing.assert_array_equal(g["sem"][i], want)


def test_patch_row_layout():
    rgb, depth, label, cam = _frame(seed=3)
    pix = np.array([[0, 0], [6, 4], [11, 8], [3, 7]])
    X = oi.patch_features(rgb, depth, label, cam, pix)
    assert X.shape == (4, 2048) and not X[:, 2009:].any()
    for b, (x0, y0) in enumerate(pix):
        rows = X[b, :2009].reshape(49, 41)
        for n in range(49):
            x, y = x0 + n % 7 - 3, y0 + n // 7 - 3
            f = rows[n]
            if not (0 <= x < 12 and 0 <= y < 9):
                assert not f.any(), (b, n)
                continue
            assert np.array_equal(f[0:3], rgb[:, y, x])
            d = depth[y, x]
            assert f[3] == (d if d > 0 else 0.0) and f[39] == (1.0 if d > 0 else 0.0)
            onehot = f[4:36]
            assert onehot.sum() == (1.0 if 0 <= label[y, x] < 32 else 0.0)
            if 0 <= label[y, x] < 32:
                assert onehot[label[y, x]] == 1.0
            # the unit ray through the neighbour's pixel centre: projects onto (x, y)
            ray = f[36:39]
            assert np.linalg.norm(ray) == pytest.approx(1.0, abs=1e-14) and ray[2] > 0
            assert cam["fx"] * ray[0] / ray[2] + cam["cx"] == pytest.approx(x, abs=1e-12)
            assert cam["fy"] * ray[1] / ray[2] + cam["cy"] == pytest.approx(y, abs=1e-12)
            assert f[40] == pytest.approx(1 / cam["fx"], rel=1e-15)
        # the centre neighbour (dx = dy = 0) is the pixel itself
        assert np.array_equal(rows[24, 0:3], rgb[:, y0, x0])


def test_standardised_outputs_round_trip():
    rng = np.random.default_rng(4)
    B, C = 50, 16
    mu = rng.normal(size=32)
    sd = rng.uniform(0.1, 2.0, size=32)
    tgt = rng.normal(size=(B, 32)) * sd + mu
    Y = (tgt - mu) / sd
    out = oi.apply_mlp_init(Y, mu, sd, C)
    np.testing.assert_allclose(out["log_scale"], tgt[:, 0:3], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["opacity_logit"], tgt[:, 3], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["sem"], tgt[:, 4:20], rtol=1e-12, atol=1e-12)
