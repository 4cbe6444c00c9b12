"""Pins of the oracle's hand-written adjoint (Sec. III-D backpropagation through Eq. 7-9
and Eq. 2-3) by FP64 central finite differences.

The method's skip (alpha < 1/255) and stop (T < 1e-4) rules make the rendered image a
discontinuous function of the parameters, so a finite step that moves one pixel across a
threshold produces a jump.  Two checks avoid that without weakening the adjoint check:
  * the whole-image gradient of every parameter with both thresholds switched off (the
    adjoint is the same code; only the branch decisions differ), including a Gaussian
    whose Jacobian clamp is active and one whose alpha clamps at 0.99;
  * per-pixel gradients with the default thresholds, skipping pixels whose contributor
    count changes between the two finite-difference evaluations.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic

KEYS = ["mean", "log_scale", "quat", "opacity_logit", "rgb", "sem"]


def tiny_scene(n=12, C=4, seed=5):
    rng = np.random.default_rng(seed)
    g = {k: np.asarray(v, np.float64)[:n].copy() for k, v in synthetic.cloud_scene(200, C, seed=seed).items()}
    g["mean"][:, 2] = rng.uniform(1.5, 2.5, n)
    g["mean"][:, :2] *= 0.3
    g["log_scale"] += 1.5
    # one Gaussian far to the side: its Jacobian clamp is active but its footprint is visible
    g["mean"][n - 1] = [2.6, 0.1, 2.0]
    g["log_scale"][n - 1] = np.log([0.3, 0.2, 0.25])
    # one Gaussian with alpha clamped at 0.99 around its centre
    g["opacity_logit"][3] = 6.0
    return g


def fd_check(g, cam, cfg, up, h=1e-5, n_check=None):
    def L(gg):
        r = oracle.render(gg, cam, cfg)
        return (up[0] * r["rgb"]).sum() + (up[1] * r["depth"]).sum() + (up[2] * r["sem"]).sum()
    an = oracle.render_backward(g, cam, *up, cfg=cfg)
    worst = {}
    for key in KEYS:
        arr = g[key]
        errs = []
        for ix in np.ndindex(arr.shape):
            gp = {k: v.copy() for k, v in g.items()}
            gm = {k: v.copy() for k, v in g.items()}
            gp[key][ix] += h
            gm[key][ix] -= h
            fd = (L(gp) - L(gm)) / (2 * h)
            errs.append(abs(fd - an[key][ix]) / (abs(fd) + 1e-3))
        worst[key] = max(errs)
    return worst


def test_adjoint_matches_fd_all_parameters():
    g = tiny_scene()
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24)
    cfg = dict(alpha_min=0.0, T_min=0.0)
    pr = oracle.project(g, cam, cfg)
    assert pr[-1, oracle.P["CLX"]] == 1           # the clamped-Jacobian branch is exercised
    rng = np.random.default_rng(0)
    up = (rng.normal(size=(3, 48, 64)), rng.normal(size=(48, 64)), rng.normal(size=(4, 48, 64)))
    worst = fd_check(g, cam, cfg, up)
    for key, w in worst.items():
        assert w < 2e-5, (key, w)


def test_adjoint_matches_fd_with_background_and_dilation_off():
    g = tiny_scene(seed=8)
    cam = synthetic.make_camera(48, 40, 50, 55, 23.5, 20.0)
    cfg = dict(alpha_min=0.0, T_min=0.0, bg=(0.3, 0.9, 0.1), dilation=0.0)
    rng = np.random.default_rng(1)
    up = (rng.normal(size=(3, 40, 48)), rng.normal(size=(40, 48)), rng.normal(size=(4, 40, 48)))
    worst = fd_check(g, cam, cfg, up)
    for key, w in worst.items():
        assert w < 2e-5, (key, w)


def rodrigues(axis, angle):
    """Rotation matrix of angle (rad) about axis (Rodrigues' formula)."""
    k = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


def test_adjoint_matches_fd_rotated_translated_camera():
    """A general camera pose (rotation about a skew axis, non-zero translation): the chain
    through t = R_cw mean + t_cw and through the view rotation in the EWA Jacobian is
    checked with a rotation that is not its own transpose."""
    g = tiny_scene(seed=13)
    R = rodrigues([0.3, 1.0, 0.2], 0.25)
    assert np.abs(R - R.T).max() > 0.1
    t = np.array([0.06, -0.04, 0.12])
    # keep the means in view: place them so that R mean + t is where tiny_scene put them
    g["mean"] = (g["mean"] - t) @ R
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24, R_cw=R, t_cw=t)
    cfg = dict(alpha_min=0.0, T_min=0.0)
    rng = np.random.default_rng(2)
    up = (rng.normal(size=(3, 48, 64)), rng.normal(size=(48, 64)), rng.normal(size=(4, 48, 64)))
    worst = fd_check(g, cam, cfg, up)
    for key, w in worst.items():
        assert w < 2e-5, (key, w)


def test_adjoint_matches_fd_jacobian_clamped_in_y():
    """The clamp branch of the Jacobian in y (a Gaussian below the image whose footprint
    still reaches it) next to the x one, with fx != fy and W != H."""
    g = tiny_scene(seed=17)
    # t_y / t_z = 0.71 > 1.3 (H/2) / fy = 0.39; its depth differs from the x-clamped one's
    # (2.0), so that no finite-difference step swaps the two in the depth order
    g["mean"][0] = [0.1, 1.5, 2.1]
    g["log_scale"][0] = np.log([0.25, 0.35, 0.3])
    cam = synthetic.make_camera(72, 40, 62, 66, 35.5, 19.5)
    cfg = dict(alpha_min=0.0, T_min=0.0)
    pr = oracle.project(g, cam, cfg)
    assert pr[0, oracle.P["CLY"]] == 1 and pr[0, oracle.P["CLX"]] == 0
    assert pr[-1, oracle.P["CLX"]] == 1
    rng = np.random.default_rng(3)
    up = (rng.normal(size=(3, 40, 72)), rng.normal(size=(40, 72)), rng.normal(size=(4, 40, 72)))
    worst = fd_check(g, cam, cfg, up)
    for key, w in worst.items():
        assert w < 2e-5, (key, w)


def test_adjoint_per_pixel_default_thresholds():
    """Default alpha_min = 1/255, T_min = 1e-4: per-pixel FD, excluding pixels whose branch
    decisions differ between the +h and -h evaluations."""
    g = tiny_scene(n=14, seed=11)
    rng = np.random.default_rng(4)
    g["mean"][:, :2] = rng.uniform(-0.12, 0.12, size=(14, 2))
    g["mean"][:, 2] = rng.uniform(1.5, 2.5, 14)
    g["log_scale"] = np.log(rng.uniform(0.08, 0.2, size=(14, 3)))
    g["opacity_logit"][:] = 3.0                    # dense, so the stop rule triggers
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24)
    pix = np.stack([rng.integers(16, 48, 150), rng.integers(12, 36, 150)], 1)
    base = oracle.render(g, cam, pixels=pix)
    assert (base["T"] < 0.01).any()
    h = 1e-6
    checked = 0
    for k in rng.choice(len(pix), 25, replace=False):
        if base["n_contrib"][k] == 0:
            continue
        p = pix[k:k + 1]
        gu = rng.normal(size=(3, 1)); gd = rng.normal(size=1); gs = rng.normal(size=(4, 1))
        an = oracle.render_backward(g, cam, gu, gd, gs, pixels=p)
        for key in ("mean", "log_scale", "quat", "opacity_logit"):
            for i in range(g[key].shape[0]):
                for c in range(g[key].shape[1] if g[key].ndim > 1 else 1):
                    ix = (i, c) if g[key].ndim > 1 else (i,)
                    gp = {kk: v.copy() for kk, v in g.items()}
                    gm = {kk: v.copy() for kk, v in g.items()}
                    gp[key][ix] += h
                    gm[key][ix] -= h
                    rp = oracle.render(gp, cam, pixels=p)
                    rm = oracle.render(gm, cam, pixels=p)
                    if rp["n_contrib"][0] != rm["n_contrib"][0]:
                        continue
                    Lp = (gu[:, 0] * rp["rgb"][:, 0]).sum() + gd[0] * rp["depth"][0] + (gs[:, 0] * rp["sem"][:, 0]).sum()
                    Lm = (gu[:, 0] * rm["rgb"][:, 0]).sum() + gd[0] * rm["depth"][0] + (gs[:, 0] * rm["sem"][:, 0]).sum()
                    fd = (Lp - Lm) / (2 * h)
                    assert fd == pytest.approx(an[key][ix], rel=1e-4, abs=1e-6), (key, ix, k)
                    checked += 1
    assert checked > 200


def test_clamped_alpha_has_zero_opacity_gradient():
    """At a pixel where o*G >= 0.99 the clamp is active: d alpha / d opacity = 0."""
    s = np.log([0.05] * 3)
    g = dict(mean=np.array([[0, 0, 2.0]]), log_scale=np.array([s]), quat=np.array([[1.0, 0, 0, 0]]),
             opacity_logit=np.array([8.0]), rgb=np.array([[1.0, 1, 1]]), sem=np.array([[1.0, 1.0]]))
    cam = synthetic.cloud_camera()
    an = oracle.render_backward(g, cam, np.ones((3, 1)), np.zeros(1), np.zeros((2, 1)), pixels=[[80, 60]])
    assert an["opacity_logit"][0] == 0.0
    assert np.all(an["mean"] == 0.0)
    assert an["rgb"][0] == pytest.approx([0.99] * 3)


def test_adjoint_matches_fd_eq2_isotropic_mode():
    """The Eq. 2 projection's adjoint: gradients reach the mean, log_scale[0], opacity and
    the features; the rotation and the other log-scales get exactly zero (FD agrees)."""
    g = tiny_scene(seed=11)
    cam = synthetic.make_camera(56, 44, 58, 52, 27.5, 21.5)
    cfg = dict(alpha_min=0.0, T_min=0.0, isotropic=1)
    rng = np.random.default_rng(4)
    up = (rng.normal(size=(3, 44, 56)), rng.normal(size=(44, 56)), rng.normal(size=(4, 44, 56)))
    worst = fd_check(g, cam, cfg, up)
    for key, w in worst.items():
        assert w < 2e-5, (key, w)
    an = oracle.render_backward(g, cam, *up, cfg=cfg)
    assert not an["quat"].any() and not an["log_scale"][:, 1:].any()
    assert np.abs(an["log_scale"][:, 0]).max() > 0
