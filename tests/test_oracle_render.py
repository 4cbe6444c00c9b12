"""Pins of the oracle's compositing (Eq. 7-9): closed forms for one and two Gaussians,
the textbook "over" operator, transmittance/weight invariants and the stop rule."""
import math

import numpy as np
import pytest

import oracle
import synthetic


def gauss(means, log_scales, logits, rgb, sem=None, quats=None):
    n = len(means)
    return dict(mean=np.array(means, float), log_scale=np.array(log_scales, float),
                quat=np.array(quats if quats is not None else [[1, 0, 0, 0]] * n, float),
                opacity_logit=np.array(logits, float), rgb=np.array(rgb, float),
                sem=np.array(sem if sem is not None else [[0.0, 1.0]] * n, float))


def sigmoid(x):
    return 1 / (1 + math.exp(-x))


def alpha_closed_form(cam, mean, s, logit, px, py, b=0.3):
    """Axis-aligned Gaussian on a camera with identity pose: Sigma2D diagonal closed form."""
    z = mean[2]
    u = cam["fx"] * mean[0] / z + cam["cx"]
    v = cam["fy"] * mean[1] / z + cam["cy"]
    # off-axis J has a third column; axis-aligned Sigma makes Sigma2D still closed form:
    J = np.array([[cam["fx"] / z, 0, -cam["fx"] * mean[0] / z ** 2],
                  [0, cam["fy"] / z, -cam["fy"] * mean[1] / z ** 2]])
    S2 = J @ np.diag(np.exp(2 * np.asarray(s))) @ J.T + b * np.eye(2)
    d = np.stack([px - u, py - v])
    Q = np.linalg.inv(S2)
    sig = 0.5 * np.einsum("in,ij,jn->n", d, Q, d)
    return np.minimum(0.99, sigmoid(logit) * np.exp(-sig))


def test_single_gaussian_closed_form():
    cam = synthetic.cloud_camera()
    mean, s, logit = [0.1, -0.05, 2.0], np.log([0.05, 0.03, 0.04]), 1.5
    g = gauss([mean], [s], [logit], [[0.3, 0.6, 0.9]], sem=[[2.0, -1.0]])
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(76, 100, 1000), rng.integers(46, 67, 1000)], 1)
    r = oracle.render(g, cam, pixels=pix)
    a = alpha_closed_form(cam, mean, s, logit, pix[:, 0].astype(float), pix[:, 1].astype(float))
    a = np.where(a < 1 / 255, 0.0, a)
    assert (a > 0).sum() > 200
    assert np.allclose(r["rgb"], a[None] * np.array([0.3, 0.6, 0.9])[:, None], atol=1e-12)
    assert np.allclose(r["depth"], a * 2.0, atol=1e-12)
    assert np.allclose(r["sem"], a[None] * np.array([2.0, -1.0])[:, None], atol=1e-12)
    assert np.allclose(r["T"], 1 - a, atol=1e-12)
    assert np.array_equal(r["n_contrib"], (a > 0).astype(int))


def test_two_gaussians_over_operator_both_orders():
    """C = a1 c1 + (1-a1) a2 c2 with the nearer Gaussian first, whichever id it has."""
    cam = synthetic.cloud_camera()
    s = np.log([0.05, 0.05, 0.05])
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.0, 0.7, 0.4])
    px = np.array([[80, 60], [83, 58], [76, 64]])
    for z1, z2 in [(2.0, 3.0), (3.0, 2.0)]:
        g = gauss([[0, 0, z1], [0, 0, z2]], [s, s], [0.5, 1.0], [c1, c2])
        r = oracle.render(g, cam, pixels=px)
        a1 = alpha_closed_form(cam, [0, 0, z1], s, 0.5, px[:, 0] * 1.0, px[:, 1] * 1.0)
        a2 = alpha_closed_form(cam, [0, 0, z2], s, 1.0, px[:, 0] * 1.0, px[:, 1] * 1.0)
        (fa, fc, fz), (ba, bc, bz) = ((a1, c1, z1), (a2, c2, z2)) if z1 < z2 else ((a2, c2, z2), (a1, c1, z1))
        C = fa[None] * fc[:, None] + ((1 - fa) * ba)[None] * bc[:, None]
        assert np.allclose(r["rgb"], C, atol=1e-12)
        assert np.allclose(r["depth"], fa * fz + (1 - fa) * ba * bz, atol=1e-12)
        assert np.allclose(r["T"], (1 - fa) * (1 - ba), atol=1e-12)


def test_equal_depth_ties_break_by_id():
    cam = synthetic.cloud_camera()
    s = np.log([0.05] * 3)
    c1, c2 = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    g = gauss([[0, 0, 2.0], [0, 0, 2.0]], [s, s], [0.0, 0.0], [c1, c2])
    r = oracle.render(g, cam, pixels=[[80, 60]])
    a = 0.5
    assert np.allclose(r["rgb"][:, 0], a * c1 + (1 - a) * a * c2)


def test_invariants_weights_sum_and_constant_colour():
    """With every colour 1 and background 0: C = 1 - T_final = sum_i w_i at every pixel."""
    g = synthetic.cloud_scene(2000, 8, seed=1)
    g1 = dict(g, rgb=np.ones_like(g["rgb"]))
    cam = synthetic.cloud_camera()
    r = oracle.render(g1, cam)
    for ch in range(3):
        assert np.allclose(r["rgb"][ch], 1 - r["T"], atol=1e-12)
    assert r["T"].min() >= 1e-4 * (1 - 0.99) - 1e-15
    # background colour enters as T_final * bg
    r2 = oracle.render(g1, cam, cfg=dict(bg=(0.25, 0.5, 1.0)))
    for ch, bgv in enumerate((0.25, 0.5, 1.0)):
        assert np.allclose(r2["rgb"][ch], 1 - r["T"] + r["T"] * bgv, atol=1e-12)


def test_transmittance_is_product_of_one_minus_alpha():
    """A stack of k identical Gaussians at the same pixel: T = (1-a)^k, C = 1-(1-a)^k."""
    cam = synthetic.cloud_camera()
    s = np.log([0.05] * 3)
    for k in (1, 2, 3, 5):
        g = gauss([[0, 0, 2.0 + 0.01 * i] for i in range(k)], [s] * k, [-1.0] * k, [[1, 1, 1]] * k)
        r = oracle.render(g, cam, pixels=[[80, 60]])
        a = sigmoid(-1.0)
        assert r["T"][0] == pytest.approx((1 - a) ** k, rel=1e-12)
        assert r["rgb"][0, 0] == pytest.approx(1 - (1 - a) ** k, rel=1e-12)
        assert r["n_contrib"][0] == k


def test_opaque_front_hides_the_rest_and_stop_rule():
    """alpha clamps at 0.99; after two such layers T = 1.0000000000000018e-4 (kept), the
    third would give 1e-6 < 1e-4 so compositing stops before adding it."""
    cam = synthetic.cloud_camera()
    s = np.log([0.05] * 3)
    g = gauss([[0, 0, 2.0], [0, 0, 2.1], [0, 0, 2.2], [0, 0, 1.0e1]], [s] * 4, [8.0] * 4,
              [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]])
    r = oracle.render(g, cam, pixels=[[80, 60]])
    assert r["n_contrib"][0] == 2
    assert np.allclose(r["rgb"][:, 0], [0.99, 0.99 * 0.01, 0.0], atol=1e-14)
    assert r["T"][0] == pytest.approx(0.01 * 0.01, rel=1e-12)
    # moving the hidden ones further back changes nothing
    g2 = dict(g, mean=g["mean"] + np.array([[0, 0, 0], [0, 0, 0], [0, 0, 3.0], [0, 0, 5.0]]))
    r2 = oracle.render(g2, cam, pixels=[[80, 60]])
    assert np.allclose(r2["rgb"], r["rgb"], atol=0)


def test_skip_below_threshold():
    """A Gaussian whose alpha is below 1/255 at a pixel contributes nothing there."""
    cam = synthetic.cloud_camera()
    s = np.log([0.02] * 3)
    g = gauss([[0, 0, 2.0]], [s], [0.0], [[1, 1, 1]])
    # find the pixel row where alpha crosses 1/255 along x
    xs = np.arange(80, 100)
    a = alpha_closed_form(cam, [0, 0, 2.0], s, 0.0, xs * 1.0, np.full(xs.shape, 60.0))
    r = oracle.render(g, cam, pixels=np.stack([xs, np.full_like(xs, 60)], 1))
    expect = np.where(a < 1 / 255, 0.0, a)
    assert (a < 1 / 255).any() and (a >= 1 / 255).any()
    assert np.allclose(r["rgb"][0], expect, atol=1e-14)


def test_pixel_list_equals_full_image():
    g = synthetic.cloud_scene(500, 4, seed=3)
    cam = synthetic.cloud_camera()
    full = oracle.render(g, cam)
    rng = np.random.default_rng(2)
    pix = np.stack([rng.integers(0, 160, 300), rng.integers(0, 120, 300)], 1)
    part = oracle.render(g, cam, pixels=pix)
    assert np.array_equal(part["rgb"], full["rgb"][:, pix[:, 1], pix[:, 0]])
    assert np.array_equal(part["n_contrib"], full["n_contrib"][pix[:, 1], pix[:, 0]])


def _logit(p):
    return math.log(p / (1 - p))


def test_skip_and_clamp_flags_mark_only_the_band_of_the_alpha_error():
    """At the mean's pixel sigma = 0, so raw alpha = o: alpha within tol (relative) of 1/255
    or of 0.99 is flagged (a float32 alpha with that error may take the other branch), alpha
    three tolerances away is not."""
    cam = synthetic.cloud_camera()  # identity pose, (cx, cy) = (80, 60): the mean (0, 0, z) hits pixel (80, 60)
    s = np.log([0.05] * 3)
    tol = 1e-5
    for o, flag in ((1 / 255 * (1 + 0.5 * tol), oracle.FLAG_SKIP), (1 / 255 * (1 + 3 * tol), 0),
                    (0.99 * (1 - 0.5 * tol), oracle.FLAG_CLAMP), (0.99 * (1 + 0.5 * tol), oracle.FLAG_CLAMP),
                    (0.99 * (1 - 3 * tol), 0)):
        g = gauss([[0, 0, 2.0]], [s], [_logit(o)], [[1, 1, 1]])
        r = oracle.render(g, cam, pixels=[[80, 60]], tol=tol)
        assert r["flags"][0] & (oracle.FLAG_SKIP | oracle.FLAG_CLAMP) == flag, (o, r["flags"][0])
    # one pixel to the right sigma = conic_a / 2: raw alpha just below the skip threshold there
    # is flagged too (skipped, but a float32 alpha may pass)
    ca = oracle.project(gauss([[0, 0, 2.0]], [s], [0.0], [[1, 1, 1]]), cam)[0][oracle.P["CA"]]
    for f, flag in ((1 - 0.5 * tol, oracle.FLAG_SKIP), (1 - 3 * tol, 0)):
        o = 1 / 255 * f * math.exp(0.5 * ca)
        g = gauss([[0, 0, 2.0]], [s], [_logit(o)], [[1, 1, 1]])
        r = oracle.render(g, cam, pixels=[[81, 60]], tol=tol)
        assert r["flags"][0] & oracle.FLAG_SKIP == flag and r["n_contrib"][0] == 0, (f, r["flags"][0])


def test_stop_flag_marks_only_the_band_of_the_transmittance_error():
    """Two layers at one pixel: a clamped front (alpha = 0.99, T = 0.01) and a second with
    alpha = 0.99 - 0.01 delta, so T' = 1e-4 (1 + delta): the stop decision is flagged when
    delta lies within the transmittance band tol_T, and not three bands away."""
    cam = synthetic.cloud_camera()
    s = np.log([0.05] * 3)
    for delta, tol_T, flagged in ((1e-5, 2e-5, True), (6e-5, 2e-5, False), (1e-5, 0.0, False), (1e-5, 5e-5, True)):
        a2 = 0.99 - 0.01 * delta
        g = gauss([[0, 0, 2.0], [0, 0, 3.0]], [s, s], [8.0, _logit(a2)], [[1, 0, 0], [0, 1, 0]])
        r = oracle.render(g, cam, pixels=[[80, 60]], tol_T=tol_T)
        assert bool(r["flags"][0] & oracle.FLAG_STOP) == flagged, (delta, tol_T, r["flags"][0])
        assert r["n_contrib"][0] == 2


def test_depth_flag_marks_an_undecided_key_next_to_a_neighbour():
    """A depth exactly halfway between two float32 values (1 + 2^-24) has no decided key; the
    order against a Gaussian whose key is one float32 step away (1 + 2^-23) is then not fixed
    and the pixel is flagged.  Far apart, or both keys decided, nothing is flagged."""
    cam = synthetic.cloud_camera()
    s = np.log([0.05] * 3)
    for z1, z2, flagged in ((1.0 + 2.0 ** -24, 1.0 + 2.0 ** -23, True), (1.0 + 2.0 ** -24, 1.5, False),
                            (1.0, 1.0 + 2.0 ** -23, False), (1.0 + 2.0 ** -24, 1.0, True)):
        g = gauss([[0, 0, z1], [0, 0, z2]], [s, s], [-1.0, -1.0], [[1, 0, 0], [0, 1, 0]])
        r = oracle.render(g, cam, pixels=[[80, 60]])
        assert bool(r["flags"][0] & oracle.FLAG_DEPTH) == flagged, (z1, z2)
