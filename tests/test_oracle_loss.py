"""Pins of the oracle's losses (Eq. 10-13): L1 closed form, SSIM against an independent
library computation (scipy's Gaussian filter) and its identity SSIM(x, x) = 1, the SSIM
gradient by finite differences, and cross-entropy against torch (CPU, float64)."""
import numpy as np
import pytest
import torch

import oracle


def scipy_ssim(x, y):
    """SSIM with scipy.ndimage.gaussian_filter: sigma 1.5, radius 5 (11 taps), zero
    padding ('constant'); the 1-D taps are normalised over the 11 taps by scipy."""
    from scipy.ndimage import gaussian_filter
    f = lambda a: gaussian_filter(a, sigma=1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    vals = []
    for ch in range(x.shape[0]):
        a, b = x[ch], y[ch]
        mx, my = f(a), f(b)
        sxx, syy, sxy = f(a * a) - mx * mx, f(b * b) - my * my, f(a * b) - mx * my
        vals.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)))
    return float(np.mean(vals))


def test_ssim_identity_and_range():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(3, 20, 31))
    assert oracle.ssim(x, x) == pytest.approx(1.0, abs=1e-12)
    y = rng.uniform(size=(3, 20, 31))
    assert -1.0 <= oracle.ssim(x, y) < 1.0


def test_ssim_matches_scipy_gaussian_filter():
    rng = np.random.default_rng(1)
    for shape in [(3, 17, 23), (1, 40, 12), (2, 11, 11)]:
        x = rng.uniform(size=shape)
        y = np.clip(x + rng.normal(0, 0.2, size=shape), 0, 1)
        assert oracle.ssim(x, y) == pytest.approx(scipy_ssim(x, y), rel=1e-12, abs=1e-12)


def test_ssim_gradient_fd():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(2, 13, 15))
    y = rng.uniform(size=(2, 13, 15))
    _, g = oracle.ssim(x, y, grad=True)
    h = 1e-6
    for _ in range(40):
        ix = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[ix] += h
        xm[ix] -= h
        fd = (oracle.ssim(xp, y) - oracle.ssim(xm, y)) / (2 * h)
        assert g[ix] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_l1_closed_form_and_mask():
    x = np.array([[1.0, 2.0], [3.0, 0.0]])
    y = np.array([[0.0, 2.0], [5.0, 1.0]])
    v, g = oracle.l1(x, y)
    assert v == pytest.approx((1 + 0 + 2 + 1) / 4)
    assert np.array_equal(g, np.array([[0.25, 0.0], [-0.25, -0.25]]))
    v, g = oracle.l1(x, y, mask=np.array([[True, False], [True, False]]))
    assert v == pytest.approx(1.5)
    assert np.array_equal(g, np.array([[0.5, 0.0], [-0.5, 0.0]]))
    assert oracle.l1(x, y, mask=np.zeros_like(x, bool))[0] == 0.0


def test_level_loss_depth_term_masks_invalid_targets():
    """Eq. 11 through level_loss: the depth L1 is the mean over pixels with a valid target
    depth (> 0) only, and pixels without one get zero gradient (worked by hand)."""
    r_d = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    g_d = np.array([[0.0, 2.5, 1.0], [0.0, 5.0, 7.0]])
    rgb = np.full((3, 2, 3), 0.5)
    sem = np.zeros((2, 2, 3))
    lab = np.zeros((2, 3), dtype=np.int32)
    _, terms, grads = oracle.level_loss(rgb, r_d, sem, rgb, g_d, lab)
    # valid: |2 - 2.5| + |3 - 1| + |5 - 5| + |6 - 7| = 3.5 over 4 pixels
    assert terms["L_d"] == pytest.approx(0.875, rel=1e-15)
    assert np.array_equal(grads["depth"], np.array([[0.0, -0.25, 0.25], [0.0, 0.0, -0.25]]))


def test_cross_entropy_matches_torch():
    rng = np.random.default_rng(3)
    z = rng.normal(size=(8, 9, 11)) * 3
    lab = rng.integers(-1, 8, size=(9, 11))
    v, g = oracle.cross_entropy(z, lab)
    zt = torch.tensor(z.reshape(8, -1).T, dtype=torch.float64, requires_grad=True)
    lt = torch.tensor(lab.reshape(-1), dtype=torch.long)
    ref = torch.nn.functional.cross_entropy(zt, lt, ignore_index=-1, reduction="mean")
    ref.backward()
    assert v == pytest.approx(ref.item(), rel=1e-12)
    assert np.allclose(g.reshape(8, -1).T, zt.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_level_loss_gradients_fd():
    """Eq. 13 total (RGB L1 + D-SSIM, masked depth L1, CE through a decoder): every
    gradient by central differences."""
    rng = np.random.default_rng(4)
    H, W, C, K = 12, 14, 4, 6
    r_rgb = rng.uniform(size=(3, H, W)); g_rgb = rng.uniform(size=(3, H, W))
    r_d = rng.uniform(1, 3, size=(H, W)); g_d = np.where(rng.uniform(size=(H, W)) < 0.2, 0.0, rng.uniform(1, 3, size=(H, W)))
    r_s = rng.normal(size=(C, H, W)); lab = rng.integers(-1, K, size=(H, W))
    dec = rng.normal(size=(K, C))
    # term weights other than 1, so that a weight missing from a value or a gradient shows
    wts = dict(w_depth=0.7, w_sem=1.3)
    tot, terms, grads = oracle.level_loss(r_rgb, r_d, r_s, g_rgb, g_d, lab, decoder=dec, **wts)
    assert tot == pytest.approx(terms["L_r"] + terms["L_d"] + terms["L_s"])
    # each weighted term is its weight times the unweighted term
    _, t1, _ = oracle.level_loss(r_rgb, r_d, r_s, g_rgb, g_d, lab, decoder=dec)
    assert terms["L_d"] == pytest.approx(0.7 * t1["L_d"], rel=1e-14)
    assert terms["L_s"] == pytest.approx(1.3 * t1["L_s"], rel=1e-14)
    h = 1e-6
    f = lambda a, b, c, d: oracle.level_loss(a, b, c, g_rgb, g_d, lab, decoder=d, **wts)[0]
    for name, arr, idx in [("rgb", r_rgb, 0), ("depth", r_d, 1), ("sem", r_s, 2), ("decoder", dec, 3)]:
        for _ in range(15):
            ix = tuple(rng.integers(0, s) for s in arr.shape)
            args_p = [r_rgb.copy(), r_d.copy(), r_s.copy(), dec.copy()]
            args_m = [r_rgb.copy(), r_d.copy(), r_s.copy(), dec.copy()]
            args_p[idx][ix] += h
            args_m[idx][ix] -= h
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            assert grads[name][ix] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, ix)


def test_paper_mode_semantic_loss_fd():
    """Eq. 12 mode: L1 + D-SSIM on a semantic colour image."""
    rng = np.random.default_rng(5)
    H, W = 11, 13
    r_s = rng.uniform(size=(3, H, W)); g_s = rng.uniform(size=(3, H, W))
    r_rgb = rng.uniform(size=(3, H, W)); r_d = rng.uniform(1, 2, size=(H, W))
    kw = dict(sem_mode="paper", lambda_r=0.35, lambda_s=0.15, w_sem=1.25)   # lambda_r != lambda_s
    tot, terms, grads = oracle.level_loss(r_rgb, r_d, r_s, r_rgb, r_d, g_s, **kw)
    l1 = np.abs(r_s - g_s).mean()
    assert terms["L_s"] == pytest.approx(1.25 * (0.85 * l1 + 0.15 * (1 - oracle.ssim(r_s, g_s))))
    assert terms["L_r"] == pytest.approx(0.0, abs=1e-12) and terms["L_d"] == 0.0
    h = 1e-6
    for _ in range(10):
        ix = tuple(rng.integers(0, s) for s in r_s.shape)
        sp, sm = r_s.copy(), r_s.copy()
        sp[ix] += h
        sm[ix] -= h
        fd = (oracle.level_loss(r_rgb, r_d, sp, r_rgb, r_d, g_s, **kw)[0]
              - oracle.level_loss(r_rgb, r_d, sm, r_rgb, r_d, g_s, **kw)[0]) / (2 * h)
        assert grads["sem"][ix] == pytest.approx(fd, rel=1e-5, abs=1e-9)
