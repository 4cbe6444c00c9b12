"""Pins of the oracle's view-dependent colour (spherical-harmonic colour, Sec. III-B): the real
basis against scipy's complex spherical harmonics and against orthonormality on the sphere,
its polynomial gradient by finite differences, the colour's dependence on the camera centre
only, and the adjoint through colour -> (sh, rgb, mean) by FP64 central differences of the
rendered images."""
import numpy as np
import pytest

import oracle
import synthetic

sp = pytest.importorskip("scipy.special")


def unit_dirs(n, seed=0):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def real_sh_from_scipy(d, degree):
    """Real SH in the graphics order from scipy's complex Y_l^m (Condon-Shortley phase kept):
    m < 0: sqrt(2) Im Y_l^|m|, m = 0: Y_l^0, m > 0: sqrt(2) Re Y_l^m."""
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = []
    for l in range(1, degree + 1):
        for m in range(-l, l + 1):
            y = sp.sph_harm_y(l, abs(m), theta, phi)
            out.append(np.sqrt(2) * y.imag if m < 0 else (y.real if m == 0 else np.sqrt(2) * y.real))
    return np.stack(out, 1)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_basis_matches_scipy(degree):
    d = unit_dirs(500, seed=degree)
    Y = oracle.sh_basis(d, degree)
    assert Y.shape == (500, (degree + 1) ** 2 - 1)
    np.testing.assert_allclose(Y, real_sh_from_scipy(d, degree), atol=1e-12)


def test_basis_orthonormal_on_sphere():
    # Gauss-Legendre in cos(theta) x uniform azimuth: exact for the degree-6 products Y_i Y_j
    nt, nphi = 8, 16
    ct, wt = np.polynomial.legendre.leggauss(nt)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    CT, PHI = np.meshgrid(ct, phi, indexing="ij")
    ST = np.sqrt(1 - CT ** 2)
    d = np.stack([ST * np.cos(PHI), ST * np.sin(PHI), CT], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).reshape(-1)
    Y = oracle.sh_basis(d, 3)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(15), atol=1e-12)
    # orthogonal to the constant (degree 0) function as well
    np.testing.assert_allclose(w @ Y, 0, atol=1e-12)


def test_basis_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(size=(40, 3))          # off the sphere: the gradient is the polynomial's
    J = oracle.sh_basis_grad(p, 3)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3); e[j] = h
        fd = (oracle.sh_basis(p + e, 3) - oracle.sh_basis(p - e, 3)) / (2 * h)
        np.testing.assert_allclose(J[:, :, j], fd, rtol=1e-7, atol=1e-7)


def test_view_colour_depends_on_camera_centre_only():
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(50, 4, seed=1).items()}
    g["sh"] = np.random.default_rng(2).normal(size=(50, 15, 3)) * 0.3
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24)
    # the same centre c = 0 under another rotation
    a = 0.4
    R2 = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    cam2 = dict(cam, R_cw=R2, t_cw=np.zeros(3))
    c1 = oracle.view_colours(g, dict(cam, t_cw=np.zeros(3)))[0]
    c2 = oracle.view_colours(g, cam2)[0]
    np.testing.assert_allclose(c1, c2, atol=1e-13)
    # seen along +z from the origin, only the m = 0 terms of each degree survive:
    # Y_1^0 = sqrt(3/4pi), Y_2^0 = sqrt(5/4pi), Y_3^0 = sqrt(7/4pi) at the north pole
    g1 = {k: v[:1].copy() for k, v in g.items()}
    g1["mean"][0] = [0, 0, 3.0]
    col = oracle.view_colours(g1, dict(cam, R_cw=np.eye(3), t_cw=np.zeros(3)))[0][0]
    sh = g1["sh"][0]
    exp = g1["rgb"][0] + sum(np.sqrt((2 * l + 1) / (4 * np.pi)) * sh[l * l + l - 1] for l in (1, 2, 3))
    np.testing.assert_allclose(col, exp, atol=1e-13)


def test_view_direction_is_the_camera_ray():
    """For a general pose the unit view direction d is the camera-space position of the mean
    (R_cw mean + t_cw), normalised and rotated back to the world frame, and |mean - c| is its
    length: the camera centre is the point the pose maps to the camera origin."""
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(40, 4, seed=3).items()}
    g["sh"] = np.zeros((40, 3, 3))
    a, b = 0.35, -0.6
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    R = Rz @ Rx
    t = np.array([0.4, -0.25, 1.1])
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24, R_cw=R, t_cw=t)
    d, n, _ = oracle.view_basis(g, cam)
    tc = g["mean"] @ R.T + t
    nc = np.linalg.norm(tc, axis=1)
    np.testing.assert_allclose(n, nc, rtol=1e-13)
    np.testing.assert_allclose(d, (tc / nc[:, None]) @ R, atol=1e-13)


def test_zero_sh_is_degree_zero():
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(60, 4, seed=2).items()}
    cam = synthetic.make_camera(32, 24, 30, 30, 16, 12)
    r0 = oracle.render(g, cam)
    gz = dict(g, sh=np.zeros((60, 8, 3)))
    r1 = oracle.render(gz, cam)
    for k in ("rgb", "depth", "sem"):
        np.testing.assert_array_equal(r0[k], r1[k])
    rng = np.random.default_rng(0)
    up = (rng.normal(size=(3, 24, 32)), rng.normal(size=(24, 32)), rng.normal(size=(4, 24, 32)))
    b0 = oracle.render_backward(g, cam, *up)
    b1 = oracle.render_backward(gz, cam, *up)
    # the oracle's threaded backward sums in a run-dependent order: equal up to rounding
    for k in ("mean", "log_scale", "quat", "opacity_logit", "rgb", "sem"):
        np.testing.assert_allclose(b0[k], b1[k], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("degree, keys", [(1, ("sh",)), (3, ("sh",)), (2, ("sem_sh",)), (2, ("sh", "sem_sh"))])
def test_sh_adjoint_matches_fd(degree, keys):
    from test_oracle_backward import tiny_scene
    g = tiny_scene(n=8, seed=11)
    K = (degree + 1) ** 2 - 1
    rng4 = np.random.default_rng(4)
    if "sh" in keys:
        g["sh"] = rng4.normal(size=(8, K, 3)) * 0.4
    if "sem_sh" in keys:
        g["sem_sh"] = rng4.normal(size=(8, K, g["sem"].shape[1])) * 0.4
    # a camera off the origin, so that the centre enters the view direction
    cam = synthetic.make_camera(40, 32, 40, 40, 20, 16)
    cam = dict(cam, t_cw=np.array([0.05, -0.03, 0.1]))
    cfg = dict(alpha_min=0.0, T_min=0.0)
    rng = np.random.default_rng(7)
    up = (rng.normal(size=(3, 32, 40)), rng.normal(size=(32, 40)), rng.normal(size=(4, 32, 40)))

    def L(gg):
        r = oracle.render(gg, cam, cfg)
        return (up[0] * r["rgb"]).sum() + (up[1] * r["depth"]).sum() + (up[2] * r["sem"]).sum()

    an = oracle.render_backward(g, cam, *up, cfg=cfg)
    h = 1e-5
    for key in keys + ("rgb", "sem", "mean"):
        for ix in np.ndindex(g[key].shape):
            gp = {k: v.copy() for k, v in g.items()}
            gm = {k: v.copy() for k, v in g.items()}
            gp[key][ix] += h
            gm[key][ix] -= h
            fd = (L(gp) - L(gm)) / (2 * h)
            assert abs(fd - an[key][ix]) <= 2e-5 * (abs(fd) + 1e-3), (key, ix, fd, an[key][ix])


def test_semantic_sh_view_dependence():
    """The semantic feature follows the same view dependence as the colour: with sem_sh equal
    to the colour's coefficients on 3 channels, the two agree channel by channel; zero sem_sh
    renders exactly the plain semantic feature."""
    g = {k: np.asarray(v, np.float64) for k, v in synthetic.cloud_scene(40, 4, seed=3).items()}
    sh = np.random.default_rng(9).normal(size=(40, 8, 3)) * 0.3
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24, t_cw=[0.2, 0.0, -0.1])
    g2 = dict(g, sh=sh, sem_sh=np.concatenate([sh, np.zeros((40, 8, 1))], 2),
              sem=np.concatenate([g["rgb"], np.zeros((40, 1))], 1))
    col = oracle.view_colours(g2, cam)[0]
    sem = oracle.view_semantics(g2, cam)
    np.testing.assert_allclose(sem[:, :3], col, atol=1e-14)
    r0 = oracle.render(g, cam)
    r1 = oracle.render(dict(g, sem_sh=np.zeros((40, 3, 4))), cam)
    np.testing.assert_array_equal(r0["sem"], r1["sem"])
