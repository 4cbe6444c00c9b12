"""Pins of the oracle's projection (Eq. 2-3, EWA generalisation) to closed forms and to
numerical differentiation of the pinhole map -- nothing here re-types the oracle."""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import P


def one(mean, log_scale, quat=(1, 0, 0, 0), logit=2.0, n_sem=4):
    return dict(mean=np.array([mean], float), log_scale=np.array([log_scale], float),
                quat=np.array([quat], float), opacity_logit=np.array([logit], float),
                rgb=np.array([[0.2, 0.5, 0.9]]), sem=np.arange(n_sem, dtype=float)[None] / n_sem)


def test_isotropic_on_axis_matches_eq2():
    """Eq. 2: r2D = f r / d for an isotropic Gaussian on the optical axis (no dilation)."""
    cam = synthetic.make_camera(200, 100, 150.0, 150.0, 100.0, 50.0)
    for r, d in [(0.01, 1.0), (0.05, 2.5), (0.2, 7.0)]:
        g = one([0, 0, d], [math.log(r)] * 3, quat=(0.3, -0.5, 0.7, 0.1))
        pr = oracle.project(g, cam, dict(dilation=0.0))[0]
        r2d = 150.0 * r / d
        assert pr[P["VALID"]] == 1
        assert pr[P["S00"]] == pytest.approx(r2d ** 2, rel=1e-12)
        assert pr[P["S11"]] == pytest.approx(r2d ** 2, rel=1e-12)
        assert abs(pr[P["S01"]]) < 1e-12 * r2d ** 2
        assert pr[P["U"]] == pytest.approx(100.0) and pr[P["V"]] == pytest.approx(50.0)
        assert pr[P["DEPTH"]] == pytest.approx(d)


def test_axis_aligned_on_axis_closed_form():
    """Sigma2D = diag(fx^2 e^{2 s0}/z^2, fy^2 e^{2 s1}/z^2) + b I on the axis."""
    cam = synthetic.make_camera(320, 240, 300.0, 250.0, 160.0, 120.0)
    s = np.log([0.03, 0.01, 0.2])
    z = 3.0
    g = one([0, 0, z], s)
    pr = oracle.project(g, cam, dict(dilation=0.3))[0]
    assert pr[P["S00"]] == pytest.approx(300.0 ** 2 * math.exp(2 * s[0]) / z ** 2 + 0.3, rel=1e-12)
    assert pr[P["S11"]] == pytest.approx(250.0 ** 2 * math.exp(2 * s[1]) / z ** 2 + 0.3, rel=1e-12)
    det = pr[P["S00"]] * pr[P["S11"]] - pr[P["S01"]] ** 2
    assert pr[P["CA"]] == pytest.approx(pr[P["S11"]] / det)
    assert pr[P["CC"]] == pytest.approx(pr[P["S00"]] / det)


def _pinhole(cam, pw):
    t = cam["R_cw"] @ pw + cam["t_cw"]
    return np.array([cam["fx"] * t[0] / t[2] + cam["cx"], cam["fy"] * t[1] / t[2] + cam["cy"]])


def test_ewa_matches_numerical_jacobian_off_axis():
    """Off-axis, rotated camera: Sigma2D = A Sigma A^T + bI with A = d(u,v)/d(world point),
    A taken by central differences of the pinhole map (independent of the oracle's J)."""
    rng = np.random.default_rng(3)
    cam = synthetic.look_camera(synthetic.SCANNET_LIKE, [1.0, 2.0, 1.5], 0.4, -0.2)
    for _ in range(20):
        ahead = np.array([math.cos(0.4), math.sin(0.4), -0.1])
        mu = np.array([1.0, 2.0, 1.5]) + rng.uniform(1.0, 4.0) * ahead + rng.normal(0, 0.3, 3)
        s = rng.uniform(math.log(0.005), math.log(0.1), 3)
        q = rng.normal(size=4)
        g = one(mu, s, q)
        pr = oracle.project(g, cam, dict(dilation=0.3))[0]
        if pr[P["CLX"]] or pr[P["CLY"]]:
            continue
        h = 1e-6
        A = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = h
            A[:, k] = (_pinhole(cam, mu + e) - _pinhole(cam, mu - e)) / (2 * h)
        qn = q / np.linalg.norm(q)
        w, x, y, z = qn
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        # independent check that R is a rotation taking e_k to its columns
        assert np.allclose(R @ R.T, np.eye(3)) and np.linalg.det(R) == pytest.approx(1.0)
        Sig = R @ np.diag(np.exp(2 * s)) @ R.T
        S2 = A @ Sig @ A.T + 0.3 * np.eye(2)
        assert pr[P["S00"]] == pytest.approx(S2[0, 0], rel=1e-6)
        assert pr[P["S11"]] == pytest.approx(S2[1, 1], rel=1e-6)
        assert pr[P["S01"]] == pytest.approx(S2[0, 1], rel=1e-6, abs=1e-9 * abs(S2).max())
        uv = _pinhole(cam, mu)
        assert pr[P["U"]] == pytest.approx(uv[0]) and pr[P["V"]] == pytest.approx(uv[1])


def test_ewa_clamped_jacobian_is_the_jacobian_at_the_clamped_point():
    """Reading of the support rules: the Jacobian of Eq. 3 is taken at the mean with t_x/t_z
    clamped to +-1.3 (W/2)/fx and t_y/t_z to +-1.3 (H/2)/fy.  So Sigma2D = A Sigma A^T + bI
    with A the numerical Jacobian of the pinhole map at the world point whose camera
    coordinates are the clamped ones.  A camera with fx != fy and W != H tells the two
    limits apart; means inside, beyond one limit and beyond both are all checked."""
    a = 0.3
    R = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    t0 = np.array([0.1, -0.2, 0.3])
    cam = synthetic.make_camera(160, 90, 120.0, 150.0, 79.5, 44.5, R_cw=R, t_cw=t0)
    limx, limy = 1.3 * 80 / 120.0, 1.3 * 45 / 150.0
    rng = np.random.default_rng(8)
    seen = set()
    for rx, ry in [(0.2, 0.1), (0.78, 0.1), (-1.1, 0.2), (0.3, 0.36), (0.1, -0.5), (0.3, 0.6),
                   (1.0, -0.7), (-0.95, 0.45)]:
        tz = rng.uniform(1.5, 3.0)
        tc = np.array([rx * tz, ry * tz, tz])
        mu = R.T @ (tc - t0)
        s = rng.uniform(math.log(0.01), math.log(0.1), 3)
        q = rng.normal(size=4)
        pr = oracle.project(one(mu, s, q), cam, dict(dilation=0.3))[0]
        cx_, cy_ = abs(rx) > limx, abs(ry) > limy
        assert (pr[P["CLX"]], pr[P["CLY"]]) == (cx_, cy_), (rx, ry)
        seen.add((cx_, cy_))
        tcl = np.array([np.clip(rx, -limx, limx) * tz, np.clip(ry, -limy, limy) * tz, tz])
        mcl = R.T @ (tcl - t0)
        h = 1e-6
        A = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = h
            A[:, k] = (_pinhole(cam, mcl + e) - _pinhole(cam, mcl - e)) / (2 * h)
        qn = q / np.linalg.norm(q)
        w, x, y, z = qn
        Rq = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                       [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                       [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        S2 = A @ (Rq @ np.diag(np.exp(2 * s)) @ Rq.T) @ A.T + 0.3 * np.eye(2)
        assert pr[P["S00"]] == pytest.approx(S2[0, 0], rel=1e-6), (rx, ry)
        assert pr[P["S11"]] == pytest.approx(S2[1, 1], rel=1e-6), (rx, ry)
        assert pr[P["S01"]] == pytest.approx(S2[0, 1], rel=1e-6, abs=1e-9 * abs(S2).max()), (rx, ry)
        # the 2D mean is the unclamped projection
        uv = _pinhole(cam, mu)
        assert pr[P["U"]] == pytest.approx(uv[0]) and pr[P["V"]] == pytest.approx(uv[1])
    assert seen == {(False, False), (True, False), (False, True), (True, True)}


def test_quaternion_sign_and_scale_invariance():
    g = synthetic.cloud_scene(50, 4, seed=9)
    cam = synthetic.cloud_camera()
    base = oracle.project(g, cam)
    for f in (-1.0, 3.7, -0.2):
        g2 = dict(g, quat=g["quat"].astype(np.float64) * f)
        assert np.allclose(oracle.project(g2, cam), base, rtol=1e-12, atol=1e-12)


def test_near_plane_and_tiny_opacity_cull():
    cam = synthetic.cloud_camera()
    assert oracle.project(one([0, 0, 0.2], [-3] * 3), cam)[0][P["VALID"]] == 0
    assert oracle.project(one([0, 0, -1.0], [-3] * 3), cam)[0][P["VALID"]] == 0
    assert oracle.project(one([0, 0, 0.2001], [-3] * 3), cam)[0][P["VALID"]] == 1
    # o = sigmoid(-6) < 1/255: can never reach the skip threshold
    assert oracle.project(one([0, 0, 2.0], [-3] * 3, logit=-6.0), cam)[0][P["VALID"]] == 0


def test_depth_key_is_camera_depth_rounded_to_float32():
    """The ordering key of the sorted set N (Eq. 7-9) is the camera-space depth t_z rounded to
    the nearest float32: for a general pose it equals float32(R20 x + R21 y + R22 z + t_z0)
    summed exactly (fractions), and only depths within 2^-40 of their terms' magnitude of a
    float32 rounding midpoint are flagged as undecided."""
    from fractions import Fraction as F
    rng = np.random.default_rng(6)
    a = 0.5
    R = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]]) @ \
        np.array([[math.cos(0.3), 0, math.sin(0.3)], [0, 1, 0], [-math.sin(0.3), 0, math.cos(0.3)]])
    R = R.astype(np.float32).astype(np.float64)
    t0 = np.array([0.3, -0.2, 0.7], np.float32).astype(np.float64)
    cam = synthetic.make_camera(64, 48, 60, 60, 32, 24, R_cw=R, t_cw=t0)
    for _ in range(300):
        m = rng.uniform(-3, 3, 3).astype(np.float32).astype(np.float64)
        exact = sum(F(float(R[2, i])) * F(float(m[i])) for i in range(3)) + F(float(t0[2]))
        pr = oracle.project(one(m, [-3] * 3), cam)[0]
        assert pr[P["DKEY"]] == float(np.float32(float(exact))), (m, pr[P["DKEY"]], float(exact))
        if float(exact) > 0.5:  # no cancellation: far from any midpoint at this band
            assert pr[P["DAMB"]] == 0
    # an exact midpoint between 1.0f and the next float32 is undecided; its neighbours are not
    cam0 = synthetic.make_camera(64, 48, 60, 60, 32, 24)
    for z, amb in ((1.0 + 2.0 ** -24, 1), (1.0 + 2.0 ** -23, 0), (1.0, 0), (1.0 + 2.0 ** -24 + 2.0 ** -38, 0)):
        pr = oracle.project(one([0.0, 0.0, z], [-3] * 3), cam0)[0]
        assert pr[P["DAMB"]] == amb, z
        assert pr[P["DKEY"]] == float(np.float32(z))


def test_extents_are_exact_bounds():
    """Outside the half extents alpha < 1/255 (checked by brute force on a fine grid);
    on the boundary's extreme point alpha equals 1/255."""
    rng = np.random.default_rng(1)
    cam = synthetic.cloud_camera()
    for _ in range(10):
        g = one(rng.uniform([-0.3, -0.3, 1.5], [0.3, 0.3, 3]), rng.uniform(-4, -2.5, 3),
                rng.normal(size=4), logit=rng.normal(1, 1))
        pr = oracle.project(g, cam)[0]
        if not pr[P["VALID"]]:
            continue
        a, b, c, o = pr[P["CA"]], pr[P["CB"]], pr[P["CC"]], pr[P["OPAC"]]
        ex, ey = pr[P["EXTX"]], pr[P["EXTY"]]
        dy = np.linspace(-3 * ey, 3 * ey, 4001)
        # on the vertical line dx = ex the largest alpha is attained at dy* = -b ex / c
        for sgn in (1, -1):
            dx = sgn * ex * (1 + 1e-6)
            sig = 0.5 * (a * dx * dx + c * dy * dy) + b * dx * dy
            assert (o * np.exp(-sig)).max() < 1 / 255
            dstar = -b * (sgn * ex) / c
            sig_star = 0.5 * (a * ex * ex + c * dstar ** 2) + b * (sgn * ex) * dstar
            assert o * math.exp(-sig_star) == pytest.approx(1 / 255, rel=1e-6)


def test_eq2_isotropic_mode_equals_ewa_on_axis():
    """Eq. 2 mode (isotropic = 1) and the EWA projection are different code paths; for an
    isotropic Gaussian on the optical axis they must give the same 2D Gaussian."""
    cam = synthetic.make_camera(240, 160, 180.0, 170.0, 120.0, 80.0)
    for r, d, dil in [(0.02, 1.5, 0.3), (0.1, 4.0, 0.0), (0.3, 9.0, 0.3)]:
        g = one([0, 0, d], [math.log(r)] * 3, quat=(0.2, 0.4, -0.6, 0.3))
        ewa = oracle.project(g, cam, dict(dilation=dil))[0]
        iso = oracle.project(g, cam, dict(dilation=dil, isotropic=1))[0]
        for k in ("VALID", "U", "V", "DEPTH", "S00", "S11", "CA", "CB", "CC", "EXTX", "EXTY"):
            assert iso[P[k]] == pytest.approx(ewa[P[k]], rel=1e-9, abs=1e-12), k


def test_eq2_isotropic_mode_invariances():
    """Eq. 2 uses only the radius e^{s0}: rotation and the other log-scales do not matter,
    and the 2D radius is invariant to scaling radius and camera distance together."""
    rng = np.random.default_rng(9)
    cam = synthetic.look_camera(synthetic.SCANNET_LIKE, [0.5, -1.0, 1.2], 0.7, 0.1)
    ahead = np.array([math.cos(0.7), math.sin(0.7), 0.1])
    for _ in range(10):
        mu = np.array([0.5, -1.0, 1.2]) + rng.uniform(1.5, 3.0) * ahead + rng.normal(0, 0.2, 3)
        s0 = math.log(rng.uniform(0.01, 0.1))
        a = oracle.project(one(mu, [s0, -3.0, -1.0], quat=(1, 0, 0, 0)), cam, dict(isotropic=1, dilation=0.0))[0]
        b = oracle.project(one(mu, [s0, -0.5, -6.0], quat=tuple(rng.normal(size=4))), cam,
                           dict(isotropic=1, dilation=0.0))[0]
        for k in ("S00", "S01", "S11", "CA", "CB", "CC", "EXTX", "EXTY", "U", "V"):
            assert a[P[k]] == pytest.approx(b[P[k]], rel=1e-12, abs=1e-15), k
        # the same Gaussian twice as large and twice as far along its viewing ray
        c_w = -cam["R_cw"].T @ cam["t_cw"]
        mu2 = c_w + 2.0 * (mu - c_w)
        c = oracle.project(one(mu2, [s0 + math.log(2.0), 0, 0]), cam, dict(isotropic=1, dilation=0.0))[0]
        assert c[P["S00"]] == pytest.approx(a[P["S00"]], rel=1e-9)
        assert c[P["S11"]] == pytest.approx(a[P["S11"]], rel=1e-9)
        assert abs(a[P["S01"]]) == 0.0
