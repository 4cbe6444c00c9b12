"""FP64 CPU oracle of the multi-level-pyramid Gaussian-splatting hot path (RGBDS-SLAM).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg, never by the product package.  It shares no code with the
CUDA path; the two meet only through the seeded generators in ``synthetic``.

Pieces and the passages they follow:

* ``project``            Eq. 2-3 (EWA covariance projection; C file ``sg_oracle.c``).
* ``render``             Eq. 7-9 brute-force compositing per pixel (C).
* ``render_backward``    hand-derived adjoint of Eq. 7-9 and Eq. 2-3 (Sec. III-D) (C).
* ``sh_basis``,          view-dependent colour and semantic feature of Sec. III-B: rgb (sem)
  ``view_colours``,      + sum of real spherical harmonics of degree 1..3 of the
  ``view_semantics``     camera-to-mean direction (numpy); ``render`` and ``render_backward``
                         take them, and their adjoint to the SH coefficients, rgb, sem and the
                         mean, when the parameters carry ``sh`` and/or ``sem_sh``.
* ``ssim``               SSIM of Wang et al. 2004 used by Eq. 10 and 12 (C).
* ``level_cameras``,     Eq. 4-6 image pyramid: 2x2 box mean for RGB, valid-only mean for
  ``build_pyramid``      depth, 2x2 majority for labels; per-level intrinsics keep pixel
                         centres consistent (numpy).
* ``level_loss``         Eq. 10-13 per pyramid level with D-SSIM = 1 - SSIM, masked depth L1,
                         and either cross-entropy on composited semantic logits or the
                         paper's L1 + D-SSIM on a semantic colour image (numpy + C SSIM).
* ``tile_reach``,        the set N of Eq. 7-9 restricted to a screen tile, by definition:
  ``tile_pairs``         a Gaussian belongs to a tile's set when its alpha reaches alpha_min
                         at one of the tile's pixels (FP64 brute force over the tile's pixel
                         centres), plus the least exponent over the tile's pixel-centre
                         rectangle (how close a footprint comes to a tile it misses) (numpy).
* ``tile_lists``         integer reference of the order of those sets: (record, tile) pairs
                         ordered by (tile, float32 depth key bits, record index) (numpy
                         lexsort), with per-tile ranges.

Submodules: ``mlp`` (the learned initializer's network) and ``init`` (insertion of new
Gaussians: the heuristic initializer, the network's patch features and the application of
its outputs).

Parity pins: the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` tie every function
here to closed forms, invariants, library routines and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB = os.path.join(_HERE, "libsg_oracle.so")
_lib = None

DEFAULT_CFG = dict(alpha_max=0.99, alpha_min=1.0 / 255.0, T_min=1e-4, z_near=0.2,
                   dilation=0.3, bg=(0.0, 0.0, 0.0), fov_clamp=1.3, isotropic=0)

# projection record fields (must match the enum in sg_oracle.c)
P = dict(VALID=0, U=1, V=2, DEPTH=3, OPAC=4, CA=5, CB=6, CC=7, S00=8, S01=9, S11=10,
         TX=11, TY=12, TZ=13, CLX=14, CLY=15, EXTX=16, EXTY=17, LIMX=18, LIMY=19, DKEY=20, DAMB=21, GEXTX=22, GEXTY=23)
FLAG_SKIP, FLAG_STOP, FLAG_DEPTH, FLAG_CLAMP = 1, 2, 4, 8


def build(force=False):
    """Compile the C oracle with gcc (OpenMP, -O2; portable flags for x86 and Arm)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        lib.oc_project.argtypes = [ctypes.c_int, D, D, D, D, D, D, D]
        lib.oc_render.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, ctypes.c_int, I,
                                  ctypes.c_double, ctypes.c_double, D, D, D, D, I, I]
        lib.oc_render_backward.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, D, D, D,
                                           ctypes.c_int, I, D, D, D, D, D, D, D, D, D, D]
        lib.oc_ssim.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, D]
        lib.oc_ssim.restype = ctypes.c_double
        lib.oc_proj_stride.restype = ctypes.c_int
        lib.oc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads():
    return _load().oc_num_threads()


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _null(kind=ctypes.c_double):
    return ctypes.POINTER(kind)()


def pack_camera(cam):
    return np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["W"], cam["H"],
                     *np.asarray(cam["R_cw"], np.float64).reshape(9),
                     *np.asarray(cam["t_cw"], np.float64).reshape(3)], dtype=np.float64)


def pack_cfg(cfg=None):
    c = dict(DEFAULT_CFG)
    if cfg:
        c.update(cfg)
    bg = c["bg"]
    return np.array([c["alpha_max"], c["alpha_min"], c["T_min"], c["z_near"], c["dilation"],
                     bg[0], bg[1], bg[2], c["fov_clamp"], float(c["isotropic"])], dtype=np.float64)


# ------------------------------------------------------------------------------------------
# Eq. 2-3 and Eq. 7-9
# ------------------------------------------------------------------------------------------

def project(g, cam, cfg=None):
    """Per-Gaussian projection records (N x 24 float64, fields in ``P``)."""
    lib = _load()
    N = g["mean"].shape[0]
    m, pm = _d(g["mean"]); s, ps = _d(g["log_scale"]); q, pq = _d(g["quat"])
    o, po = _d(g["opacity_logit"]); c, pc = _d(pack_camera(cam)); f, pf = _d(pack_cfg(cfg))
    out = np.zeros((N, lib.oc_proj_stride()), dtype=np.float64)
    lib.oc_project(N, pm, ps, pq, po, pc, pf, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# ------------------------------------------------------------------------------------------
# View-dependent colour: real spherical harmonics of degree 1..3 (the SH colour of Sec. III-B)
# ------------------------------------------------------------------------------------------

def sh_basis(d, degree):
    """Real spherical harmonics Y_1 .. Y_K, K = (degree+1)^2 - 1, at unit directions d (n, 3),
    in the usual graphics order (m = -l..l within each degree l, Condon-Shortley signs):
      l = 1: -c1 y, c1 z, -c1 x                                        c1 = sqrt(3 / 4pi)
      l = 2: a xy, -a yz, b (2z^2 - x^2 - y^2), -a xz, c (x^2 - y^2)
             a = sqrt(15/pi)/2, b = sqrt(5/pi)/4, c = sqrt(15/pi)/4
      l = 3: -e y (3x^2 - y^2), f xyz, -h y (4z^2 - x^2 - y^2), k z (2z^2 - 3x^2 - 3y^2),
             -h x (4z^2 - x^2 - y^2), m z (x^2 - y^2), -e x (x^2 - 3y^2)
             e = sqrt(35/2pi)/4, f = sqrt(105/pi)/2, h = sqrt(21/2pi)/4, k = sqrt(7/pi)/4,
             m = sqrt(105/pi)/4.
    Returns (n, K)."""
    d = np.asarray(d, np.float64)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = np.pi
    out = []
    if degree >= 1:
        c1 = np.sqrt(3 / (4 * pi))
        out += [-c1 * y, c1 * z, -c1 * x]
    if degree >= 2:
        a, b, c = np.sqrt(15 / pi) / 2, np.sqrt(5 / pi) / 4, np.sqrt(15 / pi) / 4
        out += [a * x * y, -a * y * z, b * (2 * z * z - x * x - y * y), -a * x * z, c * (x * x - y * y)]
    if degree >= 3:
        e, f, h = np.sqrt(35 / (2 * pi)) / 4, np.sqrt(105 / pi) / 2, np.sqrt(21 / (2 * pi)) / 4
        k, m = np.sqrt(7 / pi) / 4, np.sqrt(105 / pi) / 4
        out += [-e * y * (3 * x * x - y * y), f * x * y * z, -h * y * (4 * z * z - x * x - y * y),
                k * z * (2 * z * z - 3 * x * x - 3 * y * y), -h * x * (4 * z * z - x * x - y * y),
                m * z * (x * x - y * y), -e * x * (x * x - 3 * y * y)]
    return np.stack(out, 1) if out else np.zeros((len(d), 0))


def sh_basis_grad(d, degree):
    """d Y_k / d(x, y, z) of the polynomials of sh_basis (before restriction to the sphere):
    (n, K, 3)."""
    d = np.asarray(d, np.float64)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    o = np.zeros_like(x)
    pi = np.pi
    g = []
    if degree >= 1:
        c1 = np.sqrt(3 / (4 * pi))
        g += [(o, -c1 + o, o), (o, o, c1 + o), (-c1 + o, o, o)]
    if degree >= 2:
        a, b, c = np.sqrt(15 / pi) / 2, np.sqrt(5 / pi) / 4, np.sqrt(15 / pi) / 4
        g += [(a * y, a * x, o), (o, -a * z, -a * y), (-2 * b * x, -2 * b * y, 4 * b * z), (-a * z, o, -a * x),
              (2 * c * x, -2 * c * y, o)]
    if degree >= 3:
        e, f, h = np.sqrt(35 / (2 * pi)) / 4, np.sqrt(105 / pi) / 2, np.sqrt(21 / (2 * pi)) / 4
        k, m = np.sqrt(7 / pi) / 4, np.sqrt(105 / pi) / 4
        g += [(-6 * e * x * y, -e * (3 * x * x - 3 * y * y), o),
              (f * y * z, f * x * z, f * x * y),
              (2 * h * x * y, -h * (4 * z * z - x * x - 3 * y * y), -8 * h * y * z),
              (-6 * k * x * z, -6 * k * y * z, k * (6 * z * z - 3 * x * x - 3 * y * y)),
              (-h * (4 * z * z - 3 * x * x - y * y), 2 * h * x * y, -8 * h * x * z),
              (2 * m * x * z, -2 * m * y * z, m * (x * x - y * y)),
              (-e * (3 * x * x - 3 * y * y), 6 * e * x * y, o)]
    if not g:
        return np.zeros((len(d), 0, 3))
    return np.stack([np.stack(t, 1) for t in g], 1)


def sh_degree_of(g):
    """SH degree D of a parameter dict: g["sh"] is N x ((D+1)^2 - 1) x 3 (colour) and/or
    g["sem_sh"] is N x ((D+1)^2 - 1) x C (semantic feature), one D for both; 0 without them."""
    Ks = {np.asarray(g[k]).shape[1] for k in ("sh", "sem_sh") if g.get(k) is not None}
    Ks.discard(0)
    if not Ks:
        return 0
    assert len(Ks) == 1, "sh and sem_sh must have the same degree"
    K = Ks.pop()
    D = int(round(np.sqrt(K + 1))) - 1
    assert (D + 1) ** 2 - 1 == K and 1 <= D <= 3, K
    return D


def view_basis(g, cam):
    """Unit directions d from the camera centre c = -R_cw^T t_cw to the means, |mean - c| and
    the basis Y_k(d) (N, K); all None when the parameters carry no SH."""
    D = sh_degree_of(g)
    if D == 0:
        return None, None, None
    R = np.asarray(cam["R_cw"], np.float64).reshape(3, 3)
    c = -R.T @ np.asarray(cam["t_cw"], np.float64).reshape(3)
    v = np.asarray(g["mean"], np.float64) - c
    n = np.linalg.norm(v, axis=1)
    d = v / n[:, None]
    return d, n, sh_basis(d, D)


def view_colours(g, cam):
    """Colour of every Gaussian seen from cam: rgb + sum_k sh_k Y_k(d) (no offset, no clamp:
    degree 0 is rgb itself).  Returns (colour (N, 3), d (N, 3), |mean - c| (N,), Y (N, K))."""
    rgb = np.asarray(g["rgb"], np.float64)
    d, n, Y = view_basis(g, cam)
    if Y is None or g.get("sh") is None:
        return rgb, d, n, Y
    return rgb + np.einsum("nk,nkc->nc", Y, np.asarray(g["sh"], np.float64)), d, n, Y


def view_semantics(g, cam):
    """Semantic feature of every Gaussian seen from cam: sem + sum_k sem_sh_k Y_k(d), the same
    view dependence as the colour; sem itself without sem_sh."""
    sem = np.asarray(g["sem"], np.float64).reshape(np.asarray(g["mean"]).shape[0], -1)
    if g.get("sem_sh") is None:
        return sem
    Y = view_basis(g, cam)[2]
    return sem + np.einsum("nk,nkc->nc", Y, np.asarray(g["sem_sh"], np.float64))


def render(g, cam, cfg=None, pixels=None, tol=1e-5, tol_T=2e-5):
    """Render RGB, depth and C semantic channels.

    ``pixels``: None for the whole W x H image (outputs shaped (ch, H, W)), else an (n, 2)
    int array of (x, y) pixel coordinates (outputs shaped (ch, n)).  Also returns the final
    transmittance ``T``, the contributor count ``n_contrib`` and per-pixel ambiguity
    ``flags`` (FLAG_*): some decision of the pixel is not fixed for an evaluation whose alpha
    carries a relative error up to ``tol`` and whose transmittance one up to ``tol_T`` -- the
    exact alpha lies within ``tol`` of the skip threshold (FLAG_SKIP) or of the clamp
    (FLAG_CLAMP), the transmittance after a contributor within ``tol_T`` of T_min (FLAG_STOP),
    or a contributor's float32 depth key is undecided next to a neighbouring key (FLAG_DEPTH).
    """
    lib = _load()
    proj = project(g, cam, cfg)
    N = proj.shape[0]
    C = g["sem"].shape[1]
    colour = view_colours(g, cam)[0]
    pr, ppr = _d(proj); rgb, prgb = _d(colour); sem, psem = _d(view_semantics(g, cam))
    c, pc = _d(pack_camera(cam)); f, pf = _d(pack_cfg(cfg))
    if pixels is None:
        n = cam["W"] * cam["H"]
        pix_ptr = _null(ctypes.c_int)
        shape = (cam["H"], cam["W"])
    else:
        pixels, pix_ptr = _i(np.asarray(pixels).reshape(-1, 2))
        n = pixels.shape[0]
        shape = (n,)
    o_rgb = np.zeros((3, n)); o_d = np.zeros(n); o_s = np.zeros((C, n)); o_T = np.zeros(n)
    o_nc = np.zeros(n, dtype=np.int32); o_fl = np.zeros(n, dtype=np.int32)
    P_ = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    I_ = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    lib.oc_render(N, C, ppr, prgb, psem, pc, pf, n, pix_ptr, float(tol), float(tol_T), P_(o_rgb), P_(o_d),
                  P_(o_s), P_(o_T), I_(o_nc), I_(o_fl))
    return dict(rgb=o_rgb.reshape(3, *shape), depth=o_d.reshape(shape),
                sem=o_s.reshape(C, *shape), T=o_T.reshape(shape),
                n_contrib=o_nc.reshape(shape), flags=o_fl.reshape(shape), proj=proj)


def render_backward(g, cam, g_rgb, g_depth, g_sem, cfg=None, pixels=None):
    """Gradients of sum(g_rgb*rgb + g_depth*depth + g_sem*sem) with respect to all
    Gaussian parameters.  Upstream arrays are (ch, H, W) for the whole image or (ch, n)
    for a pixel list.  Returns dict with mean, log_scale, quat, opacity_logit, rgb, sem and
    the per-Gaussian 2D gradients ``g2d`` (N x 8: u v conic_a conic_b conic_c opacity
    depth 0)."""
    lib = _load()
    proj = project(g, cam, cfg)
    N = proj.shape[0]
    C = g["sem"].shape[1]
    colour, sh_d, sh_n, sh_Y = view_colours(g, cam)
    m, pm = _d(g["mean"]); s, ps = _d(g["log_scale"]); q, pq = _d(g["quat"])
    pr, ppr = _d(proj); rgb, prgb = _d(colour); sem, psem = _d(view_semantics(g, cam))
    c, pc = _d(pack_camera(cam)); f, pf = _d(pack_cfg(cfg))
    if pixels is None:
        n = cam["W"] * cam["H"]
        pix_ptr = _null(ctypes.c_int)
    else:
        pixels, pix_ptr = _i(np.asarray(pixels).reshape(-1, 2))
        n = pixels.shape[0]
    gr, pgr = _d(np.asarray(g_rgb).reshape(3, n)); gd, pgd = _d(np.asarray(g_depth).reshape(n))
    gs, pgs = _d(np.asarray(g_sem).reshape(C, n))
    out = dict(mean=np.zeros((N, 3)), log_scale=np.zeros((N, 3)), quat=np.zeros((N, 4)),
               opacity_logit=np.zeros(N), rgb=np.zeros((N, 3)), sem=np.zeros((N, C)),
               g2d=np.zeros((N, 8)))
    P_ = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib.oc_render_backward(N, C, pm, ps, pq, ppr, prgb, psem, pc, pf, n, pix_ptr, pgr, pgd, pgs,
                           P_(out["mean"]), P_(out["log_scale"]), P_(out["quat"]),
                           P_(out["opacity_logit"]), P_(out["rgb"]), P_(out["sem"]), P_(out["g2d"]))
    if sh_Y is not None:
        # f = f0 + sum_k coef_k Y_k(d) for the colour (rgb, sh) and the semantic feature
        # (sem, sem_sh): dL/dcoef_k = Y_k dL/df; dL/df0 = dL/df (as computed);
        # dL/dmean += (I - d d^T) / |v| * sum_k (coef_k . dL/df) grad Y_k(d)
        w = np.zeros_like(sh_Y)
        for key, gf in (("sh", out["rgb"]), ("sem_sh", out["sem"])):
            if g.get(key) is not None:
                out[key] = np.einsum("nk,nc->nkc", sh_Y, gf)
                w += np.einsum("nkc,nc->nk", np.asarray(g[key], np.float64), gf)
        gdir = np.einsum("nk,nkj->nj", w, sh_basis_grad(sh_d, sh_degree_of(g)))
        gdir -= sh_d * (gdir * sh_d).sum(1, keepdims=True)
        out["mean"] += gdir / sh_n[:, None]
    return out


# ------------------------------------------------------------------------------------------
# Eq. 4-6: pyramid
# ------------------------------------------------------------------------------------------

def level_cameras(cam, levels):
    """Cameras of pyramid levels 0..levels-1.  Level l+1 pixel x covers level-l pixels
    2x and 2x+1 whose centres average to 2x+0.5, so u_{l+1} = (u_l - 0.5)/2, i.e.
    f_{l+1} = f_l/2, c_{l+1} = (c_l - 0.5)/2; sizes floor(W/2) x floor(H/2)."""
    out = [dict(cam)]
    for _ in range(1, levels):
        p = out[-1]
        out.append(dict(p, W=p["W"] // 2, H=p["H"] // 2, fx=p["fx"] / 2, fy=p["fy"] / 2,
                        cx=(p["cx"] - 0.5) / 2, cy=(p["cy"] - 0.5) / 2))
    return out


def downsample(rgb, depth, label):
    """One pyramid step: 2x2 box mean of RGB, mean of the valid (>0) depths of the 2x2
    block (0 if none), majority label of the block's valid (>=0) labels with ties to the
    lowest id (-1 if none)."""
    C, H, W = rgb.shape
    h, w = H // 2, W // 2
    r = np.asarray(rgb, np.float64)[:, :2 * h, :2 * w].reshape(C, h, 2, w, 2)
    rgb2 = r.mean(axis=(2, 4))
    d = np.asarray(depth, np.float64)[:2 * h, :2 * w].reshape(h, 2, w, 2)
    valid = d > 0
    cnt = valid.sum(axis=(1, 3))
    depth2 = np.where(cnt > 0, (d * valid).sum(axis=(1, 3)) / np.maximum(cnt, 1), 0.0)
    lab = np.asarray(label)[:2 * h, :2 * w].reshape(h, 2, w, 2).transpose(0, 2, 1, 3).reshape(h, w, 4)
    label2 = np.full((h, w), -1, dtype=np.int32)
    for yy in range(h):
        for xx in range(w):
            vals = [v for v in lab[yy, xx] if v >= 0]
            if not vals:
                continue
            best, bc = None, -1
            for v in sorted(set(vals)):
                cc = vals.count(v)
                if cc > bc:
                    best, bc = v, cc
            label2[yy, xx] = best
    return rgb2, depth2, label2


def build_pyramid(rgb, depth, label, levels):
    out = [(np.asarray(rgb, np.float64), np.asarray(depth, np.float64), np.asarray(label, np.int32))]
    for _ in range(1, levels):
        out.append(downsample(*out[-1]))
    return out


# ------------------------------------------------------------------------------------------
# Eq. 10-13: per-level loss and its gradient
# ------------------------------------------------------------------------------------------

def ssim(x, y, grad=False):
    """Mean SSIM of planar images x, y (ch, H, W); with grad=True also d(mean SSIM)/dx."""
    lib = _load()
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.ndim == 2:
        x, y = x[None], y[None]
    nch, H, W = x.shape
    xa, px = _d(x); ya, py = _d(y)
    if grad:
        gx = np.zeros_like(xa)
        val = lib.oc_ssim(H, W, nch, px, py, gx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return val, gx
    return lib.oc_ssim(H, W, nch, px, py, _null())


def l1(x, y, mask=None):
    """mean |x - y| over the masked entries and its gradient (sign/n; 0 where equal)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if mask is None:
        mask = np.ones(x.shape, bool)
    n = int(mask.sum())
    if n == 0:
        return 0.0, np.zeros_like(x)
    d = (x - y) * mask
    return float(np.abs(d).sum() / n), np.sign(d) / n


def cross_entropy(logits, label):
    """Mean over pixels with label >= 0 of -log softmax(logits)[label]; logits (K, H, W).
    Returns the value and its gradient with respect to logits."""
    z = np.asarray(logits, np.float64)
    lab = np.asarray(label)
    valid = lab >= 0
    n = int(valid.sum())
    if n == 0:
        return 0.0, np.zeros_like(z)
    zmax = z.max(axis=0, keepdims=True)
    e = np.exp(z - zmax)
    ssum = e.sum(axis=0, keepdims=True)
    logp = z - zmax - np.log(ssum)
    safe = np.where(valid, lab, 0)
    picked = np.take_along_axis(logp, safe[None], axis=0)[0]
    val = float(-(picked * valid).sum() / n)
    grad = e / ssum
    onehot = np.zeros_like(z)
    np.put_along_axis(onehot, safe[None], 1.0, axis=0)
    grad = (grad - onehot) * valid[None] / n
    return val, grad


def level_loss(r_rgb, r_depth, r_sem, gt_rgb, gt_depth, gt_sem, lambda_r=0.2, lambda_s=0.2,
               w_depth=1.0, w_sem=1.0, sem_mode="ce", decoder=None):
    """Eq. 13 at one pyramid level: L_r + w_depth*L_d + w_sem*L_s.

    L_r = (1-lambda_r) mean|R - R_gt| + lambda_r (1 - SSIM(R, R_gt))      (Eq. 10)
    L_d = mean over {D_gt > 0} of |D - D_gt|                               (Eq. 11)
    L_s = "ce":    mean CE(softmax(decoder @ S), label) over label >= 0    (semantic logits)
          "paper": (1-lambda_s) mean|S - S_gt| + lambda_s (1 - SSIM(S, S_gt))  (Eq. 12)
    ``decoder``: (K, C) matrix applied per pixel to S (identity when None).
    Returns (total, dict of terms, dict of gradients rgb/depth/sem[/decoder]).
    """
    lr, g_l1 = l1(r_rgb, gt_rgb)
    s_val, g_s = ssim(r_rgb, gt_rgb, grad=True)
    L_r = (1 - lambda_r) * lr + lambda_r * (1 - s_val)
    g_rgb = (1 - lambda_r) * g_l1 - lambda_r * g_s.reshape(np.shape(r_rgb))
    ld, g_d = l1(r_depth, gt_depth, mask=np.asarray(gt_depth) > 0)
    L_d = w_depth * ld
    g_depth = w_depth * g_d
    grads = dict(rgb=g_rgb, depth=g_depth)
    S = np.asarray(r_sem, np.float64)
    if sem_mode == "ce":
        Cc = S.shape[0]
        if decoder is not None:
            Wd = np.asarray(decoder, np.float64)
            logits = np.einsum("kc,chw->khw", Wd, S)
        else:
            logits = S
        ce, g_log = cross_entropy(logits, gt_sem)
        L_s = w_sem * ce
        if decoder is not None:
            grads["sem"] = w_sem * np.einsum("kc,khw->chw", Wd, g_log)
            grads["decoder"] = w_sem * np.einsum("khw,chw->kc", g_log, S)
        else:
            grads["sem"] = w_sem * g_log
    else:
        ls, g_ls1 = l1(S, gt_sem)
        ss, g_ss = ssim(S, gt_sem, grad=True)
        L_s = w_sem * ((1 - lambda_s) * ls + lambda_s * (1 - ss))
        grads["sem"] = w_sem * ((1 - lambda_s) * g_ls1 - lambda_s * g_ss.reshape(S.shape))
    total = L_r + L_d + L_s
    return total, dict(L_r=L_r, L_d=L_d, L_s=L_s), grads


# ------------------------------------------------------------------------------------------
# Tile-instance lists (integer reference; the depth sort of Eq. 7-9's set N per tile)
# ------------------------------------------------------------------------------------------

def tile_pairs(proj, cam, tile_w, tile_h):
    """(Gaussian, tile x, tile y) for every tile of each Gaussian's FP64 support rectangle:
    the tiles holding a pixel centre within the half extents (EXTX, EXTY) of its 2D mean,
    outside which alpha < alpha_min (an exact bound).  Culled Gaussians give none."""
    p = np.asarray(proj, np.float64)
    gs, txs, tys = [], [], []
    for i in np.nonzero(p[:, P["VALID"]] > 0)[0]:
        u, v, ex, ey = p[i, P["U"]], p[i, P["V"]], p[i, P["EXTX"]], p[i, P["EXTY"]]
        x0, x1 = max(0, int(np.ceil(u - ex))), min(cam["W"] - 1, int(np.floor(u + ex)))
        y0, y1 = max(0, int(np.ceil(v - ey))), min(cam["H"] - 1, int(np.floor(v + ey)))
        if x0 > x1 or y0 > y1:
            continue
        tx, ty = np.meshgrid(np.arange(x0 // tile_w, x1 // tile_w + 1), np.arange(y0 // tile_h, y1 // tile_h + 1))
        gs.append(np.full(tx.size, i)); txs.append(tx.ravel()); tys.append(ty.ravel())
    if not gs:
        z = np.zeros(0, np.int64)
        return z, z, z
    return np.concatenate(gs), np.concatenate(txs), np.concatenate(tys)


def tile_reach(proj, cam, gauss, tx, ty, tile_w, tile_h, chunk=4096):
    """For (Gaussian, tile) pairs, from the FP64 projection:
    ``alpha``: the largest alpha = o exp(-sigma) of the Gaussian over the tile's pixel centres
    (Eq. 3; the Gaussian belongs to the tile's set N iff this reaches alpha_min; 0 for a culled
    Gaussian), ``sigma_min``: the least sigma = 1/2 d^T conic d over the continuous rectangle
    spanned by the tile's pixel centres, and ``thr`` = ln(o / alpha_min) (alpha >= alpha_min
    needs sigma <= thr).  sigma is a positive definite quadratic: its minimum over the
    rectangle is 0 when the rectangle holds the mean, else the least of the clamped 1-D
    minima along the four edges."""
    p = np.asarray(proj, np.float64)
    gauss, tx, ty = (np.asarray(a, np.int64) for a in (gauss, tx, ty))
    n = len(gauss)
    alpha, smin = np.zeros(n), np.full(n, np.inf)
    alpha_min = 1.0 / 255.0
    o = p[gauss, P["OPAC"]]
    with np.errstate(divide="ignore"):
        thr = np.where(o > 0, np.log(np.maximum(o, 1e-300) / alpha_min), -np.inf)
    ox, oy = np.meshgrid(np.arange(tile_w), np.arange(tile_h))
    ox, oy = ox.ravel(), oy.ravel()
    for s in range(0, n, chunk):
        sl = slice(s, min(n, s + chunk))
        pg = p[gauss[sl]]
        ok = pg[:, P["VALID"]] > 0
        a, b, c = pg[:, P["CA"]], pg[:, P["CB"]], pg[:, P["CC"]]
        X0, Y0 = tx[sl] * tile_w, ty[sl] * tile_h
        X1 = np.minimum(X0 + tile_w - 1, cam["W"] - 1)
        Y1 = np.minimum(Y0 + tile_h - 1, cam["H"] - 1)
        xs, ys = X0[:, None] + ox[None], Y0[:, None] + oy[None]
        inside = (xs <= X1[:, None]) & (ys <= Y1[:, None])
        dx, dy = xs - pg[:, P["U"]][:, None], ys - pg[:, P["V"]][:, None]
        sig = 0.5 * (a[:, None] * dx * dx + c[:, None] * dy * dy) + b[:, None] * dx * dy
        al = np.where(inside, pg[:, P["OPAC"]][:, None] * np.exp(-np.maximum(sig, 0.0)), 0.0)
        alpha[sl] = np.where(ok, al.max(1), 0.0)
        # least sigma over [x0, x1] x [y0, y1] (offsets from the mean), A = a/2, B = b/2, C = c/2
        x0, x1 = X0 - pg[:, P["U"]], X1 - pg[:, P["U"]]
        y0, y1 = Y0 - pg[:, P["V"]], Y1 - pg[:, P["V"]]
        A, B, C = 0.5 * a, 0.5 * b, 0.5 * c
        with np.errstate(all="ignore"):
            q = lambda x, y: A * x * x + 2 * B * x * y + C * y * y
            best = np.full(len(A), np.inf)
            for x in (x0, x1):
                best = np.minimum(best, q(x, np.clip(-B * x / C, y0, y1)))
            for y in (y0, y1):
                best = np.minimum(best, q(np.clip(-B * y / A, x0, x1), y))
        holds = (x0 <= 0) & (x1 >= 0) & (y0 <= 0) & (y1 >= 0)
        smin[sl] = np.where(ok, np.where(holds, 0.0, best), np.inf)
    return dict(alpha=alpha, sigma_min=smin, thr=thr)


def tile_lists(rects, depth, n_tiles_x, tile_offset, n_total_tiles, n_per_view, keep=None):
    """Reference tile-instance lists from per-record tile rectangles.

    rects:   (R, 4) int half-open tile rectangles (tx0, ty0, tx1, ty1) of each record
             (record r belongs to view r // n_per_view); empty rectangles emit nothing.
    depth:   (R,) float32 depths (ordering key: their bit patterns, all positive).
    n_tiles_x, tile_offset: per-view tile-grid width and first global tile id.
    keep:    optional function (records, tx, ty) -> bool array deciding which (record,
             tile) pairs of the rectangles are listed (all of them without it).
    Returns (tile_ids, record_ids, ranges) with instances ordered by (global tile id,
    depth bits, record id) and ranges (n_total_tiles, 2) = [start, end) per tile.
    """
    rects = np.asarray(rects, np.int64)
    R = rects.shape[0]
    view = np.arange(R) // n_per_view
    tiles, recs = [], []
    for r in range(R):
        tx0, ty0, tx1, ty1 = rects[r]
        if tx1 <= tx0 or ty1 <= ty0:
            continue
        v = view[r]
        for ty in range(ty0, ty1):
            for tx in range(tx0, tx1):
                tiles.append(tile_offset[v] + ty * n_tiles_x[v] + tx)
                recs.append(r)
    tiles = np.asarray(tiles, np.int64)
    recs = np.asarray(recs, np.int64)
    if keep is not None and len(recs):
        v = view[recs]
        local = tiles - np.asarray(tile_offset, np.int64)[v]
        ntx = np.asarray(n_tiles_x, np.int64)[v]
        k = np.asarray(keep(recs, local % ntx, local // ntx), bool)
        tiles, recs = tiles[k], recs[k]
    dbits = np.asarray(depth, np.float32).view(np.int32).astype(np.int64)[recs] if len(recs) else np.zeros(0, np.int64)
    order = np.lexsort((recs, dbits, tiles))
    tiles, recs = tiles[order], recs[order]
    ranges = np.zeros((n_total_tiles, 2), np.int64)
    if len(tiles):
        starts = np.searchsorted(tiles, np.arange(n_total_tiles), side="left")
        ends = np.searchsorted(tiles, np.arange(n_total_tiles), side="right")
        ranges[:, 0], ranges[:, 1] = starts, ends
        empty = starts == ends
        ranges[empty] = 0
    return tiles, recs, ranges
