"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds scene content only: Gaussian clouds, a procedural room with boxes,
a camera trajectory, a ray caster that produces ground-truth RGB-D-semantic frames, and
random target images.  It contains none of the splatting method's arithmetic
(projection, compositing, losses, pyramid construction live in the CUDA path and,
independently, in the oracle).

The paper evaluates on Replica (1200x680 RGB-D-semantic frames) and ScanNet (640x480);
neither dataset is available, so these generators stand in for them with the same image
sizes, Gaussian counts and class counts (Sec. IV-A).  Nothing here reproduces any item
of those datasets.

Conventions
-----------
* Camera frame: x right, y down, z forward (pinhole, pixel centres at integer
  coordinates).  ``R_cw``/``t_cw`` map world points into the camera frame.
* World frame of the room: z up, the room occupies [0,Lx] x [0,Ly] x [0,Lz] metres.
* Gaussians: mean (N,3), log_scale (N,3), quat (N,4) in (w,x,y,z) order,
  opacity_logit (N,), rgb (N,3), sem (N,C); all float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "cloud_scene", "cloud_camera", "random_targets", "Room", "make_camera",
    "REPLICA_LIKE", "SCANNET_LIKE", "look_camera",
]

# Image geometry of the two workload families (builder's choice: the paper prints no
# intrinsics).  Replica-like frames are 1200x680, ScanNet-like 640x480.
REPLICA_LIKE = dict(W=1200, H=680, fx=600.0, fy=600.0, cx=599.5, cy=339.5)
SCANNET_LIKE = dict(W=640, H=480, fx=580.0, fy=580.0, cx=319.5, cy=239.5)


def make_camera(W, H, fx, fy, cx, cy, R_cw=None, t_cw=None):
    """A pinhole camera as a plain dict (float64 values)."""
    R = np.eye(3) if R_cw is None else np.asarray(R_cw, dtype=np.float64).reshape(3, 3)
    t = np.zeros(3) if t_cw is None else np.asarray(t_cw, dtype=np.float64).reshape(3)
    return dict(W=int(W), H=int(H), fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy),
                R_cw=R.copy(), t_cw=t.copy())


def look_camera(intr: dict, position, yaw, pitch=0.0):
    """Camera at ``position`` looking along heading ``yaw`` (about world z) tilted by
    ``pitch`` (positive = up).  Returns a camera dict with world->camera pose."""
    c = np.asarray(position, dtype=np.float64)
    f = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
    right = np.array([f[1], -f[0], 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R_wc = np.stack([right, down, f], axis=1)  # columns: camera axes in world coords
    R_cw = R_wc.T
    t_cw = -R_cw @ c
    return make_camera(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], R_cw, t_cw)


# --------------------------------------------------------------------------------------
# Random Gaussian cloud in front of an identity camera (160x120 single-level workload)
# --------------------------------------------------------------------------------------

def cloud_camera():
    """160x120 pinhole, fx=fy=150, cx=80, cy=60, identity pose."""
    return make_camera(160, 120, 150.0, 150.0, 80.0, 60.0)


def cloud_scene(n=2000, n_sem=8, seed=1):
    """N Gaussians: means x,y~U[-1,1] m, z~U[1,4] m; log-scales ~U[ln .005, ln .05]^3;
    unit quaternions from normalised N(0,I4); opacity logits ~N(0,1); rgb~U[0,1]^3;
    semantic logits ~N(0,1)^C."""
    rng = np.random.default_rng(seed)
    mean = np.empty((n, 3))
    mean[:, 0:2] = rng.uniform(-1.0, 1.0, size=(n, 2))
    mean[:, 2] = rng.uniform(1.0, 4.0, size=n)
    log_scale = rng.uniform(math.log(0.005), math.log(0.05), size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity_logit = rng.normal(size=n)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    sem = rng.normal(size=(n, n_sem))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(mean=f32(mean), log_scale=f32(log_scale), quat=f32(q),
                opacity_logit=f32(opacity_logit), rgb=f32(rgb), sem=f32(sem))


def sh_coefficients(n, degree, scale=0.2, seed=3, channels=3):
    """Seeded view-dependent feature coefficients: N x ((D+1)^2 - 1) x channels float32
    (3 for colour, C for the semantic feature), the degree-l rows ~ N(0, (scale / l)^2)
    (higher degrees carry less energy, as fitted SH colour does)."""
    rng = np.random.default_rng(seed)
    K = (degree + 1) ** 2 - 1
    l = np.floor(np.sqrt(np.arange(1, K + 1))).astype(np.float64)   # degree of row k
    sh = rng.normal(size=(n, K, channels)) * (scale / l)[None, :, None]
    return np.ascontiguousarray(sh, dtype=np.float32)


def random_targets(H, W, n_classes, seed=2):
    """Seeded target frame: rgb~U[0,1] (3,H,W), depth~U[1,4] (H,W), label~U{0..n-1}."""
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(0.0, 1.0, size=(3, H, W)).astype(np.float32)
    depth = rng.uniform(1.0, 4.0, size=(H, W)).astype(np.float32)
    label = rng.integers(0, n_classes, size=(H, W)).astype(np.int32)
    return dict(rgb=rgb, depth=depth, label=label)


# --------------------------------------------------------------------------------------
# Procedural room: 6 inner faces + axis-aligned boxes resting on the floor
# --------------------------------------------------------------------------------------

def _hash01(i, j, salt):
    """Integer lattice hash -> [0,1).  Deterministic, vectorised (uint64 arithmetic,
    wrapping on overflow)."""
    with np.errstate(over="ignore"):
        return _hash01_impl(i, j, salt)


def _hash01_impl(i, j, salt):
    x = (np.asarray(i, dtype=np.int64).astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
         ^ np.asarray(j, dtype=np.int64).astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F)
         ^ np.asarray(salt, dtype=np.uint64) * np.uint64(0x165667B19E3779F9))
    x ^= x >> np.uint64(31)
    x *= np.uint64(0xBF58476D1CE4E5B9)
    x ^= x >> np.uint64(29)
    return (x >> np.uint64(11)).astype(np.float64) / float(1 << 53)


def _value_noise(a, b, cell, salt):
    sa, sb = a / cell, b / cell
    ia, ib = np.floor(sa), np.floor(sb)
    fa, fb = sa - ia, sb - ib
    fa = fa * fa * (3 - 2 * fa)
    fb = fb * fb * (3 - 2 * fb)
    h00 = _hash01(ia, ib, salt)
    h10 = _hash01(ia + 1, ib, salt)
    h01 = _hash01(ia, ib + 1, salt)
    h11 = _hash01(ia + 1, ib + 1, salt)
    return (h00 * (1 - fa) + h10 * fa) * (1 - fb) + (h01 * (1 - fa) + h11 * fa) * fb


def _checker(a, b, s):
    return (np.mod(np.floor(a / s) + np.floor(b / s), 2.0)).astype(np.float64)


@dataclass
class _Surface:
    origin: np.ndarray
    u: np.ndarray          # edge vector (metres)
    v: np.ndarray          # edge vector (metres)
    normal: np.ndarray     # unit normal towards the visible side
    label: int
    base: np.ndarray       # base colour
    salt: int

    @property
    def area(self):
        return float(np.linalg.norm(self.u) * np.linalg.norm(self.v))


@dataclass
class Room:
    """A seeded Lx x Ly x Lz room with ``n_boxes`` boxes on the floor.

    Every surface carries a procedural texture (checkers at three scales plus value
    noise) and a constant semantic class: floor, ceiling and the four walls are classes
    0..5; box k has class 6 + k mod (n_classes - 6).
    """
    size: tuple = (6.0, 5.0, 3.0)
    n_boxes: int = 20
    n_classes: int = 32
    seed: int = 3
    boxes: list = field(default_factory=list, init=False)
    surfaces: list = field(default_factory=list, init=False)

    def __post_init__(self):
        rng = np.random.default_rng(self.seed)
        Lx, Ly, Lz = self.size
        E = np.eye(3)
        def surf(o, u, v, n, label):
            base = rng.uniform(0.15, 0.9, size=3)
            self.surfaces.append(_Surface(np.asarray(o, float), np.asarray(u, float),
                                          np.asarray(v, float), np.asarray(n, float), label,
                                          base, int(rng.integers(1, 2**31))))
        # room faces (normals point inwards)
        surf([0, 0, 0], [Lx, 0, 0], [0, Ly, 0], E[2], 0)          # floor
        surf([0, 0, Lz], [Lx, 0, 0], [0, Ly, 0], -E[2], 1)        # ceiling
        surf([0, 0, 0], [0, Ly, 0], [0, 0, Lz], E[0], 2)          # x = 0
        surf([Lx, 0, 0], [0, Ly, 0], [0, 0, Lz], -E[0], 3)        # x = Lx
        surf([0, 0, 0], [Lx, 0, 0], [0, 0, Lz], E[1], 4)          # y = 0
        surf([0, Ly, 0], [Lx, 0, 0], [0, 0, Lz], -E[1], 5)        # y = Ly
        for k in range(self.n_boxes):
            s = rng.uniform(0.2, 1.0, size=3)
            x0 = rng.uniform(0.1, Lx - s[0] - 0.1)
            y0 = rng.uniform(0.1, Ly - s[1] - 0.1)
            lo = np.array([x0, y0, 0.0])
            hi = lo + s
            self.boxes.append((lo, hi))
            label = 6 + k % max(1, self.n_classes - 6)
            # faces: top, -x, +x, -y, +y (outward normals); the bottom rests on the floor
            surf([lo[0], lo[1], hi[2]], [s[0], 0, 0], [0, s[1], 0], E[2], label)
            surf([lo[0], lo[1], lo[2]], [0, s[1], 0], [0, 0, s[2]], -E[0], label)
            surf([hi[0], lo[1], lo[2]], [0, s[1], 0], [0, 0, s[2]], E[0], label)
            surf([lo[0], lo[1], lo[2]], [s[0], 0, 0], [0, 0, s[2]], -E[1], label)
            surf([lo[0], hi[1], lo[2]], [s[0], 0, 0], [0, 0, s[2]], E[1], label)

    # ---- appearance -----------------------------------------------------------------
    def texture(self, sid, a, b):
        """RGB in [0,1] of surface ``sid`` at metric surface coordinates (a, b)."""
        s = self.surfaces[sid]
        ch = 0.55 + 0.2 * _checker(a, b, 0.5) + 0.12 * _checker(a, b, 0.17) + 0.06 * _checker(a, b, 0.05)
        nz = _value_noise(a, b, 0.08, s.salt) - 0.5
        col = s.base[None, :] * ch[:, None] + 0.25 * nz[:, None]
        return np.clip(col, 0.0, 1.0)

    # ---- Gaussians ------------------------------------------------------------------
    def sample_gaussians(self, n, n_sem, seed, sem_mode="zeros", kappa=5.0,
                         log_scale_range=(math.log(0.005), math.log(0.05)),
                         opacity_logit_mean=2.0, opacity_logit_std=0.5, normal_std=0.002):
        """Sample ``n`` Gaussians area-proportionally on the room's surfaces.

        Means lie on the surfaces, offset along the normal by N(0, normal_std); log-scales
        are log-uniform in ``log_scale_range``; quaternions random unit; opacity logits
        N(mean, std); rgb from the surface texture.  ``sem_mode``: "zeros" (C zeros),
        "onehot" (kappa * one-hot of the class; needs n_sem == n_classes) or "random"
        (N(0,1)).  Also returns the per-Gaussian class in ``label``.
        """
        rng = np.random.default_rng(seed)
        areas = np.array([s.area for s in self.surfaces])
        sid = rng.choice(len(self.surfaces), size=n, p=areas / areas.sum())
        a01 = rng.uniform(size=n)
        b01 = rng.uniform(size=n)
        mean = np.empty((n, 3))
        rgb = np.empty((n, 3))
        label = np.empty(n, dtype=np.int32)
        for k, s in enumerate(self.surfaces):
            m = sid == k
            if not m.any():
                continue
            p = s.origin[None] + a01[m, None] * s.u[None] + b01[m, None] * s.v[None]
            p += rng.normal(0.0, normal_std, size=(m.sum(), 1)) * s.normal[None]
            mean[m] = p
            rgb[m] = self.texture(k, a01[m] * np.linalg.norm(s.u), b01[m] * np.linalg.norm(s.v))
            label[m] = s.label
        log_scale = rng.uniform(log_scale_range[0], log_scale_range[1], size=(n, 3))
        q = rng.normal(size=(n, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        opacity_logit = rng.normal(opacity_logit_mean, opacity_logit_std, size=n)
        if sem_mode == "onehot":
            assert n_sem == self.n_classes
            sem = np.zeros((n, n_sem))
            sem[np.arange(n), label] = kappa
        elif sem_mode == "random":
            sem = rng.normal(size=(n, n_sem))
        else:
            sem = np.zeros((n, n_sem))
        f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
        return dict(mean=f32(mean), log_scale=f32(log_scale), quat=f32(q),
                    opacity_logit=f32(opacity_logit), rgb=f32(rgb), sem=f32(sem), label=label)

    # ---- trajectory -----------------------------------------------------------------
    def trajectory(self, n_frames, intr, seed=7, duration=1.0):
        """Seeded smooth trajectory: position and yaw are sums of three sinusoids,
        staying >= 0.5 m from the walls and above the boxes."""
        rng = np.random.default_rng(seed)
        Lx, Ly, Lz = self.size
        centre = np.array([Lx / 2, Ly / 2, 1.6])
        amp = np.array([Lx / 2 - 1.0, Ly / 2 - 1.0, 0.3])
        w = rng.uniform(0.5, 2.0, size=(3, 3)) * 2 * math.pi
        ph = rng.uniform(0, 2 * math.pi, size=(3, 3))
        wa = rng.uniform(0.3, 1.0, size=(3, 3))
        wa /= wa.sum(axis=1, keepdims=True)
        yw = rng.uniform(0.3, 1.2, size=3) * 2 * math.pi
        yph = rng.uniform(0, 2 * math.pi, size=3)
        yaw0 = rng.uniform(0, 2 * math.pi)
        cams = []
        for f in range(n_frames):
            s = duration * f / max(1, n_frames)
            pos = centre + amp * np.array([np.sum(wa[d] * np.sin(w[d] * s + ph[d])) for d in range(3)])
            yaw = yaw0 + 1.5 * np.sum(np.sin(yw * s + yph)) / 3.0 * math.pi
            pitch = -0.25 + 0.1 * math.sin(2 * math.pi * s + yph[0])
            cams.append(look_camera(intr, pos, yaw, pitch))
        return cams

    # ---- ground truth frames ------------------------------------------------------------
    def raycast(self, cam, depth_noise=0.0, seed=0):
        """Ground-truth RGB (3,H,W), depth (H,W, camera z, metres) and label (H,W) of the
        room seen by ``cam``, by casting one ray through every pixel centre."""
        W, H = cam["W"], cam["H"]
        R_wc = cam["R_cw"].T
        c = -R_wc @ cam["t_cw"]
        xs, ys = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
        dc = np.stack([(xs - cam["cx"]) / cam["fx"], (ys - cam["cy"]) / cam["fy"], np.ones_like(xs)], -1)
        d = dc.reshape(-1, 3) @ R_wc.T          # world directions with unit camera-z
        P = d.shape[0]
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            L = np.array(self.size)
            # exit through the room box
            t_lo = (0.0 - c) * inv
            t_hi = (L - c) * inv
            t_far = np.maximum(t_lo, t_hi)
            t_far = np.where(np.isfinite(t_far), t_far, np.inf)
            axis = np.argmin(t_far, axis=1)
            t_best = t_far[np.arange(P), axis]
            upper = d[np.arange(P), axis] > 0
            # wall index: axis z -> floor(0)/ceiling(1); x -> 2/3; y -> 4/5
            wall_of = np.array([[2, 3], [4, 5], [0, 1]])
            sid = wall_of[axis, upper.astype(int)]
            for k, (lo, hi) in enumerate(self.boxes):
                a0 = (lo - c) * inv
                a1 = (hi - c) * inv
                tmin = np.minimum(a0, a1)
                tmax = np.maximum(a0, a1)
                tmin = np.where(np.isnan(tmin), -np.inf, tmin)
                tmax = np.where(np.isnan(tmax), np.inf, tmax)
                t_enter = tmin.max(axis=1)
                t_exit = tmax.min(axis=1)
                hit = (t_enter <= t_exit) & (t_enter > 1e-6) & (t_enter < t_best)
                if not hit.any():
                    continue
                ax = np.argmax(tmin, axis=1)
                neg = d[np.arange(P), ax] > 0   # entering through the low face
                # face order: top(0), -x(1), +x(2), -y(3), +y(4)
                face = np.where(ax == 2, 0, np.where(ax == 0, np.where(neg, 1, 2), np.where(neg, 3, 4)))
                t_best = np.where(hit, t_enter, t_best)
                sid = np.where(hit, 6 + 5 * k + face, sid)
        p = c[None] + t_best[:, None] * d
        rgb = np.zeros((P, 3))
        label = np.zeros(P, dtype=np.int32)
        for k in np.unique(sid):
            s = self.surfaces[k]
            m = sid == k
            rel = p[m] - s.origin[None]
            a = rel @ (s.u / np.linalg.norm(s.u))
            b = rel @ (s.v / np.linalg.norm(s.v))
            rgb[m] = self.texture(k, a, b)
            label[m] = s.label
        depth = t_best.copy()
        if depth_noise > 0:
            depth += np.random.default_rng(seed).normal(0.0, depth_noise, size=depth.shape)
        return dict(rgb=np.ascontiguousarray(rgb.T.reshape(3, H, W), dtype=np.float32),
                    depth=np.ascontiguousarray(depth.reshape(H, W), dtype=np.float32),
                    label=np.ascontiguousarray(label.reshape(H, W), dtype=np.int32))
