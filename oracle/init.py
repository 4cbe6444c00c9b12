"""FP64 reference of the Gaussian insertion step (TEST INFRASTRUCTURE ONLY).

Sec. III-A has the mapping thread turn keyframe pixels into Gaussian primitives; the paper
gives no formulas, so these follow the readings the library documents:

* ``heuristic_init``: for each inserted pixel (x, y) with depth D at level 0, the mean is the
  back-projection (camera point ((x - cx) / fx D, (y - cy) / fy D, D), world point
  R_cw^T (t - t_cw)); the colour is the pixel's; the log-scale is ln(D / fx) on all three axes,
  the scale whose Eq. 2 footprint f r / d is one pixel; the rotation is the identity; the
  opacity logit is 0 (opacity 0.5); the semantic feature is kappa * code[label] for a label in
  [0, n_classes) when a code table is given, else 0.
* ``patch_features``: the learned initializer's input, the 7 x 7 neighbourhood of the pixel,
  41 channels per neighbour (rgb 3, depth in metres 1 (0 where invalid), one-hot label 32,
  unit ray direction in the camera frame 3, depth-valid flag 1, 1 / fx 1), neighbour-major with
  the neighbours in row-major order (offset dy, then dx, from -3 to 3): 49 x 41 = 2009 features,
  zero-padded to 2048.  Neighbours outside the image contribute zeros.
* ``apply_mlp_init``: the network's standardised outputs back to parameters,
  value = y * std + mean, for the log-scale (outputs 0-2), the opacity logit (3) and the
  semantic feature (4 .. 4 + C - 1).
"""
import numpy as np

PATCH, PATCH_CH, N_IN, N_OUT, N_LABELS = 7, 41, 2048, 32, 32


def heuristic_init(rgb, depth, label, cam, pixels, code=None, kappa=1.0):
    """rgb (3, H, W), depth (H, W), label (H, W) or None, pixels (B, 2) int (x, y),
    code (n_classes, C) or None.  Returns a dict of the new Gaussians' parameters."""
    rgb = np.asarray(rgb, np.float64)
    depth = np.asarray(depth, np.float64)
    pixels = np.asarray(pixels, np.int64)
    R = np.asarray(cam["R_cw"], np.float64).reshape(3, 3)
    t = np.asarray(cam["t_cw"], np.float64).reshape(3)
    xs, ys = pixels[:, 0], pixels[:, 1]
    D = depth[ys, xs]
    D = np.where(D > 0, D, 1.0)  # only valid-depth pixels are inserted; kept finite otherwise
    pc = np.stack([(xs - cam["cx"]) / cam["fx"] * D, (ys - cam["cy"]) / cam["fy"] * D, D], 1)
    mean = (pc - t) @ R            # rows: R^T (p - t)
    B = len(xs)
    ls = np.log(D / cam["fx"])
    out = dict(mean=mean, log_scale=np.repeat(ls[:, None], 3, 1),
               quat=np.tile([1.0, 0.0, 0.0, 0.0], (B, 1)), opacity_logit=np.zeros(B),
               rgb=rgb[:, ys, xs].T.copy())
    if code is not None:
        code = np.asarray(code, np.float64)
        lab = np.asarray(label)[ys, xs] if label is not None else np.full(B, -1)
        ok = (lab >= 0) & (lab < code.shape[0])
        sem = np.zeros((B, code.shape[1]))
        sem[ok] = kappa * code[lab[ok]]
        out["sem"] = sem
    return out


def patch_features(rgb, depth, label, cam, pixels):
    """Learned-initializer input rows, (B, 2048) float64 (before the network's bf16 storage)."""
    rgb = np.asarray(rgb, np.float64)
    depth = np.asarray(depth, np.float64)
    H, W = depth.shape
    pixels = np.asarray(pixels, np.int64)
    X = np.zeros((len(pixels), N_IN))
    for b, (x0, y0) in enumerate(pixels):
        for n in range(PATCH * PATCH):
            x = x0 + n % PATCH - PATCH // 2
            y = y0 + n // PATCH - PATCH // 2
            if not (0 <= x < W and 0 <= y < H):
                continue
            f = X[b, n * PATCH_CH:(n + 1) * PATCH_CH]
            f[0:3] = rgb[:, y, x]
            d = depth[y, x]
            f[3] = d if d > 0 else 0.0
            if label is not None and 0 <= label[y, x] < N_LABELS:
                f[4 + int(label[y, x])] = 1.0
            ray = np.array([(x - cam["cx"]) / cam["fx"], (y - cam["cy"]) / cam["fy"], 1.0])
            f[36:39] = ray / np.linalg.norm(ray)
            f[39] = 1.0 if d > 0 else 0.0
            f[40] = 1.0 / cam["fx"]
    return X


def apply_mlp_init(Y, y_mean, y_std, C):
    """(B, 32) standardised outputs -> log_scale (B, 3), opacity_logit (B,), sem (B, C)."""
    V = np.asarray(Y, np.float64) * np.asarray(y_std, np.float64) + np.asarray(y_mean, np.float64)
    n = min(C, N_OUT - 4)
    sem = np.zeros((V.shape[0], C))
    sem[:, :n] = V[:, 4:4 + n]
    return dict(log_scale=V[:, 0:3].copy(), opacity_logit=V[:, 3].copy(), sem=sem)
