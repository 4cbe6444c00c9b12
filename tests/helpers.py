"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

import oracle

# Forward tolerance per pixel and channel: |g - o| <= 1e-4 |o| + 1e-5.
FWD_REL, FWD_ABS = 1e-4, 1e-5
# Gradient tolerance per element: |g - o| <= 2e-3 |o| + floor, floor = 1e-5 * max|o| of the
# parameter group (FP32 atomics sum hundreds of signed terms in arbitrary order; the floor
# is the size of that summation's rounding relative to the group's largest entry).
GRAD_REL, GRAD_FLOOR = 2e-3, 1e-5

# Depth order is decided on the same float32 key on both sides (no ambiguity left there).
AMBIGUOUS = oracle.FLAG_SKIP | oracle.FLAG_STOP
AMBIGUOUS_GRAD = AMBIGUOUS | oracle.FLAG_CLAMP


def check_close(name, got, ref, rel, abs_, mask=None):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    tol = rel * np.abs(ref) + abs_
    bad = err > tol
    if mask is not None:
        bad &= np.broadcast_to(mask, bad.shape)
    if bad.any():
        idx = np.argwhere(bad)[:5]
        detail = ", ".join(f"{tuple(i)}: got {got[tuple(i)]:.8g} ref {ref[tuple(i)]:.8g}" for i in idx)
        raise AssertionError(f"{name}: {int(bad.sum())} / {bad.size} entries out of tolerance; {detail}")


def check_grads(got: dict, ref: dict, keys, rel=GRAD_REL, floor=GRAD_FLOOR):
    for k in keys:
        r = np.asarray(ref[k], np.float64)
        scale = np.abs(r).max() if r.size else 0.0
        check_close(f"grad[{k}]", got[k], r, rel, floor * scale + 1e-12)
