"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

import oracle

# Relative error of a float32 alpha = o exp(-sigma) evaluated from the float32 projection
# records (bounded on GB300 by test_gpu_parity.py::test_alpha_float32_error_is_within_the_band).
# The oracle's ambiguity flags are derived from it: a skip / clamp decision within this band
# of its threshold, or a stop decision within the transmittance error it propagates to.
ALPHA_TOL = 2e-5
# Forward tolerance per pixel and channel: |g - o| <= 1e-4 |o| + 1e-5.
FWD_REL, FWD_ABS = 1e-4, 1e-5
# Gradient tolerance per element: |g - o| <= 2e-3 |o| + 1e-6 max|o| of the parameter group.
GRAD_REL, GRAD_FLOOR = 2e-3, 1e-6

# Pixels where a decision of the method is not fixed for a float32 evaluation (skip, stop,
# undecided depth order; for gradients also the clamp, whose derivative is one-sided).
AMBIGUOUS = oracle.FLAG_SKIP | oracle.FLAG_STOP | oracle.FLAG_DEPTH
AMBIGUOUS_GRAD = AMBIGUOUS | oracle.FLAG_CLAMP
# Largest share of pixels a parity test may mask as ambiguous.
MAX_MASKED = 1e-3


def ref_render(g, cam, cfg=None, pixels=None):
    """The oracle's render with the ambiguity band of a float32 alpha."""
    return oracle.render(g, cam, cfg, pixels=pixels, tol=ALPHA_TOL)


def unambiguous(flags, bits=AMBIGUOUS, limit=MAX_MASKED):
    """Mask of the pixels whose decisions are fixed; asserts the masked share is below limit."""
    amb = (np.asarray(flags) & bits) != 0
    assert amb.mean() <= limit, f"{amb.mean():.2e} of the pixels are ambiguous (limit {limit:.0e})"
    return ~amb


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
