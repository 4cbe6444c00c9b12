"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

import oracle

# Relative errors of the kernels' float32 alpha = o exp(-sigma) (from the float32 projection
# records) and of their float32 transmittance T, measured on GB300 at 4.6e-6 (12k pixels of
# isolated Gaussians) and 5.4e-6 (40k pixels of the dense room), about half and a quarter of
# these bounds; test_gpu_parity.py::test_float32_alpha_and_transmittance_errors_are_within_the_bands
# checks them at every run.  The oracle flags a skip / clamp decision within ALPHA_TOL of its
# threshold and a stop decision within T_TOL of T_min.
ALPHA_TOL = 1e-5
T_TOL = 2e-5
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
    """The oracle's render with the ambiguity bands of the float32 alpha and transmittance."""
    return oracle.render(g, cam, cfg, pixels=pixels, tol=ALPHA_TOL, tol_T=T_TOL)


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
