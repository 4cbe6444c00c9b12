"""FP64 reference of the learned initializer's MLP (TEST INFRASTRUCTURE ONLY).

The network is a 3-layer BF16 MLP with FP32 accumulation: its weights and the activations
passed between layers are bf16 values by definition.  This reference takes the same
bf16-rounded weights, accumulates in float64 (library matmul, one step each) and rounds
the inter-layer tensors to bf16 at exactly the points where the network stores them:
  H1 = bf16(relu(X W1^T + b1)),  H2 = bf16(relu(H1 W2^T + b2)),  Y = H2 W3^T + b3
  L  = sum_o w_o mean_b (Y - T)^2
  dY = bf16(2 w (Y - T) / B),  dH2 = bf16((dY W3) * [H2 > 0]),  dH1 = bf16((dH2 W2) * [H1 > 0])
  dW3 = dY^T H2, dW2 = dH2^T H1, dW1 = dH1^T X, db = column sums of dY, dH2, dH1.
With round=False every bf16 rounding is skipped (the exact float64 network, pinned by
finite differences in the tests).  ``undecided_rows`` marks the batch rows in which a bf16
rounding is not fixed for an FP32-accumulated evaluation (parity compares the other rows
exactly).
"""
import numpy as np
import torch


def bf16(x):
    """Round float64 values to the nearest bf16 (ties to even), returned as float64."""
    return torch.as_tensor(np.asarray(x, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def forward(X, W1, b1, W2, b2, W3, b3, round=True):
    r = bf16 if round else (lambda a: np.asarray(a, np.float64))
    H1 = r(np.maximum(X @ W1.T + b1, 0.0))
    H2 = r(np.maximum(H1 @ W2.T + b2, 0.0))
    Y = H2 @ W3.T + b3
    return H1, H2, Y


def loss_and_grads(X, T, w, W1, b1, W2, b2, W3, b3, round=True):
    r = bf16 if round else (lambda a: np.asarray(a, np.float64))
    B = X.shape[0]
    H1, H2, Y = forward(X, W1, b1, W2, b2, W3, b3, round=round)
    L = float((w[None] * (Y - T) ** 2).sum() / B)
    dY = r(2.0 * w[None] * (Y - T) / B)
    dH2 = r((dY @ W3) * (H2 > 0))
    dH1 = r((dH2 @ W2) * (H1 > 0))
    return L, dict(W1=dH1.T @ X, W2=dH2.T @ H1, W3=dY.T @ H2, b1=dH1.sum(0), b2=dH2.sum(0),
                   b3=dY.sum(0)), dict(H1=H1, H2=H2, Y=Y)


def _near_bf16_boundary(v, band):
    """True where rounding v to bf16 (round to nearest even) is not fixed by a value known only
    to within +-band: v lies within band of a midpoint between two bf16 values (or of 0)."""
    v = np.asarray(v, np.float64)
    a = np.abs(v)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    ulp = np.exp2(e - 7)                      # bf16 keeps 8 significant bits
    q = a / ulp
    mid = (np.floor(q) + 0.5) * ulp           # the midpoint inside [k ulp, (k+1) ulp)
    lower = (np.floor(q) - 0.5) * ulp         # the one below (binade edges included)
    d = np.minimum(np.abs(a - mid), np.abs(a - lower))
    return (d <= band) | (a <= band)


def _relu_bf16_undecided(z, band):
    """The same for bf16(max(z, 0)): the ReLU's decision at 0, then the rounding of z > 0."""
    z = np.asarray(z, np.float64)
    return (np.abs(z) <= band) | ((z > 0) & _near_bf16_boundary(z, band))


def undecided_rows(X, T, w, W1, b1, W2, b2, W3, b3, rel=2.0 ** -22):
    """Rows b of the batch in which some bf16 rounding of the network (H1, H2, dY, dH2, dH1,
    each row depends on its own row only) is not fixed for an evaluation whose dot products
    carry an error up to rel * sum |terms| (2^-22: some 16 times the usual error of an FP32-
    accumulated dot product of these lengths, 2048 terms or fewer): the exact
    pre-rounding value lies within that error of a bf16 rounding midpoint, or of 0 where a
    ReLU decides.  Rows outside the mask have every rounding decided, so any evaluation within
    that error gives exactly this reference's bf16 activations."""
    X, T, w = (np.asarray(a, np.float64) for a in (X, T, w))
    B = X.shape[0]
    z1 = X @ W1.T + b1
    und = _relu_bf16_undecided(z1, rel * (np.abs(X) @ np.abs(W1).T + np.abs(b1))).any(1)
    H1 = bf16(np.maximum(z1, 0.0))
    z2 = H1 @ W2.T + b2
    und |= _relu_bf16_undecided(z2, rel * (H1 @ np.abs(W2).T + np.abs(b2))).any(1)
    H2 = bf16(np.maximum(z2, 0.0))
    Y = H2 @ W3.T + b3
    eY = rel * (H2 @ np.abs(W3).T + np.abs(b3))
    e = 2.0 * w[None] * (Y - T) / B
    # (plus the roundings of the scaled difference itself)
    und |= (_near_bf16_boundary(e, 2.0 * np.abs(w)[None] * eY / B + 2.0 ** -21 * np.abs(e)) & (w[None] != 0)).any(1)
    dY = bf16(e)
    z3 = dY @ W3
    und |= (_near_bf16_boundary(z3, rel * (np.abs(dY) @ np.abs(W3))) & (H2 > 0)).any(1)
    dH2 = bf16(z3 * (H2 > 0))
    z4 = dH2 @ W2
    und |= (_near_bf16_boundary(z4, rel * (np.abs(dH2) @ np.abs(W2))) & (H1 > 0)).any(1)
    return und
