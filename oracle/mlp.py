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
finite differences in the tests).
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
