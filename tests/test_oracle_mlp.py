"""Pins of the MLP reference: finite differences of the exact float64 network, and torch
float64 autograd on the same bf16-rounded operands (a library routine)."""
import numpy as np
import pytest
import torch

from oracle import mlp


def small_net(rng, din=24, h=8, dout=5):
    return (rng.normal(size=(h, din)) * 0.3, rng.normal(size=h) * 0.1, rng.normal(size=(h, h)) * 0.3,
            rng.normal(size=h) * 0.1, rng.normal(size=(dout, h)) * 0.3, rng.normal(size=dout) * 0.1)


def test_exact_network_gradients_match_fd():
    rng = np.random.default_rng(0)
    net = small_net(rng)
    X = rng.normal(size=(16, 24))
    T = rng.normal(size=(16, 5))
    w = rng.uniform(0.5, 2.0, size=5)
    L, g, _ = mlp.loss_and_grads(X, T, w, *net, round=False)
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    h = 1e-6
    for k, name in enumerate(names):
        for _ in range(8):
            ix = tuple(rng.integers(0, s) for s in net[k].shape)
            p = [a.copy() for a in net]
            m = [a.copy() for a in net]
            p[k][ix] += h
            m[k][ix] -= h
            fd = (mlp.loss_and_grads(X, T, w, *p, round=False)[0] - mlp.loss_and_grads(X, T, w, *m, round=False)[0]) / (2 * h)
            assert g[name][ix] == pytest.approx(fd, rel=1e-6, abs=1e-9), (name, ix)


def test_rounded_forward_matches_torch_autograd_chain():
    """Same bf16 rounding points, computed by torch float64 ops instead of numpy."""
    rng = np.random.default_rng(1)
    net = small_net(rng, din=64, h=16, dout=8)
    X = mlp.bf16(rng.normal(size=(32, 64)))
    W = [mlp.bf16(a) if a.ndim == 2 else a for a in net]
    H1, H2, Y = mlp.forward(X, *W)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    r = lambda a: a.to(torch.bfloat16).to(torch.float64)
    h1 = r(torch.relu(t(X) @ t(W[0]).T + t(W[1])))
    h2 = r(torch.relu(h1 @ t(W[2]).T + t(W[3])))
    y = h2 @ t(W[4]).T + t(W[5])
    assert np.array_equal(H1, h1.numpy()) and np.array_equal(H2, h2.numpy())
    assert np.allclose(Y, y.numpy(), rtol=1e-13, atol=1e-13)


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to the even 1
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert mlp.bf16(np.array([-3.0]))[0] == -3.0


def test_bf16_rounding_ambiguity_marks_exactly_the_undecided_values():
    """A value at a bf16 midpoint (1 + 2^-8 lies halfway between 1 and 1 + 2^-7) is undecided
    for any band; 1 + 2^-7 (a bf16 value) only for a band reaching the midpoints 2^-8 away;
    after a ReLU, -1 is decided (0) and a value within the band of 0 is not."""
    nb = mlp._near_bf16_boundary
    assert nb(np.array([1 + 2 ** -8]), 1e-12).all()
    assert not nb(np.array([1 + 2 ** -7]), 2 ** -9).any()
    assert nb(np.array([1 + 2 ** -7]), 2 ** -8).all()
    assert nb(np.array([-(3 + 2 ** -7)]), 1e-12).all()          # 3 + 2^-7: a midpoint in the [2, 4) binade
    assert not nb(np.array([-(3 + 2 ** -6)]), 1e-12).any()      # 3 + 2^-6: a bf16 value there
    ru = mlp._relu_bf16_undecided
    assert not ru(np.array([-1.0]), 1e-6).any()
    assert ru(np.array([-1e-7, 1e-7]), 1e-6).all()
    # the band is a rounding band: rounding decided values to bf16 lands on the same bf16 value
    rng = np.random.default_rng(4)
    v = rng.normal(size=20000)
    band = 1e-4 * np.abs(v)
    ok = ~nb(v, band)
    assert ok.mean() > 0.9
    assert np.array_equal(mlp.bf16(v[ok] + band[ok] * 0.999), mlp.bf16(v[ok]))
    assert np.array_equal(mlp.bf16(v[ok] - band[ok] * 0.999), mlp.bf16(v[ok]))


def test_undecided_rows_are_row_local():
    """Changing one row's input or target changes only that row's flag."""
    rng = np.random.default_rng(5)
    W1, b1, W2, b2, W3, b3 = (mlp.bf16(a) for a in small_net(rng, din=64, h=16, dout=8))
    X = mlp.bf16(rng.normal(size=(32, 64)))
    T = rng.normal(size=(32, 8))
    w = np.ones(8)
    und = mlp.undecided_rows(X, T, w, W1, b1, W2, b2, W3, b3, rel=2e-5)
    X2, T2 = X.copy(), T.copy()
    X2[5] = mlp.bf16(rng.normal(size=64))
    T2[9] = rng.normal(size=8)
    und2 = mlp.undecided_rows(X2, T2, w, W1, b1, W2, b2, W3, b3, rel=2e-5)
    keep = np.ones(32, bool)
    keep[[5, 9]] = False
    assert np.array_equal(und[keep], und2[keep])
    assert und.any() and not und.all()
