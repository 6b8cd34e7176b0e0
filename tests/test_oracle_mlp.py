"""Pins of the CPU reference network used to check the GPU training
kernels of the warm-start extension."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding():
    assert mlp.bf16(1.0) == 1.0
    # 1 + 2^-8 is exactly halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert mlp.bf16(-3.0) == -3.0
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    sizes = (5, 7, 6, 3)
    params = mlp.init_params(2, sizes)
    params = [(W, rng.normal(size=b.shape) * 0.1) for W, b in params]
    X = rng.normal(size=(11, 5))
    T = rng.normal(size=(11, 3))
    loss, grads = mlp.loss_and_grads(params, X, T, round_bf16=False)
    eps = 1e-6
    for l in range(len(params)):
        W, b = params[l]
        for _ in range(5):
            i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += eps
            Wm[i, j] -= eps
            pp = list(params)
            pp[l] = (Wp, b)
            lp, _ = mlp.loss_and_grads(pp, X, T, round_bf16=False)
            pp[l] = (Wm, b)
            lm, _ = mlp.loss_and_grads(pp, X, T, round_bf16=False)
            assert grads[l][0][i, j] == pytest.approx((lp - lm) / (2 * eps), rel=1e-5, abs=1e-9)
        k = rng.integers(b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[k] += eps
        bm[k] -= eps
        pp = list(params)
        pp[l] = (W, bp)
        lp, _ = mlp.loss_and_grads(pp, X, T, round_bf16=False)
        pp[l] = (W, bm)
        lm, _ = mlp.loss_and_grads(pp, X, T, round_bf16=False)
        assert grads[l][1][k] == pytest.approx((lp - lm) / (2 * eps), rel=1e-5, abs=1e-9)


def test_linear_network_closed_form():
    """One layer, no activation: y = x W^T + b, L = |y - t|^2 / (N n),
    dL/dW = 2 (y - t)^T x / (N n)."""
    rng = np.random.default_rng(3)
    W = rng.normal(size=(2, 4))
    b = rng.normal(size=2)
    X = rng.normal(size=(9, 4))
    T = rng.normal(size=(9, 2))
    loss, grads = mlp.loss_and_grads([(W, b)], X, T, round_bf16=False)
    Y = X @ W.T + b
    np.testing.assert_allclose(grads[0][0], 2 * (Y - T).T @ X / 18, rtol=1e-12)
    np.testing.assert_allclose(grads[0][1], 2 * (Y - T).sum(0) / 18, rtol=1e-12)
    assert loss == pytest.approx(np.mean((Y - T) ** 2))
