"""Pins of the surrogate network's FP64 reference: the convolution against a
library cross-correlation, gradients against finite differences of the
loss, Adam against its defining recursion, and bfloat16 rounding."""
import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_scipy_correlate():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 9, 11))
    w = rng.normal(size=(4, 3, 5, 5))
    b = rng.normal(size=4)
    y = cnn.conv2d(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = b[co] + sum(scipy_signal.correlate2d(x[n, ci], w[co, ci], mode="same", boundary="fill")
                              for ci in range(3))
            assert np.allclose(y[n, co], ref, rtol=1e-12, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = cnn.init_params(seed=2, channels=(3, 4, 4, 3))
    x = rng.normal(size=(2, 3, 7, 6))
    t = rng.normal(size=(2, 3, 7, 6))

    def loss(P, xx):
        y, _ = cnn.forward(P, xx)
        return cnn.mse(y, t)[0]

    y, cache = cnn.forward(params, x)
    L, dy = cnn.mse(y, t)
    grads, dx = cnn.backward(params, cache, dy)
    eps = 1e-6
    for li in range(len(params)):
        for key in ("w", "b"):
            arr = params[li][key]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = loss(params, x)
                flat[idx] = old - eps
                lm = loss(params, x)
                flat[idx] = old
                num = (lp - lm) / (2 * eps)
                assert abs(num - grads[li][key].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(num))
    fx = x.reshape(-1)
    for idx in rng.choice(fx.size, size=6, replace=False):
        old = fx[idx]
        fx[idx] = old + eps
        lp = loss(params, x)
        fx[idx] = old - eps
        lm = loss(params, x)
        fx[idx] = old
        assert abs((lp - lm) / (2 * eps) - dx.reshape(-1)[idx]) <= 1e-6


def test_adam_first_step_moves_by_lr():
    # with bias correction the first step is lr * g/|g| per element (eps -> 0)
    params = [{"w": np.array([1.0, -2.0]), "b": np.array([0.5])}]
    grads = [{"w": np.array([0.3, -4.0]), "b": np.array([0.0])}]
    st = cnn.adam_init(params)
    cnn.adam_step(params, grads, st, lr=0.01, eps=1e-12)
    assert np.allclose(params[0]["w"], [1.0 - 0.01, -2.0 + 0.01], rtol=0, atol=1e-9)
    assert params[0]["b"][0] == 0.5


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -3.14159, 0.0])
    r = cnn.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == 1.0 + 2 * 2 ** -7        # tie -> even (up)
    assert abs(r[4] + 3.140625) < 1e-12
    assert r[5] == 0.0


def test_training_reduces_loss_on_a_linear_target():
    """A few Adam steps on a fixed linear target (a 3x3 blur) reduce the loss:
    the recursion, backward pass and update wire together."""
    rng = np.random.default_rng(3)
    params = cnn.init_params(seed=4, channels=(3, 8, 3))
    x = rng.normal(size=(4, 3, 12, 12))
    k = np.zeros((3, 3, 5, 5))
    for c in range(3):
        k[c, c, 1:4, 1:4] = 1.0 / 9
    t = cnn.conv2d(x, k, np.zeros(3))
    st = cnn.adam_init(params)
    losses = []
    for _ in range(60):
        y, cache = cnn.forward(params, x)
        L, dy = cnn.mse(y, t)
        losses.append(L)
        g, _ = cnn.backward(params, cache, dy)
        cnn.adam_step(params, g, st, lr=3e-3)
    assert losses[-1] < 0.3 * losses[0]
