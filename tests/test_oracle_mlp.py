"""Pins of the FP64 surrogate oracle (oracle/mlp.py): central finite
differences of the loss against every analytic gradient, closed forms of a
linear layer and of the first AdamW step, and ReLU special cases."""
import numpy as np
import pytest

from oracle import mlp


def _net(dims, seed):
    p = mlp.init_params(dims, seed)
    rng = np.random.default_rng(seed + 1)
    # non-zero biases so that a dropped bias term shows
    return [(W, rng.normal(0, 0.1, size=b.shape)) for W, b in p]


@pytest.mark.parametrize("dims", [(3, 5, 2), (4, 6, 7, 3), (5, 8, 8, 8, 6)])
def test_gradients_match_central_differences(dims):
    params = _net(dims, 3)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(4, dims[0]))
    t = rng.normal(size=(4, dims[-1]))
    _, grads = mlp.backward(params, x, t)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.mse(mlp.forward(params, x)[0], t)
                arr[idx] = old - h
                lm = mlp.mse(mlp.forward(params, x)[0], t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-7 + 1e-5 * abs(fd), (li, idx, fd, g[idx])


def test_single_linear_layer_closed_form():
    """One layer y = x W^T + b: dL/dW = 2 (y - t)^T x / (B O), dL/db =
    2 sum_b (y - t) / (B O); the optimum of a consistent system has zero
    gradient."""
    rng = np.random.default_rng(1)
    W = rng.normal(size=(3, 4))
    b = rng.normal(size=3)
    x = rng.normal(size=(5, 4))
    t = x @ W.T + b
    loss, g = mlp.backward([(W, b)], x, t)
    assert loss == 0.0 and np.all(g[0][0] == 0) and np.all(g[0][1] == 0)
    t2 = t + 1.0  # every output off by one: y - t = -1
    loss, g = mlp.backward([(W, b)], x, t2)
    assert loss == pytest.approx(1.0)
    np.testing.assert_allclose(g[0][1], np.full(3, -2.0 * 5 / 15))
    np.testing.assert_allclose(g[0][0], np.tile(-2.0 * x.sum(axis=0) / 15, (3, 1)))


def test_relu_blocks_gradient_of_inactive_units():
    """Hidden units whose pre-activation is negative for every sample pass
    no gradient: their incoming weights and biases get exactly zero."""
    params = _net((3, 4, 2), 5)
    W1, b1 = params[0]
    b1[:2] = -1e3  # units 0 and 1 never fire
    rng = np.random.default_rng(2)
    x = rng.normal(size=(6, 3))
    t = rng.normal(size=(6, 2))
    _, g = mlp.backward(params, x, t)
    assert np.all(g[0][0][:2] == 0) and np.all(g[0][1][:2] == 0)
    assert np.any(g[0][0][2:] != 0)
    # and the outgoing weights of dead units see zero activations
    assert np.all(g[1][0][:, :2] == 0)


def test_forward_shapes_and_relu_on_hidden_layers_only():
    params = _net((2, 3, 2), 0)
    x = np.array([[1.0, -2.0]])
    y, cache = mlp.forward(params, x)
    (W1, b1), (W2, b2) = params
    h1 = np.maximum(x @ W1.T + b1, 0)
    np.testing.assert_allclose(y, h1 @ W2.T + b2)  # output layer is linear
    assert cache[1][0].shape == (1, 3)


def test_adamw_first_step_closed_form():
    """At step 1 the bias-corrected moments are m_hat = g, v_hat = g^2, so
    the update is lr (g / (|g| + eps) + wd p): a step of lr sign(g) for
    |g| >> eps, plus the decoupled decay."""
    p = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, 0.0])
    m0 = np.zeros(4)
    v0 = np.zeros(4)
    lr, wd, eps = 0.01, 0.1, 1e-8
    p1, m1, v1 = mlp.adamw_step(p, g, m0, v0, 1, lr, wd=wd, eps=eps)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)
    expect = p - lr * (g / (np.abs(g) + eps) + wd * p)
    np.testing.assert_allclose(p1, expect, rtol=1e-12)
    assert p1[3] == pytest.approx(3.0 - lr * wd * 3.0)  # zero gradient: decay only


def test_adamw_two_steps_by_hand():
    p, g1, g2 = 0.5, 0.2, -0.1
    b1, b2, lr = 0.9, 0.999, 0.1
    pa, m, v = mlp.adamw_step(np.array([p]), np.array([g1]), np.zeros(1), np.zeros(1), 1, lr)
    pb, m, v = mlp.adamw_step(pa, np.array([g2]), m, v, 2, lr)
    m2 = b1 * (1 - b1) * g1 + (1 - b1) * g2
    v2 = b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2
    step2 = lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + 1e-8)
    assert pb[0] == pytest.approx(pa[0] - step2, rel=1e-12)


def test_init_is_seeded_and_he_bounded():
    a = mlp.init_params((32, 64, 16), 4)
    b = mlp.init_params((32, 64, 16), 4)
    assert all(np.array_equal(x[0], y[0]) for x, y in zip(a, b))
    assert np.abs(a[0][0]).max() <= np.sqrt(6 / 32) and np.abs(a[1][0]).max() <= np.sqrt(6 / 64)
    assert a[0][0].shape == (64, 32) and np.all(a[0][1] == 0)
