"""FP64 oracle of the learned surrogate: a plain multilayer perceptron.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and the
benchmark's CPU-baseline leg use it; the CUDA library never does.

The surrogate maps the hand parameters (27 joint angles, 3-D position,
2-D velocity: 32 inputs) to the range-Doppler cube of 3 receive channels x
32 Doppler x 32 range bins (6144 reals: re and im) through

    z_1 = x W_1^T + b_1,  h_1 = relu(z_1)
    z_2 = h_1 W_2^T + b_2, h_2 = relu(z_2)
    z_3 = h_2 W_3^T + b_3, h_3 = relu(z_3)
    y   = h_3 W_4^T + b_4

with W_l stored [out][in] and the loss L = mean over samples and outputs of
(y - t)^2.  The paper has no learned part; this network, its loss and the
AdamW optimiser (Loshchilov & Hutter, "Decoupled Weight Decay
Regularization", ICLR 2019, Algorithm 2) are the build's own choice.

Everything here is written from the definitions: forward as above, the
backward pass by the chain rule (dL/dy = 2 (y - t) / (B O); for a layer
z = h W^T + b: dW = dz^T h, db = sum_b dz, dh = dz W; through relu:
dz = dh * [z > 0]) and AdamW step by step.  Pinned by central finite
differences and closed forms in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

Params = List[Tuple[np.ndarray, np.ndarray]]  # [(W [out][in], b [out])] per layer


def init_params(dims, seed: int) -> Params:
    """He-uniform weights (bound sqrt(6 / in)), zero biases, FP64; seeded."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(dims) - 1):
        n_in, n_out = dims[i], dims[i + 1]
        bound = np.sqrt(6.0 / n_in)
        out.append((rng.uniform(-bound, bound, size=(n_out, n_in)), np.zeros(n_out)))
    return out


def _keep(a):
    return a


def forward(params: Params, x: np.ndarray, store=None):
    """Returns y and the per-layer cache [(h_in, z)] (z = pre-activation).

    store: optional rounding applied where an implementation stores a value
    in a narrower format -- the weights, the network input and every hidden
    activation (the output y stays unrounded); identity by default, so the
    oracle is the exact FP64 definition unless a test asks for the storage
    points of a given precision."""
    r = store or _keep
    h = r(np.asarray(x, np.float64))
    cache = []
    for i, (W, b) in enumerate(params):
        z = h @ r(W).T + b
        cache.append((h, z))
        h = z if i == len(params) - 1 else r(np.maximum(z, 0.0))
    return h, cache


def mse(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def backward(params: Params, x: np.ndarray, t: np.ndarray, store=None):
    """Loss and gradients [(dW, db)] of L = mean((y - t)^2).

    store: as for forward, also applied to every stored gradient dz; the
    ReLU derivative is taken on the stored activation (h > 0, which is
    z > 0 for exact values)."""
    r = store or _keep
    y, cache = forward(params, x, store)
    B, O = y.shape
    dz = r(2.0 * (y - t) / (B * O))
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        h_in, z = cache[i]
        W, _ = params[i]
        grads[i] = (dz.T @ h_in, dz.sum(axis=0))
        if i > 0:
            dh = dz @ r(W)
            dz = r(dh * (cache[i][0] > 0.0))
    return mse(y, t), grads


def adamw_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, step: int, lr: float,
               beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, wd: float = 0.0):
    """One AdamW update (step counts from 1); returns new (p, m, v).

    m = beta1 m + (1 - beta1) g;  v = beta2 v + (1 - beta2) g^2;
    m_hat = m / (1 - beta1^step); v_hat = v / (1 - beta2^step);
    p = p - lr (m_hat / (sqrt(v_hat) + eps) + wd p)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v
