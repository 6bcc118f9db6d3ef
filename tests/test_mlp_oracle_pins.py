"""Pins of the cost-model oracle (CPU): a hand-computed network, central
differences for every gradient entry (independent of the back-propagation
formulas), and Adam's first steps by hand."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_hand_computed_forward():
    # d = 2, h = 2: W1 = [[1, -1], [2, 0.5]], b1 = [0, 1], W2 = [[1, 0], [-1, 2]],
    # b2 = [0.5, -3], w3 = [2, 1], b3 = 0.25
    d, h = 2, 2
    p = np.array([1, -1, 2, 0.5, 0, 1, 1, 0, -1, 2, 0.5, -3, 2, 1, 0.25], dtype=float)
    assert p.size == M.n_params(d, h)
    x = np.array([[1.0, 1.0], [-1.0, 0.5]])
    # row 0: x W1 + b1 = [3, -0.5] + [0, 1] = [3, 0.5] -> relu [3, 0.5]
    #        h1 W2 + b2 = [3 - 0.5, 1] + [0.5, -3] = [3, -2] -> relu [3, 0]
    #        y = 2 * 3 + 0 + 0.25 = 6.25
    # row 1: x W1 + b1 = [-1 + 1, 1 + 0.25] + [0, 1] = [0, 2.25] -> [0, 2.25]
    #        h1 W2 + b2 = [-2.25, 4.5] + [0.5, -3] = [-1.75, 1.5] -> [0, 1.5]
    #        y = 0 + 1.5 + 0.25 = 1.75
    y, h1, h2 = M.forward(p, x, d, h)
    assert y.tolist() == [6.25, 1.75]
    assert h1.tolist() == [[3.0, 0.5], [0.0, 2.25]]
    assert M.loss(p, x, [6.0, 2.0], d, h) == pytest.approx(((0.25) ** 2 + (0.25) ** 2) / 2)


@pytest.mark.parametrize("d,h,B,seed", [(3, 4, 5, 0), (21, 8, 16, 1), (5, 64, 7, 2)])
def test_gradient_matches_central_differences(d, h, B, seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(M.n_params(d, h)) * 0.5
    x = rng.standard_normal((B, d))
    t = rng.standard_normal(B)
    L, g = M.loss_and_grad(p, x, t, d, h)
    gn = M.numerical_grad(p, x, t, d, h)
    assert L == pytest.approx(M.loss(p, x, t, d, h), rel=1e-14)
    # away from relu kinks the central difference is accurate to ~1e-8
    np.testing.assert_allclose(g, gn, rtol=1e-5, atol=1e-7)


def test_adam_first_steps_by_hand():
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    eps = 1e-8
    p1, m1, v1 = M.adam(p, g, m, v, 1, lr=0.1, eps=eps)
    # step 1: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    step = 0.1 * g / (np.abs(g) + eps)
    assert p1 == pytest.approx(p - step, abs=1e-15)
    assert m1 == pytest.approx([0.05, -0.025])
    assert v1 == pytest.approx([0.00025, 0.0000625])
    p2, m2, v2 = M.adam(p1, g, m1, v1, 2, lr=0.1, eps=eps)
    # constant gradient: m_hat = g and v_hat = g^2 again
    assert p2 == pytest.approx(p - 2 * step, abs=1e-15)


def test_training_reduces_the_loss_on_a_smooth_target():
    rng = np.random.default_rng(3)
    d, h = 4, 16
    x = rng.uniform(-1, 1, (128, d))
    t = np.sin(x[:, 0]) + x[:, 1] * x[:, 2]
    p = rng.standard_normal(M.n_params(d, h)) * 0.3
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = M.loss(p, x, t, d, h)
    for k in range(1, 301):
        _, g = M.loss_and_grad(p, x, t, d, h)
        p, m, v = M.adam(p, g, m, v, k, lr=1e-2)
    assert M.loss(p, x, t, d, h) < 0.1 * L0
