"""Pins of the oracle's MSE loss of final positions (the differentiable-rollout
workload's loss: L = (1/N) sum_p |x_p - xhat_p|^2 over the N particles, the
mean over particles of the squared Euclidean distance), against values
worked out by hand and against central differences of the loss itself."""
import numpy as np
import pytest

import oracle


def test_mse_hand_cases():
    # two particles, offsets (1, 0, 0) and (0, 2, 0) from the target:
    # squared distances 1 and 4, mean 2.5 (a 1/(3N) normalisation gives
    # 5/6, a plain sum 5, a mean distance 1.5)
    x = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    L, g = oracle.mse_loss(x, np.zeros((2, 3)))
    assert L == 2.5
    # dL/dx_p = 2 (x_p - xhat_p) / N: (1, 0, 0) and (0, 2, 0)
    np.testing.assert_array_equal(g, [[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    # one particle at distance 3 along a diagonal direction: L = 9
    L1, g1 = oracle.mse_loss([[1.0, 2.0, 2.0]], [[0.0, 0.0, 0.0]])
    assert L1 == 9.0
    np.testing.assert_array_equal(g1, [[2.0, 4.0, 4.0]])
    # coinciding clouds: zero loss and gradient
    L0, g0 = oracle.mse_loss(x, x)
    assert L0 == 0.0 and not g0.any()


def test_mse_sign_and_translation():
    rng = np.random.default_rng(11)
    x, t = rng.normal(size=(50, 3)), rng.normal(size=(50, 3))
    L, g = oracle.mse_loss(x, t)
    # the loss only sees the offsets x - xhat
    s = rng.normal(size=3)
    Ls, gs = oracle.mse_loss(x + s, t + s)
    assert Ls == pytest.approx(L, rel=1e-14)
    np.testing.assert_allclose(gs, g, rtol=1e-12, atol=1e-15)
    # a step against the gradient lowers the loss (sign of dL/dx)
    Ld, _ = oracle.mse_loss(x - 1e-3 * g, t)
    assert Ld < L
    # moving every particle onto its target by a fraction f scales L by (1 - f)^2
    Lf, _ = oracle.mse_loss(x - 0.25 * (x - t), t)
    assert Lf == pytest.approx(0.5625 * L, rel=1e-13)


def test_mse_gradient_central_differences():
    rng = np.random.default_rng(12)
    x, t = rng.normal(size=(7, 3)), rng.normal(size=(7, 3))
    _, g = oracle.mse_loss(x, t)
    h = 1e-6
    fd = np.zeros_like(x)
    for p in range(x.shape[0]):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[p, k] += h
            xm[p, k] -= h
            fd[p, k] = (oracle.mse_loss(xp, t)[0] - oracle.mse_loss(xm, t)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-9)
