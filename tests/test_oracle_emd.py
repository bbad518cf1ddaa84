"""Pins of the oracle's Earth Mover's distance (Eq. (1)): brute force over
all one-to-one maps on tiny sets, the metric's identities, the rectangular
case |X| < |Xhat|, and the gradient against finite differences."""
import itertools

import numpy as np

import oracle


def _brute(X, Y):
    best = None
    for perm in itertools.permutations(range(Y.shape[0]), X.shape[0]):
        c = np.linalg.norm(X - Y[list(perm)], axis=1).sum()
        best = c if best is None or c < best else best
    return best


def test_brute_force_on_tiny_sets():
    rng = np.random.default_rng(1)
    for n, m in ((3, 3), (5, 5), (4, 6), (6, 7)):
        X, Y = rng.normal(size=(n, 3)), rng.normal(size=(m, 3))
        d, phi, _ = oracle.emd(X, Y)
        assert abs(d - _brute(X, Y)) < 1e-12
        assert len(set(phi)) == n and phi.min() >= 0 and phi.max() < m


def test_identities():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(50, 3))
    assert oracle.emd(X, X)[0] == 0.0
    # permutation of the target: still 0
    assert oracle.emd(X, X[rng.permutation(50)])[0] == 0.0
    # symmetric for equal sizes
    Y = rng.normal(size=(50, 3))
    assert abs(oracle.emd(X, Y)[0] - oracle.emd(Y, X)[0]) < 1e-10
    # a far translation: every point pays the translation, d = n |t| - O(spread)
    t = np.array([100.0, 0.0, 0.0])
    d = oracle.emd(X, X + t)[0]
    assert abs(d - 50 * 100.0) < 50 * 2 * np.abs(X).max()


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(3)
    X, Y = rng.normal(size=(12, 3)), rng.normal(size=(15, 3))
    d, phi, g = oracle.emd(X, Y)
    h = 1e-6
    for i in range(12):
        for k in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, k] += h
            Xm[i, k] -= h
            dp, phip, _ = oracle.emd(Xp, Y)
            dm, phim, _ = oracle.emd(Xm, Y)
            if not (np.array_equal(phip, phi) and np.array_equal(phim, phi)):
                continue       # the assignment changes within h: not differentiable there
            assert abs((dp - dm) / (2 * h) - g[i, k]) < 1e-6
