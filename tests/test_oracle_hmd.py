"""Pins of the oracle's surface observation, height map and height-map
distance (Sec. III-A, "States and observations"; Eq. (2)) against what the
paper and the definitions fix: the paper's 1600-point observation of its
initial body, single-particle and stacked cases, the tie rule, the 5-tap
cross, exact distances of shifted maps and the piecewise-linear gradient."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _grid(res=8, size=0.08, tap=0.0, c=(0.5, 0.5)):
    return oracle.ObsGrid(c[0], c[1], size, res, tap)


def _centre(g, i, j):
    h = g.size / g.res
    return g.cx - 0.5 * g.size + (i + 0.5) * h, g.cz - 0.5 * g.size + (j + 0.5) * h


def test_paper_initial_body_observation_has_1600_points():
    """Sec. III-A: the observation of the flattened body (0.28 x 0.28 x 0.07 m
    at 5e6 per m^3) over a 40 x 40 grid of 0.24 m holds 1600 particles."""
    ib, og = GOLD["initial_body"], GOLD["observation_grid"]
    x, _ = W.paper_bed(density=ib["density_per_m3"], size=(ib["box_m"][0], ib["box_m"][2], ib["box_m"][1]))
    assert x.shape[0] == ib["n_particles"]
    g = oracle.ObsGrid(0.14, 0.14, og["size_m"], og["cells"], 0.0)   # the box spans [0, 0.28] in x and z
    n, idx = oracle.surface_observation(g, x)
    assert n == og["n_points"] == g.res * g.res
    # each chosen particle is in its pixel and no particle of that pixel is higher
    h = np.float32(g.size / g.res)
    x0 = np.float32(g.cx - 0.5 * g.size)
    pi = np.floor((x[:, 0] - x0) / h).astype(np.int64)
    pj = np.floor((x[:, 2] - x0) / h).astype(np.int64)
    for p in range(g.res * g.res):
        members = np.nonzero((pi == p // g.res) & (pj == p % g.res))[0]
        assert idx[p] in members
        assert x[idx[p], 1] == x[members, 1].max()


def test_single_particle_and_stack():
    g = _grid()
    cx, cz = _centre(g, 3, 5)
    x = np.array([[cx, 0.1, cz]], np.float32)
    n, idx = oracle.surface_observation(g, x)
    assert n == 1 and idx[3 * g.res + 5] == 0 and (idx >= 0).sum() == 1
    # a column of particles: the highest is observed
    ys = np.array([0.05, 0.2, 0.12, 0.19], np.float32)
    col = np.stack([np.full(4, cx), ys, np.full(4, cz)], 1).astype(np.float32)
    n, idx = oracle.surface_observation(g, col)
    assert idx[3 * g.res + 5] == 1


def test_equal_heights_keep_the_lowest_index():
    g = _grid()
    cx, cz = _centre(g, 2, 2)
    x = np.array([[cx, 0.1, cz], [cx + 1e-4, 0.1, cz], [cx, 0.1, cz + 1e-4]], np.float32)
    for perm in ([0, 1, 2], [2, 0, 1], [1, 2, 0]):
        _, idx = oracle.surface_observation(g, x[perm])
        assert idx[2 * g.res + 2] == 0   # lowest index of the permuted list
        I, w = oracle.height_map(g, x[perm])
        assert w[2, 2] == 0


def test_outside_points_are_ignored():
    g = _grid()
    x = np.array([[g.cx - 0.6 * g.size, 0.3, g.cz], [g.cx, 0.3, g.cz + 0.51 * g.size]], np.float32)
    n, idx = oracle.surface_observation(g, x)
    assert n == 0 and (idx < 0).all()
    I, w = oracle.height_map(g, x)
    assert (I == 0).all() and (w < 0).all()


def test_tap_cross():
    """One particle at a pixel centre with the tap one pixel wide covers the
    plus-shaped 5 pixels around it, at its height."""
    g = _grid(tap=0.01)          # pixel 0.01
    cx, cz = _centre(g, 4, 4)
    x = np.array([[cx, 0.25, cz]], np.float32)
    I, w = oracle.height_map(g, x)
    want = {(4, 4), (5, 4), (3, 4), (4, 5), (4, 3)}
    got = {tuple(p) for p in np.argwhere(I > 0)}
    assert got == want
    assert np.all(I[tuple(np.array(sorted(want)).T)] == np.float32(0.25))
    # without a tap only its own pixel
    I0, _ = oracle.height_map(_grid(), x)
    assert {tuple(p) for p in np.argwhere(I0 > 0)} == {(4, 4)}


def test_zero_tap_height_map_is_the_observation():
    g = _grid(res=10, size=0.1)
    x = np.random.default_rng(1).uniform(0.45, 0.55, (3000, 3)).astype(np.float32)
    x[:, 1] = np.random.default_rng(2).uniform(0.05, 0.3, 3000).astype(np.float32)
    _, idx = oracle.surface_observation(g, x)
    I, w = oracle.height_map(g, x)
    assert np.array_equal(w.reshape(-1), idx)
    assert np.array_equal(I.reshape(-1)[idx >= 0], x[idx[idx >= 0], 1].astype(np.float64))


def test_hmd_of_shifted_bed_is_exact():
    """Raising every particle by delta (exactly representable) raises every
    covered pixel by delta: d_HMD = delta * covered pixels, gradient +1 at
    each pixel's winner."""
    g = oracle.ObsGrid(0.5, 0.5, 0.08, 16, 0.002)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.46, 0.54, (4000, 3)).astype(np.float32)
    x[:, 1] = np.float32(0.125) + np.float32(0.0625) * rng.integers(0, 4, 4000).astype(np.float32)
    Ihat, w = oracle.height_map(g, x)
    assert oracle.hmd(g, x, Ihat)[0] == 0.0
    up = x.copy()
    up[:, 1] += np.float32(0.25)
    L, grad = oracle.hmd(g, up, Ihat)
    covered = int((Ihat > 0).sum())
    assert L == 0.25 * covered
    assert grad[:, 0].sum() == 0 and grad[:, 2].sum() == 0
    assert grad[:, 1].sum() == covered
    # symmetric: the reverse distance is the same
    Iup, _ = oracle.height_map(g, up)
    assert oracle.hmd(g, x, Iup)[0] == L


def test_hmd_gradient_matches_finite_differences():
    """d_HMD is piecewise linear in the heights: away from ties a small
    change of one particle's height changes the distance by the sum of the
    signs of the pixels it wins."""
    g = oracle.ObsGrid(0.5, 0.5, 0.06, 12, 0.003)
    rng = np.random.default_rng(4)
    x = rng.uniform(0.472, 0.528, (600, 3)).astype(np.float32)
    x[:, 1] = rng.uniform(0.1, 0.2, 600).astype(np.float32)
    Ihat = rng.uniform(0.1, 0.2, (g.res, g.res))
    L, grad = oracle.hmd(g, x, Ihat)
    I, w = oracle.height_map(g, x)
    winners = np.unique(w[w >= 0])
    checked = 0
    for q in winners[:40]:
        # gap to the next height in the pixels q wins, and to the target
        eps = np.float32(1e-6)
        if np.min(np.abs(I[w == q] - Ihat[w == q])) < 1e-5:
            continue
        for sgn in (1, -1):
            xp = x.copy()
            xp[q, 1] += sgn * eps
            Lp, _ = oracle.hmd(g, xp, Ihat)
            fd = (Lp - L) / (float(xp[q, 1]) - float(x[q, 1]))
            assert abs(fd - grad[q, 1]) < 1e-3, (q, fd, grad[q, 1])
        checked += 1
    assert checked > 20
    # particles that win nothing have no gradient
    losers = np.setdiff1d(np.arange(x.shape[0]), winners)
    assert np.all(grad[losers] == 0)
