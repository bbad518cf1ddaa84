"""Pins of the oracle's gradient regularisers (Sec. III-E): dynamic scaling
and normalisation of whole adjoint vectors, with the paper's constants
(oom* = 4, delta = 1e-6, clip 1e4), as closed forms on single vectors and
as invariances of the full adjoint (identity when no vector exceeds oom*,
independence of the seed's magnitude)."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))["gradient_ops"]


def _p(**kw):
    return oracle.Params(oom_star=GOLD["oom_star"], grad_delta=GOLD["delta"], clip_value=GOLD["clip"], **kw)


def test_dynamic_scaling_closed_form():
    p = _p(grad_scale=1)
    g = np.array([3.7e7, -2.0, 5.0e3, -1.2e7])
    out = oracle.grad_op(p, g)
    # round(log10 3.7e7) = 8 -> doom = 4 -> divide by 1e4 + delta
    assert np.array_equal(out, g / (1e4 + 1e-6))
    assert np.abs(out).max() < 10 ** (GOLD["oom_star"] + 0.5)
    # already within the order: unchanged (round(log10 5e3) = 4, doom = 0)
    small = np.array([5.0e3, -1.0, 2.0])
    assert np.array_equal(oracle.grad_op(p, small), small)
    # and a zero vector stays zero
    assert np.array_equal(oracle.grad_op(p, np.zeros(5)), np.zeros(5))


def test_normalisation_closed_form():
    p = _p(grad_scale=2)
    g = np.array([3.0, 4.0, 0.0, -12.0])
    out = oracle.grad_op(p, g)
    assert np.allclose(out, g / (13.0 + 1e-6), rtol=0, atol=1e-15)
    assert abs(np.linalg.norm(out) - 13.0 / (13.0 + 1e-6)) < 1e-15


def test_clip_closed_form():
    p = _p(clip_grads=1)
    g = np.array([2e4, -3e4, 5.0, -9999.0])
    assert np.array_equal(oracle.grad_op(p, g), np.array([1e4, -1e4, 5.0, -9999.0]))


def _scenario():
    from paper_2510_17335_gb300 import workloads as W
    from _common import oracle_params, oracle_poses
    res, dx = 16, 1.0 / 16
    x0 = W.lattice_bed(41, (4, 3, 4), (6 * dx, 3 * dx, 6 * dx), dx)
    acts = np.zeros((3, 6))
    acts[:, 0] = 0.004
    acts[:, 1] = -0.003
    w = W.Workload("gops", (res,) * 3, dx, 2e-4, 6, 1e5, 0.3, 1500.0, 30.0, dx ** 3 / 8, x0,
                   W.Trajectory((7.2 * dx, 5.3 * dx, 8.1 * dx, 0.1), 2, actions=acts), shovel_half=(0.02, 0.06, 0.08))
    n = w.n
    rng = np.random.default_rng(5)
    F = np.tile(np.eye(3).ravel(), (n, 1)) + 0.01 * rng.normal(size=(n, 9))
    v = 0.05 * rng.normal(size=(n, 3))
    C = 0.2 * rng.normal(size=(n, 9))
    seed = (np.array([1.0, -0.5, 0.3]) + 0.1 * rng.normal(size=(n, 3))) / n
    return w, oracle_params, oracle_poses(w, 6), (w.x0.astype(np.float64), v, C, F), seed


def _adjoint(p, w, poses, st, gx):
    n = w.n
    s, g = oracle.rollout_adjoint(p, st[0], st[1], st[2], st[3], poses, gx=gx, gv=np.zeros((n, 3)))
    assert s == 0
    return g


def test_dynamic_scaling_is_identity_below_the_order():
    w, op, poses, st, seed = _scenario()
    base = op(w)
    g0 = _adjoint(base, w, poses, st, seed)
    p = op(w)
    p.grad_scale, p.oom_star = 1, 100.0          # no vector reaches 1e100
    g1 = _adjoint(p, w, poses, st, seed)
    for k in ("x", "v", "C", "F", "material"):
        assert np.array_equal(g0[k], g1[k]), k


def test_dynamic_scaling_is_decade_equivariant():
    """Seeds 10^6 and 10^7 times larger both exceed oom* = 4 and are scaled
    back by their own decade: the results agree (to delta)."""
    w, op, poses, st, seed = _scenario()
    p = op(w)
    p.grad_scale, p.oom_star, p.grad_delta = 1, GOLD["oom_star"], GOLD["delta"]
    unit = seed / np.abs(seed).max() * 3.0      # max |seed| = 3: order 0
    a = _adjoint(p, w, poses, st, unit * 1e6)
    b = _adjoint(p, w, poses, st, unit * 1e7)
    for k in ("x", "v", "C", "F", "material"):
        scale = np.abs(a[k]).max()
        assert np.abs(a[k] - b[k]).max() <= 1e-8 * scale, k


def test_normalisation_is_independent_of_the_seed_magnitude():
    w, op, poses, st, seed = _scenario()
    p = op(w)
    p.grad_scale, p.grad_delta = 2, GOLD["delta"]
    a = _adjoint(p, w, poses, st, seed)
    b = _adjoint(p, w, poses, st, seed * 1e3)
    for k in ("x", "v", "C", "F", "material"):
        scale = np.abs(a[k]).max()
        assert scale > 0
        assert np.abs(a[k] - b[k]).max() <= 1e-4 * scale, k
    # and differs from the plain adjoint
    g0 = _adjoint(op(w), w, poses, st, seed)
    assert not np.allclose(g0["F"], a["F"], rtol=1e-3)
