"""Host logic of the system-identification loop and of its workload, on the
CPU: the parameter ranges and step sizes of Sec. IV-B, the clamping of
candidates into the ranges, the error measure on the free parameters, and
the bed and scripted trajectory of the batched identification workload."""
import numpy as np

from paper_2510_17335_gb300 import sysid
from paper_2510_17335_gb300 import workloads as W


def test_constants_follow_the_paper():
    assert sysid.STEP == (1e4, 0.01, 50.0, 1.0)
    assert sysid.ALPHAS == (0.1, 0.5, 1.0, 1.5, 2.0)
    assert sysid.BETA == 0.9
    lo, hi = zip(*sysid.RANGES)
    assert all(a < b for a, b in zip(lo, hi))


def test_clamp_keeps_candidates_in_the_ranges():
    t = np.array([[1e6, -1.0, 1e4, 5.0], [6e4, 0.2, 1500.0, 30.0]])
    c = sysid._clamp(t)
    assert np.allclose(c[0], [2e5, 0.1, 2200.0, 10.0])
    assert np.array_equal(c[1], t[1])


def test_error_counts_only_the_free_parameters():
    truth = np.array([1e5, 0.3, 1500.0, 30.0])
    theta = np.array([[1.1e5, 0.6, 1500.0, 30.0], [1e5, 0.3, 3000.0, 31.5]])
    free = np.array([True, False, False, True])
    e = sysid._rel_error(theta, truth, free)
    assert np.allclose(e, [0.1, 0.05])


def test_identification_workload():
    w = W.cfg_sysid()
    assert w.n == 98_304 and tuple(w.res) == (64, 64, 64) and w.n_substeps == 1500
    a = np.asarray(w.traj.actions)
    assert a.shape == (150, 6)
    # insert by 0.05 m over the first half, then push by 0.05 m in x
    assert np.isclose(-a[:75, 1].sum(), 0.05) and np.isclose(a[75:, 0].sum(), 0.05)
    # the tip starts on the bed surface, a quarter along x
    assert np.isclose(w.traj.start_pose[1], w.x0[:, 1].max(), atol=w.dx)
    for k, (lo, hi) in enumerate(sysid.RANGES):
        assert lo <= (w.E, w.nu, w.rho, w.phi_deg)[k] <= hi
    # shorter rollouts keep the shovel speed
    s = W.cfg_sysid(n_substeps=300)
    b = np.asarray(s.traj.actions)
    assert np.isclose(-b[:15, 1].sum() / (15 * 10), -a[:75, 1].sum() / (75 * 10))


def test_identifiable_quantities():
    truth = np.array([1.2e5, 0.3, 1600.0, 32.0])
    # E and nu free: the bulk modulus K = E / (3 (1 - 2 nu)); candidates on
    # the curve of the true K have no error whatever E and nu are
    K = 1.2e5 / (3 * 0.4)
    nu = np.array([0.242, 0.3, 0.317])
    on_curve = np.stack([3 * K * (1 - 2 * nu), nu, np.full(3, 1600.0), np.full(3, 32.0)], axis=1)
    names, vals = sysid.identifiable(on_curve, (True, True, False, False))
    assert names == ["K"] and np.allclose(vals[:, 0], K)
    assert np.allclose(sysid._rel_error(on_curve, truth, np.array([True, True, False, False])), 0.0)
    # off the curve: the relative error of K
    off = np.array([[1.2e5 * 1.1, 0.3, 1600.0, 32.0]])
    assert np.allclose(sysid._rel_error(off, truth, np.array([True, True, False, True])), 0.1)
    # E and rho free: only E / rho; scaling both together is no error
    scaled = np.array([[2.4e5, 0.3, 3200.0, 32.0]])
    names, _ = sysid.identifiable(scaled, (True, False, True, False))
    assert names == ["E/rho"]
    assert np.allclose(sysid._rel_error(scaled, truth, np.array([True, False, True, False])), 0.0)
    # nu alone free, rho alone free, phi
    assert sysid.identifiable(truth[None, :], (False, True, False, True))[0] == ["nu", "phi"]
    assert sysid.identifiable(truth[None, :], (False, False, True, False))[0] == ["rho"]
