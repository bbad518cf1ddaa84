"""The oracle's threaded loops (OpenMP, used to time the CPU baseline on
all host cores) against its plain serial loops: the same arithmetic up to
the order of the sums, so positions and adjoints agree to FP64 summation-order
noise, and the per-node and per-particle steps without sums agree exactly."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import workloads as W

from _common import initial_state, oracle_params, oracle_poses


@pytest.fixture
def threads():
    yield
    oracle.set_threads(1)


def _run(w, nsub, n_threads, gx):
    oracle.set_threads(n_threads)
    p = oracle_params(w)
    x, v, C, F = initial_state(w.x0)
    poses = oracle_poses(w, nsub)
    st, s = oracle.rollout(p, x, v, C, F, poses)
    assert st == 0
    st, adj = oracle.rollout_adjoint(p, x, v, C, F, poses, gx=gx)
    assert st == 0
    return s, adj


@pytest.mark.parametrize("n_threads", [2, 5])
def test_threaded_oracle_equals_serial(threads, n_threads):
    w = W.cfg_small()
    gx = np.random.default_rng(3).normal(size=(w.n, 3)) / w.n
    # forward over 6 substeps: positions and state to summation-order noise
    s1, _ = _run(w, 6, 1, gx)
    sT, _ = _run(w, 6, n_threads, gx)
    assert oracle.get_threads() == n_threads
    for k in ("x", "v", "C", "F"):
        scale = max(np.abs(s1[k]).max(), 1e-300)
        assert np.abs(sT[k] - s1[k]).max() <= 1e-12 * scale, k
    # adjoint over 2 substeps. (Over longer rollouts from rest, particles
    # whose log-strain trace sits at 0 switch between the apex and elastic
    # cases of Eq. (7) on an ulp of difference in F, and the adjoint, which
    # is discontinuous there, then differs for them: that is the return
    # mapping's branch, not the threading.)
    _, a1 = _run(w, 2, 1, gx)
    _, aT = _run(w, 2, n_threads, gx)
    for k in ("x", "v", "C", "F"):
        scale = max(np.abs(a1[k]).max(), 1e-300)
        assert np.abs(aT[k] - a1[k]).max() <= 1e-13 * scale, k
    np.testing.assert_allclose(aT["material"], a1["material"], rtol=1e-9,
                               atol=1e-12 * np.abs(a1["material"]).max())
    np.testing.assert_allclose(aT["poses"], a1["poses"], rtol=1e-9, atol=1e-12 * np.abs(a1["poses"]).max())


def test_one_thread_is_the_serial_oracle(threads):
    # the serial loops are the pinned reference: setting one thread runs them
    oracle.set_threads(1)
    assert oracle.get_threads() == 1
    oracle.set_threads(0)
    assert oracle.get_threads() == 1
