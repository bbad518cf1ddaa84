"""CUDA-graph replay of repeated identical forward/backward calls: the
replayed optimisation loop gives the results of eager launches, material
changes between replays take effect, and the graphs are actually used.
Float atomics make the order of the grid sums differ from run to run, so
two eager runs already differ in the last bits: a replay must stay within
that spread (checked against a second eager run)."""
import numpy as np
import pytest

from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    mpm.lib()


def _loop(ws, graphs, iters, K, nsub, materials=None):
    """An optimisation loop: reset the start state, record nsub substeps,
    MSE loss against a shifted copy of the start, backward."""
    opts = mpm.make_options(checkpoint_every=K, cuda_graphs=graphs)
    out = []
    theta = np.array([(w.E, w.nu, w.rho, w.phi_deg) for w in ws], np.float64)
    with mpm.simulation_from_workloads(ws, opts) as sim:
        sim.forward(5)
        x0 = sim.get_state()
        target = (x0["x"] + np.float32(0.002)).astype(np.float32)
        for it in range(iters):
            if materials is not None and it in materials:
                for i, m in enumerate(materials[it]):
                    sim.set_material(i, m)
                    theta[i] = m
            sim.set_substep(5)
            sim.set_state(x0["x"], x0["v"], x0["C"], x0["F"])
            sim.forward(nsub, record=True)
            L, g = sim.loss_mse(target)
            gm, gt = sim.backward(dL_dx=g)
            out.append((sim.get_state()["x"].copy(), np.asarray(L).copy(), np.asarray(gm).copy(),
                        sim.state_grad()["F"].copy(), theta.copy()))
        info = sim.info()
    return out, info


def _close(a, b, ref_a, ref_b):
    """Each of (x, L, dL/dmaterial, dL/dF) of run a within 10x the spread of
    two eager runs (ref_a, ref_b) of run b, plus a floor: absolute for the
    positions, relative per entry for the loss, relative to the largest
    entry for dL/dF. The material gradient is compared as the sensitivities
    theta_j dL/dtheta_j (E, nu, rho, phi in their units span many decades),
    with the gradient bar of the parity tests, 2e-2, relative to the
    instance's largest sensitivity: on small beds a small entry (dL/dphi
    when few particles yield) is a near-cancelling sum whose float-atomic
    summation order moves it by a few percent of its own value. A replay
    that ignored new parameters is caught by the material-change test."""
    theta = np.asarray(b[4], np.float64)
    floors = (("abs", 1e-6), ("each", 1e-7), ("sens", 2e-2), ("max", 1e-4))
    for u, v, ru, rv, (kind, fl) in zip(a, b, ref_a, ref_b, floors):
        u, v, ru, rv = (np.asarray(t, np.float64) for t in (u, v, ru, rv))
        if kind == "sens":
            u, v, ru, rv = (t * theta for t in (u, v, ru, rv))
            tol = 10 * np.abs(ru - rv) + fl * np.abs(v).max(axis=1, keepdims=True)
            assert np.all(np.abs(u - v) <= tol), (u, v, ru, rv)
            continue
        if kind == "each":
            tol = 10 * np.abs(ru - rv) + fl * np.abs(v)
            assert np.all(np.abs(u - v) <= tol), (u, v, ru, rv)
            continue
        scale = 1.0 if kind == "abs" else max(np.abs(v).max(), 1e-30)
        spread = np.abs(ru - rv).max()
        assert np.abs(u - v).max() <= 10 * spread + fl * scale, (np.abs(u - v).max(), spread, scale)


@pytest.mark.parametrize("K", [6, 20])   # recompute of earlier segments / one segment
def test_replayed_loop_matches_eager_bitwise(K):
    ws = [W.cfg_small()]
    nsub = 12
    eager, ie = _loop(ws, 0, 4, K, nsub)
    eager2, _ = _loop(ws, 0, 4, K, nsub)
    graph, ig = _loop(ws, 1, 4, K, nsub)
    assert ie["graph_launches"] == 0
    # per call kind: the first iteration runs eagerly (and allocates), a later
    # one is captured and launched as a graph, the rest are replays
    assert ig["graph_launches"] >= 2 * 2, ig
    assert ig["kernel_launches"] == ie["kernel_launches"]
    for a, a2, b in zip(eager, eager2, graph):
        _close(b, a, a2, a)


def test_material_change_between_replays():
    ws = [W.cfg_small()]
    mats = {2: [(2e5, 0.3, 1600.0, 33.0)]}
    eager, _ = _loop(ws, 0, 4, 20, 10, mats)
    eager2, _ = _loop(ws, 0, 4, 20, 10, mats)
    graph, ig = _loop(ws, 1, 4, 20, 10, mats)
    assert ig["graph_launches"] >= 4
    for a, a2, b in zip(eager, eager2, graph):
        _close(b, a, a2, a)
    # the change took effect in the replayed run: its dL/dE after the change
    # moved far beyond the run-to-run spread of the value before it
    gE1, gE1b = float(eager[1][2][0, 0]), float(eager2[1][2][0, 0])
    noise = max(abs(gE1 - gE1b), 1e-7 * abs(gE1))
    assert abs(float(graph[2][2][0, 0]) - gE1) > 10 * noise, (gE1, gE1b, float(graph[2][2][0, 0]))


def test_batched_uneven_replay():
    ws = W.batch_uneven(4, seed=3)
    eager, _ = _loop(ws, 0, 3, 8, 8)
    eager2, _ = _loop(ws, 0, 3, 8, 8)
    graph, ig = _loop(ws, 1, 3, 8, 8)
    assert ig["graph_launches"] >= 2
    for a, a2, b in zip(eager, eager2, graph):
        _close(b, a, a2, a)
