"""GPU parity of the surface observation, the height map and the height-map
distance (Sec. III-A, Eq. (2)) and of the batched line search (Sec. III-F)
against the oracle. The observation and the map are selections: index for
index on the GPU's own FP32 state; the distance within FP64 summation order;
the gradient (integer valued) exactly."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

from _common import oracle_params, oracle_poses

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    mpm.lib()


def _bed_centre(w):
    return float(np.mean(w.x0[:, 0])), float(np.mean(w.x0[:, 2]))


def _check_instance(x, g_o, pts, cnt, hmap):
    n_o, idx = oracle.surface_observation(g_o, x)
    assert cnt == n_o
    full = idx >= 0
    assert np.array_equal(pts[full], x[idx[full]])
    assert np.isnan(pts[~full]).all()
    I, w = oracle.height_map(g_o, x)
    assert np.array_equal(hmap.reshape(-1), I.reshape(-1).astype(np.float32))


@pytest.mark.parametrize("res,size,tap", [(40, 0.24, 0.003), (17, 0.2, 0.0), (64, 0.3, 0.01)])
def test_observation_and_height_map_match_oracle(res, size, tap):
    w = W.cfg_small()
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(150)                      # the shovel has dug in
        x = sim.get_state()["x"]
        c = _bed_centre(w)
        g = mpm.make_obs_grid(c, size, res, tap)
        pts, cnt = sim.surface_observation(g)
        hm = sim.height_map(g)
    _check_instance(x, oracle.ObsGrid(c[0], c[1], size, res, tap), pts[0], cnt[0], hm[0])


def test_hmd_loss_and_gradient_match_oracle():
    w = W.cfg_small()
    c = _bed_centre(w)
    g = mpm.make_obs_grid(c, 0.24, 40, 0.003)
    g_o = oracle.ObsGrid(c[0], c[1], 0.24, 40, 0.003)
    with mpm.simulation_from_workloads([w]) as sim:
        target = sim.height_map(g)            # the flat bed
        sim.forward(150)
        x = sim.get_state()["x"]
        L, grad = sim.loss_hmd(g, target)
    Lo, go = oracle.hmd(g_o, x, target[0].astype(np.float64))
    assert Lo > 0
    assert abs(L[0] - Lo) <= 1e-12 * Lo
    assert np.array_equal(grad, go.astype(np.float32))
    assert np.abs(grad[:, 1]).sum() > 0 and not grad[:, 0].any() and not grad[:, 2].any()


def test_batched_instances_each_match_oracle():
    ws = W.batch_uneven(5, seed=11)
    grids, grids_o = [], []
    for k, w in enumerate(ws):
        c = _bed_centre(w) if w.n else (0.5, 0.5)
        size = 0.1 + 0.05 * k
        grids.append(mpm.make_obs_grid(c, size, 24, 0.002 * k))
        grids_o.append(oracle.ObsGrid(c[0], c[1], size, 24, 0.002 * k))
    with mpm.simulation_from_workloads(ws) as sim:
        sim.forward(20)
        x = sim.get_state()["x"]
        pts, cnt = sim.surface_observation(grids)
        hm = sim.height_map(grids)
        tgt = np.stack([np.full((24, 24), 0.1 + 0.01 * k, np.float32) for k in range(len(ws))])
        L, grad = sim.loss_hmd(grids, tgt)
    off = 0
    for k, w in enumerate(ws):
        xs = x[off:off + w.n]
        _check_instance(xs, grids_o[k], pts[k], cnt[k], hm[k])
        Lo, go = oracle.hmd(grids_o[k], xs, tgt[k].astype(np.float64))
        assert abs(L[k] - Lo) <= 1e-12 * max(Lo, 1e-30)
        assert np.array_equal(grad[off:off + w.n], go.astype(np.float32))
        off += w.n


def test_full_size_observation_matches_oracle():
    w = W.cfg_1m()
    c = _bed_centre(w)
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(40)
        x = sim.get_state()["x"]
        g = mpm.make_obs_grid(c, 0.24, 40, 0.0015)
        pts, cnt = sim.surface_observation(g)
        hm = sim.height_map(g)
    assert cnt[0] == 1600
    _check_instance(x, oracle.ObsGrid(c[0], c[1], 0.24, 40, 0.0015), pts[0], cnt[0], hm[0])


def test_batched_line_search_matches_oracle():
    """Five material candidates along a step direction (alpha in {0.1, 0.5,
    1, 1.5, 2}) advance together; the least height-map distance wins, as it
    does for the oracle's own forwards of the five candidates."""
    base = W.cfg_small()
    alphas = [0.1, 0.5, 1.0, 1.5, 2.0]
    step = np.array([4e4, 0.0, -300.0, -8.0])   # E, nu, rho, phi
    mats = [tuple(np.array([base.E, base.nu, base.rho, base.phi_deg]) - a * step) for a in alphas]
    nsub = 40
    # the target: the height map the ground-truth material (alpha = 1) gives
    c = _bed_centre(base)
    g = mpm.make_obs_grid(c, 0.24, 40, 0.003)
    g_o = oracle.ObsGrid(c[0], c[1], 0.24, 40, 0.003)
    ws = [base] * len(alphas)
    with mpm.simulation_from_workloads(ws) as sim:
        sim.forward(60)
        st = sim.get_state()
    n = base.n
    # target: the oracle forward of the alpha = 1 material from that state
    import dataclasses
    p_gt = oracle_params(dataclasses.replace(base, E=mats[2][0], nu=mats[2][1], rho=mats[2][2], phi_deg=mats[2][3]))
    poses = oracle_poses(base, 60 + nsub)[60:]
    sv = [np.asarray(st[k][:n], np.float64) for k in ("x", "v", "C", "F")]
    s_, ref = oracle.rollout(p_gt, sv[0], sv[1], sv[2].reshape(n, 9), sv[3].reshape(n, 9), poses)
    assert s_ == 0
    tgt, _ = oracle.height_map(g_o, ref["x"].astype(np.float32))
    tgt = tgt.astype(np.float32)
    # oracle losses of the five candidates
    Lo = []
    for m in mats:
        p = oracle_params(dataclasses.replace(base, E=m[0], nu=m[1], rho=m[2], phi_deg=m[3]))
        s_, r = oracle.rollout(p, sv[0], sv[1], sv[2].reshape(n, 9), sv[3].reshape(n, 9), poses)
        assert s_ == 0
        Lo.append(oracle.hmd(g_o, r["x"].astype(np.float32), tgt)[0])
    # the GPU: one batched handle, the five candidates from the same state
    with mpm.simulation_from_workloads(ws) as sim:
        sim.set_state(*[np.concatenate([st[k][:n]] * len(alphas)) for k in ("x", "v", "C", "F")])
        sim.set_substep(60)
        best, L = sim.line_search(nsub, g, np.stack([tgt] * len(alphas)), materials=mats)
    print("oracle", Lo, "gpu", list(L), "best", best)
    assert best == int(np.argmin(Lo)) == 2
    # FP32 and FP64 trajectories give heights a few 1e-7 apart per pixel
    assert np.allclose(L, Lo, rtol=0.02, atol=1e-3)


@pytest.mark.parametrize("n_extra", [0, 37])
def test_emd_matches_oracle(n_extra):
    """Earth Mover's distance of Eq. (1) between the observation and a target
    cloud: the GPU auction's distance lies between the optimum (oracle, by
    linear assignment on the same FP32 points) and the optimum plus
    n * eps_final; its gradient is a unit vector on every observed particle
    and zero elsewhere, and equals the oracle's where the maps agree."""
    w = W.cfg_small()
    c = _bed_centre(w)
    size = 0.24
    g = mpm.make_obs_grid(c, size, 40, 0.0)
    g_o = oracle.ObsGrid(c[0], c[1], size, 40, 0.0)
    rng = np.random.default_rng(40 + n_extra)
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(150)
        x = sim.get_state()["x"]
        pts, cnt = sim.surface_observation(g)
        X = pts[0][~np.isnan(pts[0][:, 0])]
        tgt = (X + np.array([0.004, -0.006, 0.002], np.float32)
               + 0.003 * rng.normal(size=X.shape).astype(np.float32)).astype(np.float32)
        if n_extra:
            tgt = np.concatenate([tgt, (X[:n_extra] + 0.02).astype(np.float32)])
        tgt = tgt[rng.permutation(tgt.shape[0])]
        L, grad = sim.loss_emd(g, [tgt])
    n_obs, idx = oracle.surface_observation(g_o, x)
    assert n_obs == X.shape[0] == cnt[0]
    Lo, phi, go = oracle.emd(X, tgt)
    eps_final = 1e-6 * size
    print("EMD gpu", L[0], "oracle", Lo, "n eps", n_obs * eps_final)
    assert Lo * (1 - 1e-6) <= L[0] <= Lo + n_obs * eps_final + 1e-6 * Lo
    owners = idx[idx >= 0]                       # particle of each observed pixel, pixel order
    norms = np.linalg.norm(grad[owners], axis=1)
    assert np.allclose(norms, 1.0, atol=1e-5)
    others = np.setdiff1d(np.arange(x.shape[0]), owners)
    assert not grad[others].any()
    same = np.all(np.abs(grad[owners] - go.astype(np.float32)) < 1e-4, axis=1)
    print("gradient rows equal to the oracle's:", same.mean())
    assert same.mean() > 0.9
    # the GPU's map is one-to-one: each observed point's gradient row is the
    # unit vector from its assigned target, which identifies that target
    # (the targets are in general position); no target is used twice, and
    # the assigned distances add up to the reported distance
    Xd, Td = X.astype(np.float64), tgt.astype(np.float64)
    rows = grad[owners].astype(np.float64)
    diff = Xd[:, None, :] - Td[None, :, :]
    dist = np.linalg.norm(diff, axis=2)
    unit = diff / np.maximum(dist, 1e-30)[:, :, None]
    err = np.linalg.norm(unit - rows[:, None, :], axis=2)
    assigned = err.argmin(axis=1)
    assert err[np.arange(len(assigned)), assigned].max() < 1e-3
    assert np.unique(assigned).size == assigned.size, "a target is assigned twice"
    assert abs(dist[np.arange(len(assigned)), assigned].sum() - L[0]) <= 1e-5 * L[0]
