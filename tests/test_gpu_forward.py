"""GPU forward parity: the CUDA substep (through the C ABI) against the FP64
oracle on the same seeded FP32 inputs.

Bars: positions within 1e-4 of the unit domain after 10 substeps; total
grid mass within 1e-6 relative. Velocity, C and F are checked too, against
tolerances derived from FP32 arithmetic (relative 1e-7 per operation; a few
hundred operations per value; contact decisions at nodes within rounding of
the box surface may flip, which moves the affected particles' velocity by
at most the shovel's relative speed times a B-spline weight)."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

from _common import initial_state, oracle_params, oracle_poses, oracle_rollout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    mpm.lib()


def _compare(g, ref, n_sub, label, x_bar=1e-4):
    ex = np.abs(g["x"] - ref["x"]).max()
    vmax = max(np.abs(ref["v"]).max(), 1e-6)
    ev = np.abs(g["v"] - ref["v"]).max() / vmax
    eF = np.abs(g["F"] - ref["F"]).max()
    cmax = max(np.abs(ref["C"]).max(), 1e-6)
    eC = np.abs(g["C"] - ref["C"]).max() / cmax
    print(f"{label}: substeps={n_sub} max|dx|={ex:.2e} max|dv|/vmax={ev:.2e} max|dF|={eF:.2e} max|dC|/Cmax={eC:.2e}")
    assert ex < x_bar, ex
    # 99.9% of particles far tighter than the bar
    assert np.quantile(np.abs(g["x"] - ref["x"]).max(1), 0.999) < 1e-5
    assert eF < 1e-3, eF
    return ex, ev, eF, eC


def test_small_bed_10_substeps():
    w = W.cfg_small()
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(10)
        g = sim.get_state()
        gm = sim.grid_mass()
    ref = oracle_rollout(w, 10)
    _compare(g, ref, 10, "bed8k")
    assert np.isclose(gm[0], w.n * w.rho * w.vol, rtol=1e-6)


def test_grid_mass_after_the_bed_leaves_its_blocks():
    """A uniform translation (v0 constant, C = 0, F = I, no gravity, no
    shovel) stays a translation under APIC; after 600 substeps the bed has
    moved 0.15 m in x (more than one 4-cell grid block), so blocks it occupied
    at the start are empty. The grid mass of the last substep is still
    sum_p rho V_p: nothing of the vacated blocks is counted."""
    w = W.cfg_small()
    v0 = np.array([2.5, 0.0, 1.5], np.float32)
    nsub = 600
    with mpm.simulation_from_workloads([w], shovel_on=0, gravity=(0.0, 0.0, 0.0)) as sim:
        sim.set_state(w.x0, np.tile(v0, (w.n, 1)))
        sim.forward(nsub)
        g = sim.get_state()
        gm = sim.grid_mass()
    moved = g["x"] - w.x0
    want = (v0.astype(np.float64) * w.dt * nsub)
    assert np.abs(moved - want).max() < 1e-4, np.abs(moved - want).max()
    assert want[0] > 4 * w.dx
    assert np.isclose(gm[0], w.n * w.rho * w.vol, rtol=1e-6), (gm[0], w.n * w.rho * w.vol)


def test_angular_momentum_conserved_on_the_gpu():
    """The APIC angular momentum (with its affine part, m_p eps : (C D)^T,
    D = dx^2/4 I) is constant over a rollout without gravity, walls or
    shovel, plastic flow included (the Kirchhoff stress is symmetric); on
    the GPU to FP32 rounding."""
    rng = np.random.default_rng(4)
    w = W.cfg_small()
    n = w.n
    x = (w.x0 + np.array([0.0, 0.2, 0.0], np.float32)).astype(np.float32)   # off the floor's wall zone
    ctr = x.mean(0)
    v = (np.cross(np.array([3.0, -5.0, 8.0]), x - ctr) + rng.normal(size=(n, 3)) * 0.05).astype(np.float32)
    C = (rng.normal(size=(n, 3, 3)) * 2.0).astype(np.float32)
    F = W.strained_F(rng, n, 0.05, (0.02, -0.08, 0.01)).astype(np.float32)

    def L(x, v, C):
        x, v, C = (np.asarray(a, np.float64) for a in (x, v, C))
        aff = np.stack([C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0], C[:, 1, 0] - C[:, 0, 1]], axis=1)
        return np.cross(x, v).sum(0) + 0.25 * w.dx ** 2 * aff.sum(0), \
            np.abs(np.cross(x, v)).sum() + 0.25 * w.dx ** 2 * np.abs(C).sum()

    with mpm.simulation_from_workloads([w], shovel_on=0, gravity=(0.0, 0.0, 0.0)) as sim:
        sim.set_state(x, v, C, F.reshape(n, 3, 3))
        s0 = sim.get_state()
        sim.forward(40)
        s1 = sim.get_state()
    L0, scale = L(s0["x"], s0["v"], s0["C"])
    L1, _ = L(s1["x"], s1["v"], s1["C"])
    print("angular momentum", L0, L1, "scale", scale)
    assert np.abs(L1 - L0).max() <= 1e-5 * scale, (L0, L1, scale)


def test_one_step_parity_along_200_substep_trajectory():
    """Every substep of the 200-substep rollout (insert, then push at 10 m/s)
    against the oracle run for one substep from the GPU's own state: the
    GPU substep equals the oracle's to FP32 rounding at every step
    (|dx| < 1e-6, |dv| < 1e-5 max(1, |v|max), |dF| < 1e-5), except for the
    rare particle whose contact decision (inside/outside the box, stick or
    slip) is taken within rounding of its threshold: at most 4 such particles
    per substep, each still within the 1e-4 position bar."""
    w = W.cfg_small()
    p = oracle_params(w)
    poses = oracle_poses(w, 200)
    n = w.n
    worst = [0.0, 0.0, 0.0]
    flips = 0
    with mpm.simulation_from_workloads([w]) as sim:
        g0 = sim.get_state()
        for s in range(200):
            sim.forward(1)
            g1 = sim.get_state()
            st, r = oracle.rollout(p, g0["x"].astype(np.float64), g0["v"].astype(np.float64),
                                   g0["C"].reshape(n, 9).astype(np.float64), g0["F"].reshape(n, 9).astype(np.float64),
                                   poses[s:s + 1])
            assert st == 0
            pex = np.abs(g1["x"] - r["x"]).max(1)
            pev = np.abs(g1["v"] - r["v"]).max(1) / max(1.0, np.abs(r["v"]).max())
            peF = np.abs(g1["F"] - r["F"]).reshape(n, -1).max(1)
            off = (pex >= 1e-6) | (pev >= 1e-5) | (peF >= 1e-5)
            flips += int(off.sum())
            assert off.sum() <= 4, (s, np.where(off)[0])
            assert pex.max() < 1e-4, (s, pex.max())
            ok = ~off
            worst = [max(worst[0], pex[ok].max()), max(worst[1], pev[ok].max()), max(worst[2], peF[ok].max())]
            g0 = g1
    print(f"one-step parity over 200 substeps: worst |dx| {worst[0]:.2e}, |dv|/max(1,|v|) {worst[1]:.2e}, "
          f"|dF| {worst[2]:.2e}; particle-substeps with a contact flip: {flips} of {200 * n}")
    assert flips <= 20


def test_long_rollout_drift_report():
    """Multi-step drift of the FP32 rollout from the FP64 one (parity is
    not pinned over long horizons: the impact of the shovel amplifies
    rounding differences; the one-step test above pins every substep).
    Bars: 10 substeps within 1e-4 (the parity bar), the whole rollout
    within 1e-2 for 99.9% of particles."""
    w = W.cfg_small()
    marks = [10, 25, 50, 100, 200]
    with mpm.simulation_from_workloads([w]) as sim:
        got, done = {}, 0
        for m in marks:
            sim.forward(m - done)
            done = m
            got[m] = sim.get_state()["x"]
    for m in marks:
        ref = oracle_rollout(w, m)
        ex = np.abs(got[m] - ref["x"]).max(1)
        print(f"bed8k drift after {m:3d} substeps: max {ex.max():.2e}  p99.9 {np.quantile(ex, 0.999):.2e}  "
              f"p99 {np.quantile(ex, 0.99):.2e}")
        if m == 10:
            assert ex.max() < 1e-4
        assert np.quantile(ex, 0.999) < 1e-2


def _mini_workloads():
    """Uneven instances: different grids (incl. sizes that are not a multiple
    of the 4^3 block), particle counts (1, ragged, 0), materials, contact."""
    out = []
    # 1: a single particle
    res, dx = 16, 1.0 / 16
    w = W.cfg_small()
    one = W.Workload("one", (res,) * 3, dx, 1e-4, 10, 1e5, 0.3, 1500.0, 30.0, dx ** 3 / 8,
                     np.array([[0.51, 0.4, 0.47]], np.float32),
                     W.Trajectory((0.8, 0.8, 0.8, 0.0), 5, actions=np.zeros((1, 6))))
    out.append(one)
    # 2: ragged count on a 20 x 18 x 22 grid, stiff material, shovel in contact
    res2, dx2 = (20, 18, 22), 1.0 / 20
    x2 = W.lattice_bed(11, (5, 4, 5), (6 * dx2, 3 * dx2, 7 * dx2), dx2)[:777]
    acts = np.zeros((3, 6)); acts[:, 1] = -0.003; acts[:, 3] = 0.02
    out.append(W.Workload("ragged", res2, dx2, 1e-4, 10, 3e5, 0.25, 1800.0, 35.0, dx2 ** 3 / 8, x2,
                          W.Trajectory((8.3 * dx2, 6.0 * dx2, 9.5 * dx2, 0.05), 4, actions=acts),
                          shovel_half=(0.02, 0.05, 0.08)))
    # 3: empty instance
    out.append(W.Workload("empty", (16, 16, 16), dx, 1e-4, 10, 1e5, 0.3, 1500.0, 30.0, dx ** 3 / 8,
                          np.zeros((0, 3), np.float32), W.Trajectory((0.5, 0.5, 0.5, 0.0), 5, actions=np.zeros((1, 6)))))
    # 4: soft soil sliding down with friction angle 20
    res4, dx4 = (24, 24, 24), 1.0 / 24
    x4 = W.lattice_bed(13, (6, 6, 3), (5 * dx4, 3 * dx4, 9 * dx4), dx4)
    out.append(W.Workload("soil", res4, dx4, 2e-4, 10, 5e4, 0.35, 1300.0, 20.0, dx4 ** 3 / 8, x4,
                          W.Trajectory((0.7, 0.7, 0.7, 0.0), 5, actions=np.zeros((1, 6)))))
    return out


def test_batched_uneven_instances_match_oracle_each():
    ws = _mini_workloads()
    nsub = 10
    with mpm.simulation_from_workloads(ws) as sim:
        sim.forward(nsub)
        g = sim.get_state()
        gm = sim.grid_mass()
    off = 0
    for i, w in enumerate(ws):
        n = w.n
        sl = slice(off, off + n)
        off += n
        if n == 0:
            assert gm[i] == 0.0
            continue
        ref = oracle_rollout(w, nsub)
        _compare({k: v[sl] for k, v in g.items()}, ref, nsub, w.name)
        assert np.isclose(gm[i], n * w.rho * w.vol, rtol=1e-6)


def test_batched_equals_serial():
    """Each instance of a batch gives the same result as the instance alone
    (float atomics make the order of grid sums differ: tolerance 1e-6)."""
    ws = _mini_workloads()
    nsub = 6
    with mpm.simulation_from_workloads(ws) as sim:
        sim.forward(nsub)
        gb = sim.get_state()
    off = 0
    for w in ws:
        if w.n == 0:
            continue
        with mpm.simulation_from_workloads([w]) as s1:
            s1.forward(nsub)
            g1 = s1.get_state()
        assert np.abs(gb["x"][off:off + w.n] - g1["x"]).max() < 1e-6
        off += w.n


def test_particle_collision_flag_off():
    ws = _mini_workloads()[1:2]
    with mpm.simulation_from_workloads(ws, particle_collision=0) as sim:
        sim.forward(8)
        g = sim.get_state()
    ref = oracle_rollout(ws[0], 8, particle_collision=0)
    _compare(g, ref, 8, "ragged-no-particle-contact")


def test_state_roundtrip_and_reset():
    w = W.cfg_small()
    rng = np.random.default_rng(0)
    with mpm.simulation_from_workloads([w]) as sim:
        s0 = sim.get_state()
        assert np.array_equal(s0["x"], w.x0) and (s0["v"] == 0).all() and (s0["F"] == np.eye(3, dtype=np.float32)).all()
        v = rng.normal(size=(w.n, 3)).astype(np.float32)
        C = rng.normal(size=(w.n, 3, 3)).astype(np.float32)
        F = (np.eye(3) + 0.01 * rng.normal(size=(w.n, 3, 3))).astype(np.float32)
        sim.set_state(w.x0, v, C, F)
        s1 = sim.get_state()
        for k, a in (("v", v), ("C", C), ("F", F)):
            assert np.array_equal(s1[k], a)
        sim.forward(3)
        sim.reset()
        s2 = sim.get_state()
        assert np.array_equal(s2["x"], w.x0) and (s2["v"] == 0).all()


def test_out_of_domain_is_reported():
    """A particle driven out of [dx, (res-2) dx) makes the call return
    MPM_ERR_OUT_OF_DOMAIN (kernels clamp their indices, nothing faults)."""
    res, dx = 16, 1.0 / 16
    cfg = mpm.make_config((res,) * 3, dx, 1e-3, dx ** 3 / 8, gravity=(0, 0, 0), shovel_on=0)
    x = np.array([[0.5, 0.5, 13.9 * dx]], np.float32)
    with mpm.Simulation([cfg], [(1e5, 0.3, 1500.0, 30.0)], [x]) as sim:
        sim.set_state(x, np.array([[0.0, 0.0, 50.0]], np.float32))
        with pytest.raises(mpm.MpmError) as e:
            sim.forward(2)
        assert e.value.code == -4


def test_non_finite_is_reported():
    res, dx = 16, 1.0 / 16
    cfg = mpm.make_config((res,) * 3, dx, 1e-4, dx ** 3 / 8, shovel_on=0)
    x = np.array([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5]], np.float32)
    with mpm.Simulation([cfg], [(1e5, 0.3, 1500.0, 30.0)], [x]) as sim:
        v = np.array([[0.0, 0.0, 0.0], [np.inf, 0.0, 0.0]], np.float32)
        sim.set_state(x, v)
        with pytest.raises(mpm.MpmError) as e:
            sim.forward(1)
        assert e.value.code in (-5, -4)


def test_full_size_sampled_substep():
    """1,048,576 particles on the 128^3 grid, in the bench's launch
    configuration: after 30 GPU substeps (shovel approaching, bed settling
    under gravity), one more GPU substep is compared, for 48 sampled
    particles, with the oracle run on each sample's neighbourhood (all
    particles within two cells, which is every particle that writes to a
    node the sample reads)."""
    w = W.cfg_1m()
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(30)
        s0 = sim.get_state()
        sim.forward(1)
        s1 = sim.get_state()
        gm = sim.grid_mass()
    assert np.isclose(gm[0], w.n * w.rho * w.vol, rtol=1e-6)
    assert all(np.isfinite(s1[k]).all() for k in s1)
    p = oracle_params(w)
    poses = oracle_poses(w, 31)[30:31]
    rng = np.random.default_rng(5)
    base = np.floor(s0["x"].astype(np.float64) / w.dx - 0.5).astype(np.int64)
    samples = rng.choice(w.n, 48, replace=False)
    worst = 0.0
    for q in samples:
        nb = np.where(np.abs(base - base[q]).max(1) <= 2)[0]
        j = int(np.where(nb == q)[0][0])
        xs = s0["x"][nb].astype(np.float64)
        st, r = oracle.rollout(p, xs, s0["v"][nb], s0["C"][nb].reshape(-1, 9), s0["F"][nb].reshape(-1, 9), poses)
        assert st == 0
        dx_ = np.abs(s1["x"][q] - r["x"][j]).max()
        dv_ = np.abs(s1["v"][q] - r["v"][j]).max()
        dF_ = np.abs(s1["F"][q] - r["F"][j]).max()
        worst = max(worst, dx_)
        assert dx_ < 1e-6, (q, dx_)
        assert dv_ < 1e-3 * max(1.0, np.abs(r["v"][j]).max()), (q, dv_)
        assert dF_ < 1e-5, (q, dF_)
    print(f"full-size sampled substep: worst |dx| {worst:.2e}")


def test_full_size_batch_sampled_substep():
    """The 64 uneven instances (20k-192k particles, 64^3-96^3 grids, each with
    its own material and shovel) in one handle, as the bench's batched leg
    runs them: after 20 GPU substeps, one more GPU substep is compared, for
    sampled particles of the smallest, the largest and two other instances,
    with the oracle run on each sample's neighbourhood in its own instance;
    every instance keeps its mass."""
    ws = W.batch_uneven(64)
    counts = [w.n for w in ws]
    offs = np.concatenate([[0], np.cumsum(counts)])
    with mpm.simulation_from_workloads(ws) as sim:
        sim.forward(20)
        s0 = sim.get_state()
        sim.forward(1)
        s1 = sim.get_state()
        gm = sim.grid_mass()
    for i, w in enumerate(ws):
        assert np.isclose(gm[i], w.n * w.rho * w.vol, rtol=1e-6), i
    rng = np.random.default_rng(9)
    picks = {int(np.argmin(counts)), int(np.argmax(counts))}
    picks |= set(int(i) for i in rng.choice(len(ws), 2, replace=False))
    worst = 0.0
    for i in sorted(picks):
        w = ws[i]
        sl = slice(offs[i], offs[i + 1])
        x0 = s0["x"][sl]
        p = oracle_params(w)
        poses = oracle_poses(w, 21)[20:21]
        base = np.floor(x0.astype(np.float64) / w.dx - 0.5).astype(np.int64)
        for q in rng.choice(w.n, 6, replace=False):
            nb = np.where(np.abs(base - base[q]).max(1) <= 2)[0]
            j = int(np.where(nb == q)[0][0])
            st, r = oracle.rollout(p, x0[nb].astype(np.float64), s0["v"][sl][nb], s0["C"][sl][nb].reshape(-1, 9),
                                   s0["F"][sl][nb].reshape(-1, 9), poses)
            assert st == 0
            dx_ = np.abs(s1["x"][sl][q] - r["x"][j]).max()
            dF_ = np.abs(s1["F"][sl][q] - r["F"][j]).max()
            worst = max(worst, dx_)
            assert dx_ < 1e-6, (i, q, dx_)
            assert dF_ < 1e-5, (i, q, dF_)
    print(f"full-size batch sampled substep: instances {sorted(picks)}, worst |dx| {worst:.2e}")


def test_sorted_scrambled_order_matches_oracle():
    """Particles given in a random order and re-sorted by grid block every 3
    substeps: the state (read back in the caller's order) still matches the
    oracle run on the same order."""
    w = W.cfg_small()
    rng = np.random.default_rng(21)
    w.x0 = w.x0[rng.permutation(w.n)]
    for sort_every in (3, 0):
        with mpm.simulation_from_workloads([w], mpm.make_options(sort_every=sort_every)) as sim:
            sim.forward(10)
            g = sim.get_state()
        ref = oracle_rollout(w, 10)
        _compare(g, ref, 10, f"bed8k scrambled, sort_every={sort_every}")


def test_autotune_restores_state_and_keeps_parity():
    """mpm_autotune times its candidates from the current state and restores
    it; the tuned handle still matches the oracle."""
    w = W.cfg_small()
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(3)
        before = sim.get_state()
        choice = sim.autotune(6)
        after = sim.get_state()
        for k in before:
            assert np.array_equal(before[k], after[k]), k
        assert choice["tile_scatter"] in (0, 1) and choice["sort_every"] >= 0
        sh = choice["launch_shape"]
        assert sh["p2g"] in (3, 4) and sh["g2p"] in (3, 4) and sh["fused"] in (2, 3, 4)
        # the choice is cached for the workload: a second call gives it again
        assert sim.autotune(6) == choice
        sim.forward(7)
        g = sim.get_state()
    ref = oracle_rollout(w, 10)
    _compare(g, ref, 10, f"bed8k after autotune {choice}")


def test_autotune_failure_leaves_the_handle_as_it_was():
    """A trial that fails (a particle leaves the domain within the trial
    substeps) makes mpm_autotune return the error and restore the state, its
    particle order, the substep counter, the options and the launch shape;
    the handle then runs as before."""
    res, dx = 16, 1.0 / 16
    cfg = mpm.make_config((res,) * 3, dx, 1e-3, dx ** 3 / 8, gravity=(0, 0, 0), shovel_on=0)
    x = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 13.0 * dx]], np.float32)
    v = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 30.0]], np.float32)
    with mpm.Simulation([cfg], [(1e5, 0.3, 1500.0, 30.0)], [x], mpm.make_options(sort_every=0)) as sim:
        sim.set_state(x, v)
        sim.set_launch_shape(3, 4, 2)
        before = sim.get_state()
        info0 = sim.info()
        with pytest.raises(mpm.MpmError) as e:
            sim.autotune(8)
        assert e.value.code == -4
        after = sim.get_state()
        for k in before:
            assert np.array_equal(before[k], after[k]), k
        assert sim.launch_shape() == {"p2g": 3, "g2p": 4, "fused": 2}
        info1 = sim.info()
        assert info1["substep"] == info0["substep"] and info1["recorded"] == 0
        # device memory held is what it was (the tuner's copies are released)
        assert info1["device_bytes"] >= info0["device_bytes"]
        sim.forward(1)   # one substep still runs (the particle is 3 cells from the wall)


@pytest.mark.parametrize("shape", [(3, 3, 2), (4, 4, 3), (3, 4, 4)])
def test_every_launch_shape_matches_the_oracle(shape):
    """Each register-cap instantiation of the particle kernels gives the
    oracle's positions after 10 substeps, and the same gradient (the fused
    adjoint included) as the default shape."""
    w = W.cfg_small()
    opts = mpm.make_options(checkpoint_every=16)

    def grad(sim):
        sim.reset()
        sim.forward(40, record=True)
        L, gx = sim.loss_mse(w.x0 + np.float32(0.002))
        return sim.backward(dL_dx=gx)[0]

    with mpm.simulation_from_workloads([w], opts) as sim:
        sim.set_launch_shape(*shape)
        assert tuple(sim.launch_shape().values()) == shape
        sim.forward(10)
        g = sim.get_state()
        gm = grad(sim)
        with pytest.raises(mpm.MpmError):
            sim.set_launch_shape(5, 4, 3)
    _compare(g, oracle_rollout(w, 10), 10, f"bed8k launch shape {shape}")
    with mpm.simulation_from_workloads([w], opts) as ref:
        gm0 = grad(ref)
    print("gradient", gm[0], "default shape", gm0[0])
    np.testing.assert_allclose(gm, gm0, rtol=2e-2, atol=1e-3 * np.abs(gm0).max())
