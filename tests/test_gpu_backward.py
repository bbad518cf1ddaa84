"""GPU adjoint parity: gradients from the CUDA backward (through the C ABI)
against the FP64 oracle's own adjoint and against central finite
differences of the oracle forward. Bar: 2e-2 relative per component
(relative to max(|g_ref|, 1e-3 * max|g_ref|))."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

from _common import initial_state, oracle_actions, oracle_params, oracle_poses, rel_err

pytestmark = pytest.mark.gpu
BAR = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    mpm.lib()


def _contact_workload():
    """A small bed with a tilted shovel pushing into it (grid and particle
    contact, plastic flow, walls)."""
    res, dx = 20, 1.0 / 20
    x0 = W.lattice_bed(21, (6, 4, 5), (6 * dx, 3 * dx, 7 * dx), dx)
    acts = np.zeros((4, 6))
    acts[:, 0] = 0.004
    acts[:, 1] = -0.002
    acts[:, 3] = 0.01
    return W.Workload("contact", (res,) * 3, dx, 1e-4, 12, 1e5, 0.3, 1500.0, 30.0, dx ** 3 / 8, x0,
                      W.Trajectory((7.1 * dx, 5.2 * dx, 9.3 * dx, 0.1), 3, actions=acts),
                      shovel_half=(0.025, 0.06, 0.08))


def _strained_state(w, seed):
    rng = np.random.default_rng(seed)
    n = w.n
    F = W.strained_F(rng, n, 0.01, (0.01, -0.03, 0.0)).astype(np.float32)
    v = (rng.normal(size=(n, 3)) * 0.05).astype(np.float32)
    C = (rng.normal(size=(n, 3, 3)) * 0.3).astype(np.float32)
    return w.x0, v, C, F


def _gpu_grad(ws, states, nsub, seeds, K=50, clip=0, grad_scale=0, fuse=1, tile=0):
    opts = mpm.make_options(checkpoint_every=K, clip_grads=clip, grad_scale=grad_scale, fuse_adjoint=fuse,
                            tile_scatter=tile)
    with mpm.simulation_from_workloads(ws, opts) as sim:
        if states is not None:
            sim.set_state(*[np.concatenate([s[k] for s in states]) for k in range(4)])
        sim.forward(nsub, record=True)
        out = sim.get_state()
        gx = np.concatenate([s[0] for s in seeds]).astype(np.float32)
        gv = np.concatenate([s[1] for s in seeds]).astype(np.float32)
        gm, gt = sim.backward(dL_dx=gx, dL_dv=gv)
        gs = sim.state_grad()
        ga = [sim.action_grad(i) for i in range(len(ws))]
    return out, gm, gt, gs, ga


def _oracle_grad(w, state, nsub, seed, clip=0, grad_scale=0):
    p = oracle_params(w, clip=clip, grad_scale=grad_scale)
    poses = oracle_poses(w, nsub)
    x, v, C, F = [np.asarray(a, np.float64) for a in state]
    n = w.n
    st, g = oracle.rollout_adjoint(p, x.reshape(n, 3), v.reshape(n, 3), C.reshape(n, 9), F.reshape(n, 9), poses,
                                   gx=seed[0], gv=seed[1])
    assert st == 0
    acts, jac = oracle_actions(w)
    ga = oracle.pose_table_adjoint(acts.shape[0], w.traj.substeps_per_action, w.dt, g["poses"])
    gt = None if jac is None else np.einsum("tk,tkj->j", ga, jac)
    return g, ga, gt


def _seed(w, seed):
    """Coherent loss seeds, like the MSE gradient 2 (x - xhat) / N of a target
    shifted from the final state: a common direction plus 10% noise. (Pure
    noise seeds make the parameter gradients sums that cancel ~100x, whose
    value then hinges on the few particles that sit exactly on the yield
    surface, where the FP32 and FP64 trajectories may take different
    branches.)"""
    rng = np.random.default_rng(seed)
    d = np.array([1.0, -0.5, 0.3])
    return ((d + 0.1 * rng.normal(size=(w.n, 3))) / w.n,
            (1e-3 * d + 1e-4 * rng.normal(size=(w.n, 3))) / w.n)


def test_adjoint_matches_oracle_contact_scenario():
    w = _contact_workload()
    state = _strained_state(w, 1)
    seed = _seed(w, 2)
    nsub = 12
    _, gm, gt, gs, ga = _gpu_grad([w], [state], nsub, [seed], K=5)
    g, ga_ref, _ = _oracle_grad(w, state, nsub, seed)
    print("material gpu", gm[0], "oracle", g["material"])
    assert rel_err(gm[0], g["material"]).max() < BAR
    for k in ("x", "v", "C", "F"):
        e = rel_err(gs[k].reshape(w.n, -1), g[k].reshape(w.n, -1))
        print(k, "state-grad max rel err", e.max(), "p99", np.quantile(e, 0.99))
        assert np.quantile(e, 0.99) < BAR
        assert e.max() < 10 * BAR
    assert np.abs(ga_ref).max() > 0
    e = rel_err(ga[0][0][:, :4], ga_ref[:, :4])
    print("action grad max rel err", e.max())
    assert e.max() < BAR


def test_tile_scatter_matches_oracle():
    """Option tile_scatter (the 27-node scatters of the forward P2G and of the
    G2P adjoint summed per CTA in shared memory, then flushed) against the
    oracle's forward and adjoint, in the contact scenario."""
    w = _contact_workload()
    state = _strained_state(w, 1)
    seed = _seed(w, 2)
    nsub = 12
    out, gm, _, gs, ga = _gpu_grad([w], [state], nsub, [seed], K=5, tile=1)
    p = oracle_params(w)
    x, v, C, F = [np.asarray(a, np.float64) for a in state]
    n = w.n
    st, ref = oracle.rollout(p, x.reshape(n, 3), v.reshape(n, 3), C.reshape(n, 9), F.reshape(n, 9),
                             oracle_poses(w, nsub))
    assert st == 0
    assert np.abs(out["x"] - ref["x"]).max() < 1e-4
    g, ga_ref, _ = _oracle_grad(w, state, nsub, seed)
    print("material gpu (tiled)", gm[0], "oracle", g["material"])
    assert rel_err(gm[0], g["material"]).max() < BAR
    for k in ("x", "v", "C", "F"):
        e = rel_err(gs[k].reshape(w.n, -1), g[k].reshape(w.n, -1))
        print(k, "state-grad max rel err", e.max(), "p99", np.quantile(e, 0.99))
        assert np.quantile(e, 0.99) < BAR
    e = rel_err(ga[0][0][:, :4], ga_ref[:, :4])
    assert e.max() < BAR


@pytest.mark.parametrize("unrounded", [False, True])
def test_adjoint_skill_theta_gradient(unrounded):
    """dL/dtheta through Algorithm 2's Jacobian (frozen T; rounded or, for
    the alternative mapping of Sec. III-B, real-valued phase-1/4 step
    counts): the library's chain against the oracle's (pose-table adjoint,
    then the Jacobian), on a bed dug by the skill."""
    res, dx = 32, 1.0 / 32
    x0 = W.lattice_bed(31, (10, 5, 8), (11 * dx, 3 * dx, 12 * dx), dx)
    top = 8 * dx
    traj = W.Trajectory((13.5 * dx, top - 0.005, 16 * dx, 0.0), 4, theta=(0.4, 0.3, 0.55, 0.2, -0.2, 0.5),
                        v_lin=25.0, v_ang=250.0, unrounded=unrounded)
    w = W.Workload("skill", (res,) * 3, dx, 1e-4, 40, 1e5, 0.3, 1500.0, 30.0, dx ** 3 / 8, x0, traj,
                   shovel_half=(0.02, 0.06, 0.1))
    seed = _seed(w, 3)
    state = (w.x0, np.zeros((w.n, 3), np.float32), np.zeros((w.n, 3, 3), np.float32),
             np.tile(np.eye(3, dtype=np.float32), (w.n, 1, 1)))
    nsub = 40
    _, gm, gt, gs, ga = _gpu_grad([w], None, nsub, [seed], K=10)
    g, ga_ref, gt_ref = _oracle_grad(w, state, nsub, seed)
    print("theta gpu", gt[0], "oracle", gt_ref)
    assert np.abs(gt_ref).max() > 0
    assert rel_err(gt[0], gt_ref).max() < BAR
    assert rel_err(gm[0], g["material"]).max() < BAR


def test_checkpoint_interval_does_not_change_gradients():
    w = _contact_workload()
    state = _strained_state(w, 4)
    seed = _seed(w, 5)
    a = _gpu_grad([w], [state], 12, [seed], K=3)
    b = _gpu_grad([w], [state], 12, [seed], K=50)
    assert rel_err(a[1][0], b[1][0]).max() < 1e-4
    assert np.abs(a[3]["x"] - b[3]["x"]).max() <= 1e-4 * np.abs(b[3]["x"]).max()


def test_batched_adjoint_equals_each_instance():
    w1 = _contact_workload()
    res, dx = 16, 1.0 / 16
    x2 = W.lattice_bed(41, (4, 3, 4), (6 * dx, 3 * dx, 6 * dx), dx)
    w2 = W.Workload("b2", (res,) * 3, dx, 1e-4, 8, 2e5, 0.25, 1700.0, 35.0, dx ** 3 / 8, x2,
                    W.Trajectory((0.9, 0.9, 0.9, 0.0), 2, actions=np.zeros((1, 6))))
    s1, s2 = _strained_state(w1, 6), _strained_state(w2, 7)
    e1, e2 = _seed(w1, 8), _seed(w2, 9)
    _, gm, _, _, _ = _gpu_grad([w1, w2], [s1, s2], 8, [e1, e2], K=4)
    for i, (w, s, e) in enumerate([(w1, s1, e1), (w2, s2, e2)]):
        g, _, _ = _oracle_grad(w, s, 8, e)
        assert rel_err(gm[i], g["material"]).max() < BAR, (i, gm[i], g["material"])


def test_gpu_gradient_against_central_fd():
    """The GPU material gradient against central differences of the FP64
    oracle forward. The model is piecewise smooth: most particles of this
    scenario sit on the Drucker-Prager cone, and a relative step of 1e-4 in
    phi moves the cone across some of them (the FD then averages two
    branches). The step is 1e-6 relative, where the differences have
    converged (a 1e-5 and a 1e-6 step must agree to 2e-2 before the GPU is
    compared)."""
    w = _contact_workload()
    state = _strained_state(w, 10)
    seed = _seed(w, 11)
    nsub = 8
    _, gm, _, _, _ = _gpu_grad([w], [state], nsub, [seed], K=4)
    p = oracle_params(w)
    poses = oracle_poses(w, nsub)
    x, v, C, F = [np.asarray(a, np.float64).reshape(w.n, -1) for a in state]

    def loss(pp):
        st, s = oracle.rollout(pp, x, v, C, F, poses)
        assert st == 0
        return (seed[0] * s["x"]).sum() + (seed[1] * s["v"]).sum()

    def fd_at(rel):
        out = []
        for key in ("E", "nu", "rho", "phi_deg"):
            base = getattr(p, key)
            h = rel * base
            setattr(p, key, base + h); lp = loss(p)
            setattr(p, key, base - h); lm = loss(p)
            setattr(p, key, base)
            out.append((lp - lm) / (2 * h))
        return np.array(out)

    fd, fd5 = fd_at(1e-6), fd_at(1e-5)
    print("gpu", gm[0], "fd(1e-6)", fd, "fd(1e-5)", fd5)
    assert rel_err(fd5, fd).max() < BAR
    assert rel_err(gm[0], fd).max() < BAR


def test_clipped_adjoint_matches_oracle():
    w = _contact_workload()
    state = _strained_state(w, 12)
    rng = np.random.default_rng(13)
    seed = (rng.normal(size=(w.n, 3)) * 3e4, rng.normal(size=(w.n, 3)) * 3e4)
    _, gm, _, gs, _ = _gpu_grad([w], [state], 6, [seed], K=3, clip=1)
    g, _, _ = _oracle_grad(w, state, 6, seed, clip=1)
    assert rel_err(gm[0], g["material"]).max() < BAR
    e = rel_err(gs["x"], g["x"])
    assert np.quantile(e, 0.99) < BAR


@pytest.mark.parametrize("mode", [1, 2])
def test_regularised_adjoint_matches_oracle(mode):
    """Dynamic scaling (1) and normalisation (2) of the particles' x, v, F
    adjoints and of the grid's velocity and mass adjoints, as whole vectors
    per substep (Sec. III-E), with the paper's oom* = 4 and delta = 1e-6: the
    GPU's per-CTA statistics and deferred grid factors against the oracle,
    which regularises each vector where it forms. Seeds of 1e6 make the
    scaling act from the first reversed substep."""
    w = _contact_workload()
    state = _strained_state(w, 21)
    rng = np.random.default_rng(22)
    d = np.array([1.0, -0.5, 0.3])
    seed = ((d + 0.1 * rng.normal(size=(w.n, 3))) * 1e6, (1e-3 * d + 1e-4 * rng.normal(size=(w.n, 3))) * 1e6)
    nsub = 8
    _, gm, gt, gs, ga = _gpu_grad([w], [state], nsub, [seed], K=3, grad_scale=mode)
    g, ga_ref, _ = _oracle_grad(w, state, nsub, seed, grad_scale=mode)
    print("material gpu", gm[0], "oracle", g["material"])
    assert rel_err(gm[0], g["material"]).max() < BAR
    for k in ("x", "v", "C", "F"):
        e = rel_err(gs[k].reshape(w.n, -1), g[k].reshape(w.n, -1))
        print(k, "state-grad max rel err", e.max(), "p99", np.quantile(e, 0.99))
        assert np.quantile(e, 0.99) < BAR
    assert np.abs(ga_ref).max() > 0
    e = rel_err(ga[0][0][:, :4], ga_ref[:, :4])
    print("action grad max rel err", e.max())
    assert e.max() < BAR
    # the regularisation acted: the plain parameter gradient differs
    g0, _, _ = _oracle_grad(w, state, nsub, seed)
    assert not np.allclose(g0["material"], g["material"], rtol=0.05)


@pytest.mark.parametrize("K", [4, 12])
def test_fused_adjoint_equals_unfused(K):
    """The fused P2G/G2P adjoint (ping-pong grid adjoints, segment ends
    unfused) gives the separate kernels' gradients up to the order of the
    float atomic sums."""
    w = _contact_workload()
    state = _strained_state(w, 31)
    seed = _seed(w, 32)
    nsub = 12
    _, gm1, _, gs1, ga1 = _gpu_grad([w], [state], nsub, [seed], K=K, fuse=1)
    _, gm0, _, gs0, ga0 = _gpu_grad([w], [state], nsub, [seed], K=K, fuse=0)
    assert rel_err(gm1[0], gm0[0]).max() < 1e-3
    for k in ("x", "v", "C", "F"):
        e = rel_err(gs1[k].reshape(w.n, -1), gs0[k].reshape(w.n, -1))
        assert np.quantile(e, 0.99) < 1e-3, k
    assert rel_err(ga1[0][0], ga0[0][0]).max() < 1e-3


def test_non_finite_adjoint_seed_is_reported_and_the_handle_recovers():
    """A NaN in the dL/dx seed spreads through the adjoint (the gradient
    problem that Sec. III-E's clipping addresses): mpm_backward returns
    MPM_ERR_NON_FINITE, and the same handle then gives, for a finite seed,
    the gradients of a fresh handle: the material gradient within the 2e-2
    bar, the state adjoints within three times the spread of two fresh runs
    (float atomics reorder the sums from run to run)."""
    w = W.cfg_small()
    opts = mpm.make_options(checkpoint_every=16)
    nsub = 40
    g = np.full((w.n, 3), 1.0 / w.n, np.float32)
    bad = g.copy()
    bad[17, 1] = np.nan

    def run(sim):
        sim.reset()
        sim.forward(nsub, record=True)
        gm, _ = sim.backward(dL_dx=g)
        return gm, sim.state_grad()

    with mpm.simulation_from_workloads([w], opts) as sim:
        sim.forward(nsub, record=True)
        with pytest.raises(mpm.MpmError) as e:
            sim.backward(dL_dx=bad)
        assert e.value.code == -5
        gm, sg = run(sim)
    with mpm.simulation_from_workloads([w], opts) as fresh:
        gm_ref, sg_ref = run(fresh)
    with mpm.simulation_from_workloads([w], opts) as fresh2:
        _, sg_ref2 = run(fresh2)
    assert np.isfinite(gm).all()
    print("recovered", gm[0], "fresh", gm_ref[0])
    assert (rel_err(gm[0], gm_ref[0]) < 2e-2).all()
    for k in ("x", "v", "C", "F"):
        assert np.isfinite(sg[k]).all(), k
        spread = np.linalg.norm(sg_ref2[k] - sg_ref[k])
        dev = np.linalg.norm(sg[k] - sg_ref[k])
        scale = np.linalg.norm(sg_ref[k])
        print(k, "recovered - fresh", dev / scale, "fresh - fresh", spread / scale)
        assert dev <= 3 * spread + 1e-3 * scale, k


def test_backward_without_record_fails_cleanly():
    w = _contact_workload()
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(2)
        with pytest.raises(mpm.MpmError) as e:
            sim.backward(dL_dx=np.zeros((w.n, 3), np.float32))
        assert e.value.code == -6
        sim.forward(2, record=True)
        sim.backward(dL_dx=np.zeros((w.n, 3), np.float32))
        with pytest.raises(mpm.MpmError):
            sim.backward(dL_dx=np.zeros((w.n, 3), np.float32))   # the record is consumed


def test_full_size_adjoint_against_oracle():
    """1,048,576 particles on the 128^3 grid in the bench's state (the skill
    at substep 600, shovel inserting): a 4-substep recorded rollout and its
    backward under the MSE loss against a shifted target; the material and
    skill gradients and sampled state adjoints against the oracle's FP64
    adjoint of the same rollout from the same FP32 start state."""
    w = W.cfg_1m()
    start = 600
    with mpm.simulation_from_workloads([w]) as sim:
        sim.forward(start)
        s0 = sim.get_state()
    state = (s0["x"], s0["v"], s0["C"], s0["F"])
    nsub = 4
    target = (w.x0 + np.array([0.003, -0.002, 0.001], np.float32)).astype(np.float32)
    with mpm.simulation_from_workloads([w], mpm.make_options(checkpoint_every=2)) as sim:
        sim.set_substep(start)
        sim.set_state(*state)
        sim.forward(nsub, record=True)
        L, gxs = sim.loss_mse(target)
        gm, gt = sim.backward(dL_dx=gxs)
        gs = sim.state_grad()
        xs = sim.get_state()["x"]
    p = oracle_params(w)
    poses = oracle_poses(w, start + nsub)[start:]
    x, v, C, F = [np.asarray(a, np.float64).reshape(w.n, -1) for a in state]
    st, r = oracle.rollout(p, x, v, C, F, poses)
    assert st == 0
    Lr, gx = oracle.mse_loss(r["x"], target)
    assert np.isclose(L[0], Lr, rtol=1e-5)
    st, g = oracle.rollout_adjoint(p, x, v, C, F, poses, gx=gx)
    assert st == 0
    acts, jac = oracle_actions(w)
    ga = oracle.pose_table_adjoint(acts.shape[0], w.traj.substeps_per_action, w.dt,
                                   np.concatenate([np.zeros((start, 8)), g["poses"]]))
    gt_ref = np.einsum("tk,tkj->j", ga, jac)
    print("full-size material gpu", gm[0], "oracle", g["material"])
    print("full-size theta gpu", gt[0], "oracle", gt_ref)
    assert rel_err(gm[0], g["material"]).max() < BAR
    assert rel_err(gt[0], gt_ref).max() < BAR
    rng = np.random.default_rng(17)
    idx = rng.choice(w.n, 4096, replace=False)
    e = rel_err(gs["x"][idx], g["x"][idx])
    assert np.quantile(e, 0.99) < BAR


def test_full_size_batch_adjoint_against_oracle():
    """The 64 uneven instances (20k-192k particles, 64^3-96^3 grids, each
    with its own material and shovel) in one handle, as the bench's batched
    leg runs them: a 4-substep recorded rollout from their state after 200
    substeps and its backward under each instance's MSE loss against a
    shifted target; every instance's loss, material gradient and sampled
    state adjoints against the oracle's FP64 adjoint of that instance (the
    threaded oracle, which its own tests pin to its serial loops). The beds
    have settled by then: in the first substeps from the unstrained lattice
    the trace of the log strain sits at zero, where the return mapping's
    apex test (Eqs. (6)-(7)) flips on rounding and the nu and phi gradients
    follow the rounding, not the method."""
    import os
    ws = W.batch_uneven(64)
    offs = np.concatenate([[0], np.cumsum([w.n for w in ws])])
    start, nsub = 200, 4
    with mpm.simulation_from_workloads(ws) as sim:
        sim.forward(start)
        s0 = sim.get_state()
    target = np.concatenate([w.x0 + np.array([0.003, -0.002, 0.001], np.float32) for w in ws]).astype(np.float32)
    with mpm.simulation_from_workloads(ws, mpm.make_options(checkpoint_every=2)) as sim:
        sim.set_substep(start)
        sim.set_state(s0["x"], s0["v"], s0["C"], s0["F"])
        sim.forward(nsub, record=True)
        L, gxs = sim.loss_mse(target)
        gm, _ = sim.backward(dL_dx=gxs)
        gs = sim.state_grad()
    rng = np.random.default_rng(23)
    oracle.set_threads(os.cpu_count() or 1)
    worst_m, worst_x = 0.0, 0.0
    try:
        for i, w in enumerate(ws):
            sl = slice(offs[i], offs[i + 1])
            n = w.n
            x, v, C, F = [np.asarray(s0[k][sl], np.float64).reshape(n, -1) for k in ("x", "v", "C", "F")]
            p = oracle_params(w)
            poses = oracle_poses(w, start + nsub)[start:]
            st, r = oracle.rollout(p, x, v, C, F, poses)
            assert st == 0
            Lr, gx = oracle.mse_loss(r["x"], target[sl])
            assert np.isclose(L[i], Lr, rtol=1e-5), (i, L[i], Lr)
            st, g = oracle.rollout_adjoint(p, x, v, C, F, poses, gx=gx)
            assert st == 0
            em = rel_err(gm[i], g["material"]).max()
            worst_m = max(worst_m, em)
            assert em < BAR, (i, gm[i], g["material"])
            idx = rng.choice(n, min(n, 512), replace=False)
            ex = np.quantile(rel_err(gs["x"][sl][idx], g["x"][idx]), 0.99)
            worst_x = max(worst_x, ex)
            assert ex < BAR, (i, ex)
    finally:
        oracle.set_threads(1)
    print(f"full-size batch adjoint: worst material rel err {worst_m:.2e}, worst x-bar p99 {worst_x:.2e}")


def test_sorted_segments_give_the_same_gradients():
    """Sorting the particles at every segment start (the backward undoes
    each permutation on the adjoint) changes only the order of the float
    sums: material gradients and state adjoints agree to 1e-4."""
    w = _contact_workload()
    rng = np.random.default_rng(31)
    perm = rng.permutation(w.n)
    w.x0 = w.x0[perm]
    state = _strained_state(w, 14)
    seed = _seed(w, 15)
    res = []
    for sort_every in (1, 0):
        opts = mpm.make_options(checkpoint_every=4, sort_every=sort_every)
        with mpm.simulation_from_workloads([w], opts) as sim:
            sim.set_state(*state)
            sim.forward(12, record=True)
            gm, _ = sim.backward(dL_dx=seed[0].astype(np.float32), dL_dv=seed[1].astype(np.float32))
            res.append((gm[0], sim.state_grad()))
    assert rel_err(res[0][0], res[1][0]).max() < 1e-4
    for k in ("x", "v", "F"):
        a, b = res[0][1][k], res[1][1][k]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), k
    g, _, _ = _oracle_grad(w, state, 12, seed)
    assert rel_err(res[0][0], g["material"]).max() < BAR


def test_ill_conditioned_particles_take_the_fp64_kernels():
    """About 15% of the particles start with sigma_min / sigma_max = 4e-4,
    below the 1e-3 at which the FP32 SVD hands a particle to the FP64
    constitutive kernels (forward and adjoint). State and gradients must still
    match the oracle, and the library must report those hand-offs."""
    w = _contact_workload()
    x, v, C, F = _strained_state(w, 5)
    rng = np.random.default_rng(6)
    bad = rng.random(w.n) < 0.15
    for i in np.nonzero(bad)[0]:
        F[i] = (W.random_rotation(rng) @ np.diag([1.0, 0.95, 4e-4]) @ W.random_rotation(rng)).astype(np.float32)
    state = (x, v, C, F)
    seed = _seed(w, 7)
    nsub = 3
    opts = mpm.make_options(checkpoint_every=50)
    with mpm.simulation_from_workloads([w], opts) as sim:
        sim.set_state(*state)
        sim.forward(nsub, record=True)
        out = sim.get_state()
        fb_fwd = sim.info()["fp64_fallbacks"]
        gm, _ = sim.backward(dL_dx=seed[0].astype(np.float32), dL_dv=seed[1].astype(np.float32))
        gs = sim.state_grad()
        fb_all = sim.info()["fp64_fallbacks"]
    print("FP64 hand-offs: forward", fb_fwd, "forward + adjoint", fb_all, "ill-conditioned", int(bad.sum()))
    assert fb_fwd >= bad.sum() and fb_all >= 2 * bad.sum()
    st, ref = oracle.rollout(oracle_params(w), *[np.asarray(a, np.float64) for a in state], oracle_poses(w, nsub))
    assert st == 0
    assert np.abs(out["x"] - ref["x"]).max() < 1e-5
    assert np.quantile(rel_err(out["v"], ref["v"]), 0.99) < 1e-2
    eF = rel_err(out["F"].reshape(w.n, 9)[bad], ref["F"].reshape(w.n, 9)[bad])
    print("F of the FP64 particles: max rel err", eF.max())
    assert eF.max() < 1e-3
    g, _, _ = _oracle_grad(w, state, nsub, seed)
    print("material gpu", gm[0], "oracle", g["material"])
    assert rel_err(gm[0], g["material"]).max() < BAR
    for k in ("x", "v", "C", "F"):
        e = rel_err(gs[k].reshape(w.n, -1), g[k].reshape(w.n, -1))
        print(k, "state-grad max rel err", e.max(), "p99", np.quantile(e, 0.99))
        assert np.quantile(e, 0.99) < BAR
        assert e.max() < 10 * BAR
