"""Pins of the oracle's skill-to-action mapping (Sec. III-B, Algorithm 2)
and its Jacobian to the closed forms the paper prints for rounded phase
lengths, to central differences of the mapping itself (exact for frozen
T_i), to the per-phase displacement totals of the phase equations, and to
the paper's printed constants (tests/golden/paper_numbers.json)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))

THETAS = [
    (0.5, 0.2, 0.8, 0.0, -0.5, 1.0),
    (-0.3, -0.6, 0.1, 0.7, 0.4, 0.2),
    (0.9, 0.45, -0.5, -0.8, 0.9, -0.4),
]


@pytest.mark.parametrize("theta", THETAS)
def test_summed_jacobian_matches_paper_closed_forms(theta):
    """The paper's d(a-bar)/d(theta) with rounded T (Sec. III-B) is the sum of
    the per-step derivatives over all steps and action components."""
    v_l, v_w, dt = 2.5, 25.0, 1e-3
    acts, T, jac = oracle.skill_actions(theta, v_l, v_w, dt)
    assert (T > 0).all()
    summed = jac.sum(axis=(0, 1))
    th_disp, th_rot, th_ins, th_pa, th_pd, th_lift = theta
    ph1 = th_rot * np.pi / 3
    ph2 = ph1 + np.pi / 2
    d2 = (th_ins + 1) * 0.03
    d3 = (th_pd + 1) * 0.1 + 0.04
    ph3 = (th_pa + 3) * np.pi / 3
    paper = [
        0.12,
        np.pi / 3 - d2 * np.pi / 3 * (np.sin(ph1 + np.pi / 2) + np.cos(ph1 + np.pi / 2)) - np.pi / 3,
        0.03 * (np.cos(ph2) - np.sin(ph2)),
        np.pi * d3 / 3 * (np.cos(ph3) - np.sin(ph3)),
        0.1 * (np.cos(ph3) + np.sin(ph3)),
    ]
    assert np.allclose(summed[:5], paper, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("theta", THETAS)
def test_jacobian_matches_fd_with_frozen_T(theta):
    v_l, v_w, dt = 2.5, 25.0, 1e-3
    acts, T, jac = oracle.skill_actions(theta, v_l, v_w, dt)
    h = 1e-7
    for j in range(6):
        tp, tm = np.array(theta, float), np.array(theta, float)
        tp[j] += h
        tm[j] -= h
        ap, Tp, _ = oracle.skill_actions(tp, v_l, v_w, dt)
        am, Tm, _ = oracle.skill_actions(tm, v_l, v_w, dt)
        assert (Tp == T).all() and (Tm == T).all()
        fd = (ap - am) / (2 * h)
        assert np.allclose(jac[:, :, j], fd, rtol=0, atol=1e-8)


def test_phase_lengths_and_totals():
    """Demonstration skill at v_l = 2.5 m/s, v_w = 25 rad/s, dt = 1 ms:
    T = round of the phase equations; each phase moves its full d_i along its
    direction and phase 4 undoes the tilt of phase 1."""
    theta = W.DEMO_THETA
    acts, T, _ = oracle.skill_actions(theta, 2.5, 25.0, 1e-3)
    d1 = 0.12 * theta[0]
    ph1 = theta[1] * np.pi / 3
    d2 = (theta[2] + 1) * 0.03
    d3 = (theta[4] + 1) * 0.1 + 0.04
    ph3 = (theta[3] + 3) * np.pi / 3
    d4 = (theta[5] + 1) * 0.005
    assert list(T) == [24, 22, 36, 8]
    T1, T2, T3, T4 = T
    p1 = acts[:T1].sum(0)
    p2 = acts[T1:T1 + T2].sum(0)
    p3 = acts[T1 + T2:T1 + T2 + T3].sum(0)
    p4 = acts[T1 + T2 + T3:].sum(0)
    assert np.allclose(p1, [d1, 0, 0, ph1, 0, 0], atol=1e-15)
    assert np.allclose(p2, [d2 * np.cos(ph1 + np.pi / 2), -d2 * np.sin(ph1 + np.pi / 2), 0, 0, 0, 0], atol=1e-15)
    assert np.allclose(p3, [d3 * np.cos(ph3), d3 * np.sin(ph3), 0, 0, 0, 0], atol=1e-15)
    assert np.allclose(p4, [0, d4, 0, -ph1, 0, 0], atol=1e-15)
    assert np.isclose(d4, GOLDEN["skill_constants"]["d4"])   # theta_lift = 1 is the paper's constant lift


def test_zero_length_phases_give_zero_actions():
    acts, T, jac = oracle.skill_actions((0.0, 0.0, -1.0, 0.0, -1.0, 1.0), 2.5, 25.0, 1e-3)
    assert T[0] == 0 and T[1] == 0
    assert T[2] == 16 and T[3] == 4
    assert np.isfinite(acts).all() and np.isfinite(jac).all()


def test_pose_table_and_adjoint():
    rng = np.random.default_rng(4)
    acts = rng.normal(size=(7, 6)) * 0.01
    acts[:, 4:] = 0
    N, dt, nsub = 5, 1e-4, 40   # the table runs past the last action: the shovel then rests
    start = np.array([0.4, 0.5, 0.5, 0.1])
    poses = oracle.pose_table(start, acts, N, dt, nsub)
    # pose after step t's last substep = start + sum of the first t+1 actions
    for t in range(7):
        assert np.allclose(poses[(t + 1) * N - 1, :4], start + acts[:t + 1, :4].sum(0), atol=1e-15)
        assert np.allclose(poses[t * N:(t + 1) * N, 4:], acts[t, :4] / N / dt, atol=1e-12)
    assert np.allclose(poses[35:, 4:], 0) and np.allclose(poses[35:, :4], poses[34, :4])
    g = rng.normal(size=(nsub, 8))
    ga = oracle.pose_table_adjoint(7, N, dt, g)
    d = rng.normal(size=acts.shape)
    d[:, 4:] = 0
    h = 1e-6
    fd = ((oracle.pose_table(start, acts + h * d, N, dt, nsub) - oracle.pose_table(start, acts - h * d, N, dt, nsub))
          * g).sum() / (2 * h)
    assert np.isclose((ga * d).sum(), fd, rtol=1e-8)


def test_paper_initial_body():
    g = GOLDEN["initial_body"]
    x, vol = W.paper_bed(density=g["density_per_m3"], size=(g["box_m"][0], g["box_m"][2], g["box_m"][1]))
    assert x.shape[0] == g["n_particles"]
    assert np.isclose(vol, g["particle_volume_m3"], rtol=1e-12)
    assert (x >= 0).all() and (x.max(0) <= np.array([0.28, 0.07, 0.28]) + 1e-7).all()


def test_demo_theta_constants():
    g = GOLDEN["demo_skill"]
    assert W.DEMO_THETA[1:5] == (g["theta_rotate"], g["theta_insert_dist"], g["theta_push_angle"],
                                 g["theta_push_dist"])


# ---------------------------------------------------------------------------
# unrounded phase-1/4 step counts (Sec. III-B alternative; Appendix A)
# ---------------------------------------------------------------------------
V_L, V_W, DT = 2.5, 25.0, 1e-3


def _phase_sum(jac, T, phase, j):
    t0 = int(sum(T[:phase]))
    return jac[t0:t0 + T[phase]].sum(axis=(0, 1))[j]


def _cases(theta):
    d1 = theta[0] * 0.12
    ph1 = theta[1] * np.pi / 3
    d4 = (theta[5] + 1) * 0.005
    Tfd1, Tfp1 = abs(d1 / (V_L * DT)), abs(ph1 / (V_W * DT))
    Tfd4 = d4 / (V_L * DT)
    return Tfd1, Tfp1, Tfd4, d4


@pytest.mark.parametrize("theta", [
    (0.5, 0.2, 0.8, 0.0, -0.5, 1.0),     # phase 1: d dominates; phase 4: lift dominates
    (0.1, 0.8, 0.3, 0.2, 0.1, 0.5),      # phase 1: rotation dominates; phase 4: rotation dominates
    (0.9, 0.45, -0.5, -0.8, 0.9, -0.4),
])
def test_unrounded_summed_gradients_match_appendix_a(theta):
    """Appendix A's closed forms for the unrounded variant (positive
    theta_displace / theta_rotate branches and the third cases)."""
    acts, T, jac = oracle.skill_actions(theta, V_L, V_W, DT, unrounded=True)
    assert (T > 0).all()
    Tfd1, Tfp1, Tfd4, d4 = _cases(theta)
    th_d, th_r = theta[0], theta[1]
    T1, T4 = T[0], T[3]
    # d a[0:T1] / d theta_displace
    if Tfd1 >= Tfp1:
        want = T1 * (-np.pi * th_r * V_L * DT) / (0.36 * th_d ** 2)
    else:
        want = T1 * (0.12 * V_W * DT) / (abs(th_r) * np.pi / 3)
    assert np.isclose(_phase_sum(jac, T, 0, 0), want, rtol=1e-12, atol=1e-15)
    # d a[0:T1] / d theta_rotate
    if Tfp1 > Tfd1:
        want = T1 * (-0.36 * th_d * V_W * DT) / (th_r ** 2 * np.pi)
    else:
        want = T1 * (np.pi / 3 * V_L * DT) / (abs(th_d) * 0.12)
    assert np.isclose(_phase_sum(jac, T, 0, 1), want, rtol=1e-12, atol=1e-15)
    # d a[T1+T2+T3 : T] / d theta_rotate
    if Tfp1 >= Tfd4:
        want = T4 * (-3 * d4 * V_W * DT) / (th_r ** 2 * np.pi)
    else:
        want = T4 * (-np.pi * V_L * DT) / (3 * d4)
    assert np.isclose(_phase_sum(jac, T, 3, 1), want, rtol=1e-12, atol=1e-15)
    # phase 2 keeps the rounded T2: -d2 pi/3 (sin(ph1 + pi/2) + cos(ph1 + pi/2))
    d2 = (theta[2] + 1) * 0.03
    ph1 = th_r * np.pi / 3
    want = -d2 * np.pi / 3 * (np.sin(ph1 + np.pi / 2) + np.cos(ph1 + np.pi / 2))
    assert np.isclose(_phase_sum(jac, T, 1, 1), want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("theta", [
    (0.5, 0.2, 0.8, 0.0, -0.5, 1.0),
    (-0.5, 0.2, 0.8, 0.0, -0.5, 1.0),    # theta_displace < 0
    (0.1, -0.8, 0.3, 0.2, 0.1, 0.5),     # theta_rotate < 0, rotation dominating phases 1 and 4
    (-0.2, -0.9, -0.3, 0.6, -0.2, -0.7),
])
def test_unrounded_jacobian_matches_fd_with_frozen_T(theta):
    """Every branch against central differences of the mapping itself (for
    frozen integer step counts)."""
    acts, T, jac = oracle.skill_actions(theta, V_L, V_W, DT, unrounded=True)
    h = 1e-7
    for j in range(6):
        tp, tm = np.array(theta, float), np.array(theta, float)
        tp[j] += h
        tm[j] -= h
        ap, Tp, _ = oracle.skill_actions(tp, V_L, V_W, DT, unrounded=True)
        am, Tm, _ = oracle.skill_actions(tm, V_L, V_W, DT, unrounded=True)
        assert (Tp == T).all() and (Tm == T).all()
        fd = (ap - am) / (2 * h)
        assert np.allclose(jac[:, :, j], fd, rtol=1e-6, atol=1e-9), j


def test_unrounded_per_step_displacements():
    """Phases 1 and 4 move by (total / T_float) per step; phases 2 and 3 are
    those of the rounded mapping."""
    theta = (0.5, 0.2, 0.8, 0.0, -0.5, 1.0)
    ar, Tr, _ = oracle.skill_actions(theta, V_L, V_W, DT)
    au, Tu, _ = oracle.skill_actions(theta, V_L, V_W, DT, unrounded=True)
    assert (Tr == Tu).all()
    Tfd1, Tfp1, Tfd4, d4 = _cases(theta)
    T1, T2, T3, T4 = Tu
    assert np.allclose(au[:T1, 0], theta[0] * 0.12 / max(Tfd1, Tfp1), rtol=1e-14)
    assert np.allclose(au[:T1, 3], theta[1] * np.pi / 3 / max(Tfd1, Tfp1), rtol=1e-14)
    assert np.array_equal(au[T1:T1 + T2 + T3], ar[T1:T1 + T2 + T3])
    assert np.allclose(au[T1 + T2 + T3:, 1], d4 / max(Tfp1, Tfd4), rtol=1e-14)
