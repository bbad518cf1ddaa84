"""Pins of the oracle's P2G / grid update / G2P / advection (Algorithm 1)
to invariants and closed forms: partition of unity (exact mass), the APIC
momentum identities, uniform translation, free fall, wall and shovel
projections against hand-derived cases, and hydrostatic settling."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300.workloads import lattice_bed, strained_F


def _state(x, rng=None, v=None, C=None, F=None):
    n = x.shape[0]
    v = np.zeros((n, 3)) if v is None else v
    C = np.zeros((n, 9)) if C is None else C.reshape(n, 9)
    F = np.tile(np.eye(3).ravel(), (n, 1)) if F is None else F.reshape(n, 9)
    return x.astype(np.float64), v, C, F


def _free_params(res=16, **kw):
    p = oracle.Params(res=(res, res, res), dx=1.0 / res, dt=1e-4, gravity=(0, 0, 0), shovel_on=0,
                      vol=(1.0 / res) ** 3 / 8)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _cube(seed, res=16, cells=4):
    dx = 1.0 / res
    o = (res // 2 - cells // 2) * dx
    return lattice_bed(seed, (cells,) * 3, (o, o, o), dx).astype(np.float64)


def test_p2g_mass_and_momentum_exact():
    rng = np.random.default_rng(1)
    p = _free_params()
    x = _cube(1)
    n = x.shape[0]
    v = rng.normal(size=(n, 3))
    C = rng.normal(size=(n, 9)) * 5
    F = strained_F(rng, n, 0.02, (-0.01, -0.01, -0.01))
    x, v, C, F = _state(x, v=v, C=C, F=F)
    st, m, mv, vo = oracle.grid_of_substep(p, x, v, C, F, np.zeros(8))
    assert st == 0
    mp = p.rho * p.vol
    assert np.isclose(m.sum(), n * mp, rtol=1e-14)
    # sum_i w_ip = 1 and sum_i w_ip (x_i - x_p) = 0: the affine and stress terms add no momentum
    assert np.allclose(mv.reshape(-1, 3).sum(0), mp * v.sum(0), rtol=0, atol=1e-13 * mp * np.abs(v).sum())


def test_momentum_conserved_over_rollout():
    rng = np.random.default_rng(2)
    p = _free_params()
    x = _cube(2)
    n = x.shape[0]
    v = rng.normal(size=(n, 3)) * 0.1
    x, v, C, F = _state(x, v=v, F=strained_F(rng, n, 0.01, (-0.01, -0.01, -0.01)))
    mp = p.rho * p.vol
    P0 = mp * v.sum(0)
    st, s = oracle.rollout(p, x, v, C, F, np.zeros((20, 8)))
    assert st == 0
    P1 = mp * s["v"].sum(0)
    assert np.allclose(P1, P0, rtol=0, atol=1e-12 * mp * np.abs(v).sum())


def test_uniform_translation_is_preserved():
    p = _free_params()
    x = _cube(3)
    n = x.shape[0]
    v0 = np.array([0.3, -0.2, 0.1])
    x, v, C, F = _state(x, v=np.tile(v0, (n, 1)))
    k = 15
    st, s = oracle.rollout(p, x, v, C, F, np.zeros((k, 8)))
    assert st == 0
    assert np.allclose(s["v"], v0, atol=1e-13)
    assert np.allclose(s["C"], 0, atol=1e-9)
    assert np.allclose(s["F"], np.eye(3), atol=1e-12)
    assert np.allclose(s["x"], x + k * p.dt * v0, atol=1e-13)


def test_free_fall_closed_form():
    """x_n = x_0 + dt^2 g n (n+1) / 2 and v_n = n dt g for symplectic Euler
    on a body under gravity alone."""
    p = _free_params(gravity=(0.0, -9.8, 0.0))
    x = _cube(4)
    n = x.shape[0]
    x, v, C, F = _state(x)
    k = 25
    st, s = oracle.rollout(p, x, v, C, F, np.zeros((k, 8)))
    assert st == 0
    g = np.array([0.0, -9.8, 0.0])
    assert np.allclose(s["v"], k * p.dt * g, atol=1e-13)
    assert np.allclose(s["x"], x + p.dt ** 2 * g * k * (k + 1) / 2, atol=1e-13)
    assert np.allclose(s["C"], 0, atol=1e-9)


def test_walls_stop_outward_velocity():
    p = _free_params(gravity=(0.0, -9.8, 0.0), bound=3)
    dx = p.dx
    # a particle sitting on the floor layer, moving down and sideways
    x = np.array([[8.3 * dx, 3.2 * dx, 8.1 * dx]])
    x, v, C, F = _state(x, v=np.array([[0.5, -1.0, 0.0]]))
    st, m, mv, vo = oracle.grid_of_substep(p, x, v, C, F, np.zeros(8))
    assert st == 0
    act = m > 0
    j = np.arange(p.res[1])[None, :, None] * np.ones_like(m, dtype=int)
    floor = act & (j < p.bound)
    interior = act & (j >= p.bound)
    assert floor.any() and interior.any()
    assert np.all(vo[..., 1][floor] >= 0) and np.allclose(vo[..., 1][floor], 0)
    assert np.all(vo[..., 1][interior] < 0)
    assert np.allclose(vo[..., 0][act], 0.5, atol=1e-12)


def _shovel_params():
    return oracle.Params(shovel_half=(0.01, 0.075, 0.1), friction=0.5, shovel_on=1)


def test_shovel_projection_hand_cases():
    p = _shovel_params()
    pose = np.array([0.5, 0.2, 0.5, 0.0, 0.0, 0.0, 0.0, 0.0])
    inside_near_plus_x = np.array([0.5 + 0.009, 0.25, 0.5])   # nearest face: +x (normal (1,0,0))
    outside = np.array([0.6, 0.25, 0.5])
    # outside: untouched
    assert np.allclose(oracle.shovel_project(p, [-1, 0.3, 0], outside, pose), [-1, 0.3, 0])
    # separating (u.n >= 0): untouched
    assert np.allclose(oracle.shovel_project(p, [1, 0.3, 0], inside_near_plus_x, pose), [1, 0.3, 0])
    # approaching with small tangential speed: sticks (|u_t| <= mu |u_n|)
    assert np.allclose(oracle.shovel_project(p, [-1, 0.3, 0], inside_near_plus_x, pose), [0, 0, 0])
    # approaching with large tangential speed: slides with |u_t| reduced by mu |u_n|
    assert np.allclose(oracle.shovel_project(p, [-1, 2.0, 0], inside_near_plus_x, pose), [0, 1.5, 0])
    # frictionless: only the normal component is removed
    p0 = _shovel_params(); p0.friction = 0.0
    assert np.allclose(oracle.shovel_project(p0, [-1, 0.3, 0.2], inside_near_plus_x, pose), [0, 0.3, 0.2])
    # moving shovel: the projection acts on the relative velocity
    moving = pose.copy(); moving[4:7] = [2.0, 0.0, 0.0]
    assert np.allclose(oracle.shovel_project(p0, [0.0, 0.3, 0.0], inside_near_plus_x, moving), [2.0, 0.3, 0.0])


def test_shovel_rotation_convention():
    """A tilt psi turns the shovel's pointing direction (tip minus top) to
    (-sin psi, -cos psi, 0), the insertion direction of Algorithm 2's phase 2
    in the x-up plane; the box is spun about the tip with rate psidot."""
    p = _shovel_params(); p.friction = 0.0
    psi = 0.3
    pose = np.array([0.5, 0.3, 0.5, psi, 0, 0, 0, 0])
    along = np.array([np.sin(psi), np.cos(psi), 0.0])          # from tip towards the top
    across = np.array([np.cos(psi), -np.sin(psi), 0.0])        # local +x face normal
    q = pose[:3] + 0.05 * along + 0.009 * across               # just inside the +x face
    out = oracle.shovel_project(p, -across, q, pose)
    assert np.allclose(out, 0, atol=1e-14)
    # rigid rotation: a point at r from the tip moves with psidot * (r_y, -r_x, 0)
    pose2 = pose.copy(); pose2[7] = 4.0
    r = q - pose2[:3]
    vs = np.array([4.0 * r[1], -4.0 * r[0], 0.0])
    out2 = oracle.shovel_project(p, np.zeros(3) - across, q, pose2)
    un = (np.zeros(3) - across - vs) @ across
    assert un < 0
    expect = (np.zeros(3) - across) - un * across
    assert np.allclose(out2, expect, atol=1e-13)


@pytest.mark.slow
def test_hydrostatic_settling():
    """A sand layer confined by slip walls settles to sigma_yy(depth h) =
    -rho g h; the volume integral of tau_yy then equals -rho g times the
    integral of depth (15% tolerance)."""
    res = 16
    dx = 1.0 / res
    p = oracle.Params(res=(res, res, res), dx=dx, dt=5e-4, gravity=(0, -9.8, 0), shovel_on=0, bound=3,
                      E=1e5, nu=0.3, rho=1500.0, phi_deg=30.0, vol=dx ** 3 / 8)
    H = 6
    x = lattice_bed(11, (10, H, 10), (3 * dx, 3 * dx, 3 * dx), dx).astype(np.float64)
    n = x.shape[0]
    x, v, C, F = _state(x)
    mu, lam, alpha = oracle.material(p.E, p.nu, p.phi_deg)
    state = {"x": x, "v": v, "C": C, "F": F}
    lhs, rhs = [], []
    # the column rings in its fundamental mode (period ~ 4H/c ~ 400 substeps
    # here); average the stress integral over two periods after 800 substeps
    for it in range(32):
        st, state = oracle.rollout(p, state["x"], state["v"], state["C"].reshape(n, 9),
                                   state["F"].reshape(n, 9), np.zeros((50, 8)))
        assert st == 0
        if it >= 16:
            tyy = np.array([oracle.constitutive(Fi, mu, lam, alpha)[1][1, 1] for Fi in state["F"]])
            top = state["x"][:, 1].max() + 0.25 * dx
            depth = top - state["x"][:, 1]
            lhs.append(tyy.sum() * p.vol)
            rhs.append(-p.rho * 9.8 * depth.sum() * p.vol)
    assert np.isclose(np.mean(lhs), np.mean(rhs), rtol=0.15), (np.mean(lhs), np.mean(rhs))
    assert np.abs(state["v"]).max() < 0.2


def _angular_momentum(x, v, C, mp, dx):
    """APIC angular momentum about the origin: sum_p m_p (x_p x v_p) plus the
    affine part m_p eps : (C_p D)^T with D = sum_i w_ip d d^T = (dx^2 / 4) I
    for the quadratic B-spline."""
    C = C.reshape(-1, 3, 3)
    aff = np.stack([C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0], C[:, 1, 0] - C[:, 0, 1]], axis=1)
    return mp * (np.cross(x, v).sum(0) + 0.25 * dx * dx * aff.sum(0))


def test_angular_momentum_conserved_over_rollout():
    """APIC transfers conserve angular momentum, and the Kirchhoff stress of
    the isotropic SVK/Drucker-Prager model is symmetric, so it adds none:
    without gravity, walls or shovel the APIC angular momentum (with its
    affine part) is constant over a rollout, plastic flow included. A
    transposed C in the transfer, a wrong weight second moment or an
    asymmetric stress breaks it."""
    rng = np.random.default_rng(4)
    p = _free_params()
    x = _cube(4)
    n = x.shape[0]
    omega = np.array([0.3, -0.5, 0.8])
    ctr = x.mean(0)
    v = np.cross(omega, x - ctr) + rng.normal(size=(n, 3)) * 0.05
    C = rng.normal(size=(n, 9)) * 2.0
    x, v, C, F = _state(x, v=v, C=C, F=strained_F(rng, n, 0.05, (0.02, -0.08, 0.01)))
    mp = p.rho * p.vol
    L0 = _angular_momentum(x, v, C, mp, p.dx)
    st, s = oracle.rollout(p, x, v, C, F, np.zeros((20, 8)))
    assert st == 0
    L1 = _angular_momentum(s["x"], s["v"], s["C"], mp, p.dx)
    scale = mp * (np.abs(np.cross(x, v)).sum() + 0.25 * p.dx ** 2 * np.abs(C).sum())
    assert np.abs(L1 - L0).max() <= 1e-12 * scale, (L0, L1)
    # the affine part matters: without it the sums differ
    naive0, naive1 = mp * np.cross(x, v).sum(0), mp * np.cross(s["x"], s["v"]).sum(0)
    assert np.abs(naive1 - naive0).max() > 1e3 * np.abs(L1 - L0).max()
