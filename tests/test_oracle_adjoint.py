"""Pin of the oracle's hand-written reverse-mode adjoint (Sec. III-D,
Appendix B) to central finite differences of its own FP64 forward on tiny
inputs, away from branch switches of the piecewise-smooth model."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300.workloads import lattice_bed, strained_F


def _scenario(name):
    rng = np.random.default_rng(sum(map(ord, name)))
    res = 12
    dx = 1.0 / res
    p = oracle.Params(res=(res,) * 3, dx=dx, dt=2e-4, gravity=(0.0, -9.8, 0.0), bound=3, E=1e5, nu=0.3,
                      rho=1500.0, phi_deg=30.0, vol=dx ** 3 / 8, shovel_on=0, friction=0.4)
    nsub = 8
    if name == "elastic":
        x = lattice_bed(1, (1, 1, 1), (5.2 * dx, 5.1 * dx, 5.3 * dx), dx)
        F = strained_F(rng, x.shape[0], 0.002, (-0.01, -0.012, -0.008))
        v = rng.normal(size=(x.shape[0], 3)) * 0.05
        C = rng.normal(size=(x.shape[0], 9)) * 0.2
    elif name == "plastic":
        x = lattice_bed(2, (2, 1, 2), (5.1 * dx, 5.2 * dx, 5.05 * dx), dx)
        F = strained_F(rng, x.shape[0], 0.005, (0.03, -0.06, 0.0))
        v = rng.normal(size=(x.shape[0], 3)) * 0.05
        C = rng.normal(size=(x.shape[0], 9)) * 0.5
    elif name == "contact":
        p.shovel_on = 1
        p.shovel_half = (0.06, 0.1, 0.1)
        x = lattice_bed(3, (2, 1, 1), (4.6 * dx, 4.2 * dx, 5.1 * dx), dx)
        F = strained_F(rng, x.shape[0], 0.002, (-0.01, -0.012, -0.008))
        v = np.tile([0.4, -0.1, 0.05], (x.shape[0], 1)) + rng.normal(size=(x.shape[0], 3)) * 0.02
        C = rng.normal(size=(x.shape[0], 9)) * 0.2
    elif name == "walls":
        x = lattice_bed(4, (2, 1, 1), (5.1 * dx, 3.05 * dx, 5.2 * dx), dx)
        F = strained_F(rng, x.shape[0], 0.002, (-0.01, -0.012, -0.008))
        v = np.tile([0.1, -0.3, 0.0], (x.shape[0], 1)) + rng.normal(size=(x.shape[0], 3)) * 0.02
        C = rng.normal(size=(x.shape[0], 9)) * 0.2
    else:
        raise KeyError(name)
    n = x.shape[0]
    poses = np.zeros((nsub, 8))
    if name == "contact":
        # box whose +x face cuts through the particles' stencils, pitched and moving
        for s in range(nsub):
            poses[s] = [7.1 * dx + 0.002 * s, 2.0 * dx, 5.6 * dx, 0.05 + 0.01 * s, 0.3, -0.1, 0.02, 0.4]
    state = dict(x=x.astype(np.float64), v=v, C=C.reshape(n, 9), F=F.reshape(n, 9))
    w = dict(gx=rng.normal(size=(n, 3)), gv=rng.normal(size=(n, 3)) * 1e-3,
             gC=rng.normal(size=(n, 9)) * 1e-4, gF=rng.normal(size=(n, 9)) * 1e-2)
    return p, state, poses, w


def _loss(p, st, poses, w):
    status, s = oracle.rollout(p, st["x"], st["v"], st["C"], st["F"], poses)
    assert status == 0
    n = st["x"].shape[0]
    return ((w["gx"] * s["x"]).sum() + (w["gv"] * s["v"]).sum() + (w["gC"] * s["C"].reshape(n, 9)).sum()
            + (w["gF"] * s["F"].reshape(n, 9)).sum())


def _rel_close(a, b, tol):
    return abs(a - b) <= tol * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("name", ["elastic", "plastic", "contact", "walls"])
def test_rollout_adjoint_matches_central_fd(name):
    p, st, poses, w = _scenario(name)
    status, g = oracle.rollout_adjoint(p, st["x"], st["v"], st["C"], st["F"], poses, **w)
    assert status == 0
    tol = 1e-6
    # material parameters
    for i, key in enumerate(["E", "nu", "rho", "phi_deg"]):
        base = getattr(p, key)
        h = 1e-6 * base
        setattr(p, key, base + h); lp = _loss(p, st, poses, w)
        setattr(p, key, base - h); lm = _loss(p, st, poses, w)
        setattr(p, key, base)
        fd = (lp - lm) / (2 * h)
        assert _rel_close(g["material"][i], fd, 1e-5), (name, key, g["material"][i], fd)
    # initial state, along random directions
    rng = np.random.default_rng(99)
    scale = {"x": 1e-6, "v": 1e-6, "C": 1e-5, "F": 1e-6}
    for key in ["x", "v", "C", "F"]:
        d = rng.normal(size=st[key].shape)
        h = scale[key]
        sp = dict(st); sp[key] = st[key] + h * d
        sm = dict(st); sm[key] = st[key] - h * d
        fd = (_loss(p, sp, poses, w) - _loss(p, sm, poses, w)) / (2 * h)
        ad = (g[key].reshape(d.shape) * d).sum()
        assert _rel_close(ad, fd, tol), (name, key, ad, fd)
    # shovel pose table
    if p.shovel_on:
        d = rng.normal(size=poses.shape)
        h = 1e-5     # poses are O(0.1-1); smaller steps are dominated by rounding
        fd = (_loss(p, st, poses + h * d, w) - _loss(p, st, poses - h * d, w)) / (2 * h)
        ad = (g["poses"] * d).sum()
        assert abs(ad) > 0
        assert _rel_close(ad, fd, tol), (name, "poses", ad, fd)


def test_contact_scenario_touches_the_shovel():
    """The contact scenario must exercise the contact branch (otherwise its
    pose gradient check would be vacuous)."""
    p, st, poses, w = _scenario("contact")
    status, g = oracle.rollout_adjoint(p, st["x"], st["v"], st["C"], st["F"], poses, **w)
    assert np.abs(g["poses"][:, 4:]).max() > 0


def test_clipping_bounds_the_adjoints():
    """With clipping on (Sec. III-E) the state adjoint handed back stays
    within the clip bound."""
    p, st, poses, w = _scenario("plastic")
    w = {k: v * 1e9 for k, v in w.items()}
    p.clip_grads, p.clip_value = 1, 1e4
    status, g = oracle.rollout_adjoint(p, st["x"], st["v"], st["C"], st["F"], poses, **w)
    assert status == 0
    p.clip_grads = 0
    status, g0 = oracle.rollout_adjoint(p, st["x"], st["v"], st["C"], st["F"], poses, **w)
    assert np.abs(g0["x"]).max() > 1e4
    # the returned adjoints are one substep past the last clip; bounded by a
    # small multiple of the clip value times the substep's Jacobian norm
    assert np.abs(g["x"]).max() < np.abs(g0["x"]).max()


@pytest.mark.parametrize("name", ["elastic", "plastic", "contact", "walls"])
def test_material_gradient_is_invariant_under_scaling_E_and_rho(name):
    """Scaling E and rho by the same factor scales the stresses (mu and
    lambda are linear in E) and the particle masses alike; the grid velocity
    is their quotient, so no trajectory changes, and a loss of the state has
    E dL/dE + rho dL/drho = 0. The two terms come through different chains
    (mu, lambda and the stress adjoint; m_p = rho V_p and the transfer
    adjoint), so a wrong factor in either breaks the identity."""
    p, st, poses, w = _scenario(name)
    status, g = oracle.rollout_adjoint(p, st["x"], st["v"], st["C"], st["F"], poses, **w)
    assert status == 0
    tE, trho = p.E * g["material"][0], p.rho * g["material"][2]
    assert abs(tE) > 0
    assert abs(tE + trho) <= 1e-9 * max(abs(tE), abs(trho)), (tE, trho)
