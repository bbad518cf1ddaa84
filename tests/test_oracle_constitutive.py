"""Pins of the oracle's SVD, material constants and constitutive model to
facts fixed outside the oracle: LAPACK's SVD, textbook elasticity
identities, the yield surface of Eq. (6) after projection (Eq. (7)),
Appendix B's closed-form partials of delta_gamma, and finite differences
of the SVK energy of Eq. (3)."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300.workloads import random_rotation


def _mats(rng):
    mats = [rng.normal(size=(3, 3)) for _ in range(300)]
    R1, R2 = random_rotation(rng), random_rotation(rng)
    mats += [
        np.eye(3), -np.eye(3), np.zeros((3, 3)), np.diag([1.0, 1.0, 1e-9]), np.diag([2.0, 2.0, 1.0]),
        R1 @ np.diag([1.0, 1.0, 1.0]) @ R2, R1 @ np.diag([1.3, 1.3, 0.7]) @ R2, R1 @ np.diag([1.0, 1.0 + 1e-10, 0.9]) @ R2,
        np.outer([1.0, 2.0, 3.0], [0.5, -1.0, 2.0]), R1 @ np.diag([1.0, 0.8, -0.5]) @ R2,
        R1 @ np.diag([1e3, 1.0, 1e-3]) @ R2,
    ]
    return mats


def test_svd_matches_lapack():
    rng = np.random.default_rng(7)
    for F in _mats(rng):
        U, S, V = oracle.svd3(F)
        ref = np.linalg.svd(F, compute_uv=False)
        scale = max(1.0, ref[0])
        assert np.allclose(np.abs(S), ref, rtol=0, atol=1e-13 * scale)
        assert np.allclose(U @ np.diag(S) @ V.T, F, rtol=0, atol=2e-13 * scale)
        assert np.allclose(U.T @ U, np.eye(3), atol=1e-13)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(U) - 1) < 1e-12 and abs(np.linalg.det(V) - 1) < 1e-12
        assert S[0] >= S[1] - 1e-15 >= abs(S[2]) - 2e-15
        d = np.linalg.det(F)
        if abs(d) > 1e-12:
            assert np.sign(S[2]) == np.sign(d)


def test_lame_and_friction_coefficient():
    for E, nu in [(1e5, 0.3), (3e5, 0.25), (5e4, 0.1), (2e5, 0.4)]:
        mu, lam, _ = oracle.material(E, nu, 30.0)
        # inverse relations of isotropic elasticity
        assert np.isclose(mu * (3 * lam + 2 * mu) / (lam + mu), E, rtol=1e-14)
        assert np.isclose(lam / (2 * (lam + mu)), nu, rtol=1e-14)
    # alpha_f at 30 deg: sin = 1/2 -> sqrt(2/3) * 1 / 2.5
    _, _, a30 = oracle.material(1e5, 0.3, 30.0)
    assert np.isclose(a30, np.sqrt(2.0 / 3.0) / 2.5, rtol=1e-14)
    _, _, a90 = oracle.material(1e5, 0.3, 90.0)
    assert np.isclose(a90, np.sqrt(2.0 / 3.0), rtol=1e-14)


def _trial(rng, eps):
    return random_rotation(rng) @ np.diag(np.exp(eps)) @ random_rotation(rng)


def _yield(e, beta):
    dev = e - e.mean()
    return np.linalg.norm(dev) + beta * e.sum()


@pytest.mark.parametrize("E,nu,phi", [(1e5, 0.3, 30.0), (3e5, 0.25, 35.0), (5e4, 0.4, 10.0)])
def test_drucker_prager_return_cases(E, nu, phi):
    rng = np.random.default_rng(11)
    mu, lam, alpha = oracle.material(E, nu, phi)
    beta = (3 * lam + 2 * mu) / (2 * mu) * alpha
    seen = set()
    for _ in range(400):
        eps = rng.normal(size=3) * 0.05 + rng.normal() * 0.03
        Ft = _trial(rng, eps)
        Fn, tau, info = oracle.constitutive(Ft, mu, lam, alpha)
        case = int(info[0])
        seen.add(case)
        s_new = np.linalg.svd(Fn, compute_uv=False)
        e_new = np.log(s_new)
        if case == 0:      # tension: projected to the cone tip, S^ = I
            assert eps.sum() > 0
            assert np.allclose(Fn.T @ Fn, np.eye(3), atol=1e-13)
            assert np.allclose(tau, 0, atol=1e-9)
        elif case == 1:    # inside the cone: unchanged
            assert eps.sum() <= 0 and _yield(eps, beta) <= 1e-12
            assert np.allclose(Fn, Ft, atol=1e-14)
        else:              # projected onto the cone surface
            assert eps.sum() <= 0 and _yield(eps, beta) > 0
            assert abs(_yield(e_new, beta)) < 1e-12
            assert np.isclose(e_new.sum(), eps.sum(), atol=1e-13)   # projection is deviatoric
            # the deviatoric direction is kept (radial return)
            d_old, d_new = eps - eps.mean(), np.sort(e_new - e_new.mean())
            d_old_s = np.sort(d_old)
            assert np.allclose(d_new / np.linalg.norm(d_new), d_old_s / np.linalg.norm(d_old_s), atol=1e-10)
    assert seen == {0, 1, 2}


def test_appendix_b_dgamma_partials():
    """Appendix B: d(delta_gamma)/d(mu) = -3 lam tr(eps) alpha / (2 mu^2) and
    d(delta_gamma)/d(lam) = 3 tr(eps) alpha / (2 mu)."""
    rng = np.random.default_rng(3)
    mu, lam, alpha = oracle.material(1e5, 0.3, 30.0)
    for _ in range(20):
        eps = np.array([0.03, -0.06, 0.0]) + 0.01 * rng.normal(size=3)
        Ft = _trial(rng, eps)
        tr = np.log(np.linalg.svd(Ft, compute_uv=False)).sum()
        h = 1e-4 * mu
        dg = lambda m, l: oracle.constitutive(Ft, m, l, alpha)[2][2]
        fd_mu = (dg(mu + h, lam) - dg(mu - h, lam)) / (2 * h)
        fd_lam = (dg(mu, lam + h) - dg(mu, lam - h)) / (2 * h)
        assert np.isclose(fd_mu, -3 * lam * tr * alpha / (2 * mu ** 2), rtol=1e-7)
        assert np.isclose(fd_lam, 3 * tr * alpha / (2 * mu), rtol=1e-7)


def _svk_energy(F, mu, lam):
    s = np.linalg.svd(F, compute_uv=False)
    l = np.log(s)
    return mu * (l * l).sum() + 0.5 * lam * l.sum() ** 2


def test_kirchhoff_stress_is_energy_derivative_times_Ft():
    """tau = P F^T with P = d psi / d F of the SVK energy in log strain
    (Eqs. (3)-(4)); checked by central differences of psi on elastic states."""
    rng = np.random.default_rng(5)
    mu, lam, alpha = oracle.material(1e5, 0.3, 30.0)
    for _ in range(10):
        eps = np.array([-0.010, -0.012, -0.008]) + 0.001 * rng.normal(size=3)
        F = _trial(rng, eps)
        Fn, tau, info = oracle.constitutive(F, mu, lam, alpha)
        assert int(info[0]) == 1
        P = np.zeros((3, 3))
        h = 1e-6
        for i in range(3):
            for j in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += h
                Fm[i, j] -= h
                P[i, j] = (_svk_energy(Fp, mu, lam) - _svk_energy(Fm, mu, lam)) / (2 * h)
        assert np.allclose(tau, P @ F.T, rtol=0, atol=1e-6 * np.abs(tau).max())


def test_small_strain_limit_is_linear_elasticity():
    mu, lam, alpha = oracle.material(1e5, 0.3, 30.0)
    rng = np.random.default_rng(9)
    for _ in range(10):
        A = rng.normal(size=(3, 3)) * 1e-7
        e = 0.5 * (A + A.T) - 3e-7 * np.eye(3)     # compressive, inside the cone
        _, tau, info = oracle.constitutive(np.eye(3) + e, mu, lam, alpha)
        assert int(info[0]) == 1
        lin = 2 * mu * e + lam * np.trace(e) * np.eye(3)
        assert np.allclose(tau, lin, rtol=0, atol=1e-5 * np.abs(lin).max())


def _cons_scalar(Ft, mu, lam, alpha, gFn, gtau):
    Fn, tau, _ = oracle.constitutive(Ft, mu, lam, alpha)
    return (gFn * Fn).sum() + (gtau * tau).sum()


CASES = {
    "tension": [0.03, 0.01, 0.02],
    "elastic": [-0.010, -0.012, -0.008],
    "cone": [0.03, -0.06, 0.0],
    "isotropic": "iso",
    "cone_repeated": [0.02, 0.02, -0.08],
    "elastic_repeated": [-0.01, -0.01, -0.012],
}


@pytest.mark.parametrize("name", list(CASES))
def test_constitutive_adjoint_matches_fd(name):
    rng = np.random.default_rng(sum(map(ord, name)))
    mu, lam, alpha = oracle.material(1e5, 0.3, 30.0)
    eps = CASES[name]
    # all singular values equal, strictly inside the cone (the identity itself
    # sits on the tr(eps) = 0 apex boundary where the map has a kink)
    Ft = np.exp(-0.01) * random_rotation(rng) if eps == "iso" else _trial(rng, np.array(eps))
    gFn, gtau = rng.normal(size=(3, 3)), rng.normal(size=(3, 3)) / mu
    gFt, gmu, glam, galpha = oracle.constitutive_adjoint(Ft, mu, lam, alpha, gFn, gtau)
    h = 1e-7
    fd = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            Fp, Fm = Ft.copy(), Ft.copy()
            Fp[i, j] += h
            Fm[i, j] -= h
            fd[i, j] = (_cons_scalar(Fp, mu, lam, alpha, gFn, gtau) - _cons_scalar(Fm, mu, lam, alpha, gFn, gtau)) / (2 * h)
    scale = max(np.abs(fd).max(), 1e-12)
    assert np.allclose(gFt, fd, rtol=0, atol=2e-6 * scale), (gFt, fd)
    for val, (dm, dl, da) in [(gmu, (1, 0, 0)), (glam, (0, 1, 0)), (galpha, (0, 0, 1))]:
        hm, hl, ha = 1e-6 * mu * dm, 1e-6 * mu * dl, 1e-7 * da
        hh = hm + hl + ha
        f = lambda s: _cons_scalar(Ft, mu + s * hm, lam + s * hl, alpha + s * ha, gFn, gtau)
        ref = (f(1) - f(-1)) / (2 * hh)
        assert np.isclose(val, ref, rtol=1e-5, atol=1e-9 * max(1.0, abs(ref))), (name, val, ref)
