"""FP64 CPU oracle for the DDBot MLS-MPM sand substep (arXiv 2510.17335).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA library in ``paper_2510_17335_gb300``; the only thing both sides
use is the seeded input generator module ``paper_2510_17335_gb300.workloads``,
which holds none of the method's arithmetic.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that x86 and Arm give the same bits). This module is
argument marshalling plus textbook definitions written in numpy: the MSE loss
of a final position set and its gradient, and the unnormalised Earth Mover's
distance of Eq. (1) with scipy's linear assignment as its one library step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")

OK = 0
E_INVAL = -1
E_DOMAIN = -4


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (idempotent)."""
    stale = force or not os.path.exists(_SO)
    if not stale:
        t = os.path.getmtime(_SO)
        stale = t < os.path.getmtime(_SRC) or t < os.path.getmtime(_HDR)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _declare(_lib)
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [
        ("res", ctypes.c_int * 3),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("bound", ctypes.c_int),
        ("E", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("phi_deg", ctypes.c_double),
        ("vol", ctypes.c_double),
        ("friction", ctypes.c_double),
        ("particle_collision", ctypes.c_int),
        ("sigma_min", ctypes.c_double),
        ("shovel_half", ctypes.c_double * 3),
        ("shovel_on", ctypes.c_int),
        ("clip_grads", ctypes.c_int),
        ("clip_value", ctypes.c_double),
        ("grad_scale", ctypes.c_int),
        ("oom_star", ctypes.c_double),
        ("grad_delta", ctypes.c_double),
    ]


@dataclass
class Params:
    """Simulation parameters (mirrors ``orc_params``)."""
    res: Sequence[int] = (32, 32, 32)
    dx: float = 1.0 / 32
    dt: float = 1e-4
    gravity: Sequence[float] = (0.0, -9.8, 0.0)
    bound: int = 3
    E: float = 1e5
    nu: float = 0.3
    rho: float = 1500.0
    phi_deg: float = 30.0
    vol: float = (1.0 / 32) ** 3 / 8
    friction: float = 0.5
    particle_collision: int = 1
    sigma_min: float = 1e-4
    shovel_half: Sequence[float] = (0.01, 0.075, 0.1)
    shovel_on: int = 1
    clip_grads: int = 0
    clip_value: float = 1e4
    grad_scale: int = 0          # 1 dynamic scaling, 2 normalisation (Sec. III-E)
    oom_star: float = 4.0
    grad_delta: float = 1e-6

    def c(self) -> _Params:
        p = _Params()
        p.res[:] = [int(r) for r in self.res]
        p.dx, p.dt = self.dx, self.dt
        p.gravity[:] = [float(g) for g in self.gravity]
        p.bound = self.bound
        p.E, p.nu, p.rho, p.phi_deg = self.E, self.nu, self.rho, self.phi_deg
        p.vol, p.friction = self.vol, self.friction
        p.particle_collision = self.particle_collision
        p.sigma_min = self.sigma_min
        p.shovel_half[:] = [float(h) for h in self.shovel_half]
        p.shovel_on, p.clip_grads, p.clip_value = self.shovel_on, self.clip_grads, self.clip_value
        p.grad_scale, p.oom_star, p.grad_delta = self.grad_scale, self.oom_star, self.grad_delta
        return p


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _ObsGrid(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cz", ctypes.c_double), ("size", ctypes.c_double), ("res", ctypes.c_int),
                ("tap", ctypes.c_double)]


@dataclass
class ObsGrid:
    """Observation / height-map square (Sec. III-A): res x res pixels of
    side size in the (x, z) plane, centred at (cx, cz); tap is the splat
    offset of the height map."""
    cx: float
    cz: float
    size: float = 0.24
    res: int = 40
    tap: float = 0.0

    def c(self):
        return _ObsGrid(self.cx, self.cz, self.size, self.res, self.tap)


def _declare(L):
    P = ctypes.POINTER(_Params)
    i64 = ctypes.c_int64
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_get_threads.restype = ctypes.c_int
    L.orc_svd3.argtypes = [_dp, _dp, _dp, _dp]
    L.orc_material.argtypes = [ctypes.c_double] * 3 + [_dp] * 3
    L.orc_constitutive.argtypes = [_dp] + [ctypes.c_double] * 4 + [_dp] * 3
    L.orc_constitutive_adjoint.argtypes = [_dp] + [ctypes.c_double] * 4 + [_dp] * 3 + [_dp] * 3
    L.orc_shovel_project.argtypes = [P, _dp, _dp, _dp, _dp]
    L.orc_substep.argtypes = [P, i64, _dp, _dp, _dp, _dp, _dp]
    L.orc_substep.restype = ctypes.c_int
    L.orc_rollout.argtypes = [P, i64, _dp, _dp, _dp, _dp, ctypes.c_int, _dp]
    L.orc_rollout.restype = ctypes.c_int
    L.orc_grid_of_substep.argtypes = [P, i64, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_grid_of_substep.restype = ctypes.c_int
    L.orc_rollout_adjoint.argtypes = ([P, i64] + [_dp] * 4 + [ctypes.c_int, _dp] + [_dp] * 4 + [_dp] * 4
                                      + [_dp, _dp])
    L.orc_rollout_adjoint.restype = ctypes.c_int
    L.orc_skill_actions.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    _dp, _ip, _dp]
    L.orc_skill_actions.restype = ctypes.c_int
    L.orc_pose_table.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]
    L.orc_pose_table_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
    L.orc_grad_op.argtypes = [P, _dp, i64]
    G = ctypes.POINTER(_ObsGrid)
    _fp = ctypes.POINTER(ctypes.c_float)
    _i64p = ctypes.POINTER(ctypes.c_int64)
    L.orc_surface_observation.argtypes = [G, i64, _fp, _i64p]
    L.orc_surface_observation.restype = ctypes.c_int
    L.orc_height_map.argtypes = [G, i64, _fp, _dp, _i64p]
    L.orc_hmd.argtypes = [G, i64, _fp, _dp, _dp]
    L.orc_hmd.restype = ctypes.c_double


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _arr(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out.copy()


def _opt(a, n, k):
    if a is None:
        return None
    return _arr(a, (n, k))


def _ptr(a):
    return None if a is None else _d(a)


# --------------------------------------------------------------------------
def svd3(F) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    F = _arr(F, (3, 3))
    U, S, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    _L().orc_svd3(_d(F), _d(U), _d(S), _d(V))
    return U, S, V


def material(E: float, nu: float, phi_deg: float) -> tuple[float, float, float]:
    mu, lam, al = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _L().orc_material(E, nu, phi_deg, ctypes.byref(mu), ctypes.byref(lam), ctypes.byref(al))
    return mu.value, lam.value, al.value


def constitutive(Ft, mu, lam, alpha, sigma_min=1e-4):
    Ft = _arr(Ft, (3, 3))
    Fn, tau, info = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros(4)
    _L().orc_constitutive(_d(Ft), mu, lam, alpha, sigma_min, _d(Fn), _d(tau), _d(info))
    return Fn, tau, info


def constitutive_adjoint(Ft, mu, lam, alpha, gFn, gtau, sigma_min=1e-4):
    Ft, gFn, gtau = _arr(Ft, (3, 3)), _arr(gFn, (3, 3)), _arr(gtau, (3, 3))
    gFt = np.zeros((3, 3))
    g = np.zeros(3)
    gp = [ctypes.cast(g.ctypes.data + 8 * i, _dp) for i in range(3)]
    _L().orc_constitutive_adjoint(_d(Ft), mu, lam, alpha, sigma_min, _d(gFn), _d(gtau), _d(gFt), *gp)
    return gFt, float(g[0]), float(g[1]), float(g[2])


def shovel_project(p: Params, vel, q, pose) -> np.ndarray:
    vel, q, pose = _arr(vel, (3,)), _arr(q, (3,)), _arr(pose, (8,))
    out = np.zeros(3)
    pc = p.c()
    _L().orc_shovel_project(ctypes.byref(pc), _d(vel), _d(q), _d(pose), _d(out))
    return out


def rollout(p: Params, x, v, C, F, poses) -> tuple[int, dict]:
    """Run len(poses) substeps from (x, v, C, F); returns (status, state)."""
    x = _arr(x); n = x.shape[0]
    x = x.reshape(n, 3)
    v, C, F = _arr(v, (n, 3)), _arr(C, (n, 9)), _arr(F, (n, 9))
    poses = _arr(poses).reshape(-1, 8)
    pc = p.c()
    st = _L().orc_rollout(ctypes.byref(pc), n, _d(x), _d(v), _d(C), _d(F), poses.shape[0], _d(poses))
    return st, {"x": x, "v": v, "C": C.reshape(n, 3, 3), "F": F.reshape(n, 3, 3)}


def grid_of_substep(p: Params, x, v, C, F, pose):
    x = _arr(x); n = x.shape[0]
    v, C, F = _arr(v, (n, 3)), _arr(C, (n, 9)), _arr(F, (n, 9))
    pose = _arr(pose, (8,))
    G = int(np.prod(p.res))
    m, mv, vo = np.zeros(G), np.zeros((G, 3)), np.zeros((G, 3))
    pc = p.c()
    st = _L().orc_grid_of_substep(ctypes.byref(pc), n, _d(x), _d(v), _d(C), _d(F), _d(pose), _d(m), _d(mv),
                                  _d(vo))
    shp = tuple(int(r) for r in p.res)
    return st, m.reshape(shp), mv.reshape(shp + (3,)), vo.reshape(shp + (3,))


def rollout_adjoint(p: Params, x0, v0, C0, F0, poses, gx=None, gv=None, gC=None, gF=None) -> tuple[int, dict]:
    x0 = _arr(x0); n = x0.shape[0]
    x0 = x0.reshape(n, 3)
    v0, C0, F0 = _arr(v0, (n, 3)), _arr(C0, (n, 9)), _arr(F0, (n, 9))
    poses = _arr(poses).reshape(-1, 8)
    nsub = poses.shape[0]
    gx, gv, gC, gF = _opt(gx, n, 3), _opt(gv, n, 3), _opt(gC, n, 9), _opt(gF, n, 9)
    ax, av, aC, aF = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 9)), np.zeros((n, 9))
    gmat, gposes = np.zeros(4), np.zeros((max(nsub, 1), 8))
    pc = p.c()
    st = _L().orc_rollout_adjoint(ctypes.byref(pc), n, _d(x0), _d(v0), _d(C0), _d(F0), nsub, _d(poses),
                                  _ptr(gx), _ptr(gv), _ptr(gC), _ptr(gF), _d(ax), _d(av), _d(aC), _d(aF),
                                  _d(gmat), _d(gposes))
    return st, {"x": ax, "v": av, "C": aC.reshape(n, 3, 3), "F": aF.reshape(n, 3, 3),
                "material": gmat, "poses": gposes[:nsub]}


def skill_actions(theta, v_lin: float, v_ang: float, dt_step: float, max_actions: int = 100000,
                  unrounded: bool = False):
    """Algorithm 2 -> (actions[T,6], T[4], jac[T,6,6]); unrounded: phases 1
    and 4 divide by the real-valued step counts (Sec. III-B alternative)."""
    th = _arr(theta, (6,))
    acts = np.zeros((max_actions, 6))
    jac = np.zeros((max_actions, 6, 6))
    T = (ctypes.c_int * 4)()
    n = _L().orc_skill_actions(_d(th), v_lin, v_ang, dt_step, max_actions, int(bool(unrounded)), _d(acts),
                               ctypes.cast(T, _ip), _d(jac))
    if n < 0:
        raise ValueError("max_actions too small")
    return acts[:n].copy(), np.array(T[:]), jac[:n].copy()


def pose_table(start, actions, substeps_per_action: int, dt_sub: float, nsub: int) -> np.ndarray:
    start = _arr(start, (4,))
    actions = _arr(actions).reshape(-1, 6)
    out = np.zeros((nsub, 8))
    _L().orc_pose_table(_d(start), actions.shape[0], _d(actions), substeps_per_action, dt_sub, nsub, _d(out))
    return out


def pose_table_adjoint(n_actions: int, substeps_per_action: int, dt_sub: float, gposes) -> np.ndarray:
    gposes = _arr(gposes).reshape(-1, 8)
    out = np.zeros((max(n_actions, 1), 6))
    _L().orc_pose_table_adjoint(n_actions, substeps_per_action, dt_sub, gposes.shape[0], _d(gposes), _d(out))
    return out[:n_actions]


def set_threads(n: int) -> None:
    """Threads of the oracle's particle and node loops (1: the plain serial
    loops; more: OpenMP with per-thread grids, sums in thread order)."""
    _L().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_L().orc_get_threads())


def mse_loss(x, target) -> tuple[float, np.ndarray]:
    """L = (1/N) sum_p |x_p - xhat_p|^2 and dL/dx = 2 (x - xhat) / N."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    t = np.asarray(target, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    d = x - t
    return float((d * d).sum() / n), 2.0 * d / n


def _f32pts(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, 3))
    return x, x.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def surface_observation(g: ObsGrid, x) -> tuple[int, np.ndarray]:
    """(non-empty pixels, per-pixel index of the highest particle or -1)."""
    x, xp = _f32pts(x)
    idx = np.empty(g.res * g.res, np.int64)
    gc = g.c()
    cnt = _L().orc_surface_observation(ctypes.byref(gc), x.shape[0], xp,
                                       idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return int(cnt), idx


def height_map(g: ObsGrid, x) -> tuple[np.ndarray, np.ndarray]:
    """(height map [res, res], winner particle per pixel or -1)."""
    x, xp = _f32pts(x)
    I = np.empty(g.res * g.res, np.float64)
    w = np.empty(g.res * g.res, np.int64)
    gc = g.c()
    _L().orc_height_map(ctypes.byref(gc), x.shape[0], xp, _d(I), w.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return I.reshape(g.res, g.res), w.reshape(g.res, g.res)


def hmd(g: ObsGrid, x, Ihat) -> tuple[float, np.ndarray]:
    """(d_HMD, dL/dx [n, 3])."""
    x, xp = _f32pts(x)
    Ih = np.ascontiguousarray(np.asarray(Ihat, np.float64).reshape(-1))
    assert Ih.size == g.res * g.res
    grad = np.empty((x.shape[0], 3), np.float64)
    gc = g.c()
    L = _L().orc_hmd(ctypes.byref(gc), x.shape[0], xp, _d(Ih), _d(grad))
    return float(L), grad


def grad_op(p: Params, g) -> np.ndarray:
    """Sec. III-E regulariser (clip / dynamic scaling / normalisation) of one vector."""
    g = np.ascontiguousarray(np.asarray(g, np.float64).reshape(-1)).copy()
    pc = p.c()
    _L().orc_grad_op(ctypes.byref(pc), _d(g), g.size)
    return g


def emd(X, Xhat) -> tuple[float, np.ndarray, np.ndarray]:
    """Unnormalised Earth Mover's distance of Eq. (1) (Sec. III-A, "Goal and
    reward/loss"): the least total Euclidean distance over one-to-one maps
    phi of the points X into Xhat (|X| <= |Xhat|), found by linear
    assignment. Returns (d_EMD, phi as indices into Xhat, dd/dX): with phi
    fixed, dd/dx = (x - phi(x)) / |x - phi(x)| (0 where they coincide)."""
    from scipy.optimize import linear_sum_assignment
    X = np.asarray(X, np.float64).reshape(-1, 3)
    Y = np.asarray(Xhat, np.float64).reshape(-1, 3)
    assert X.shape[0] <= Y.shape[0]
    D = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    rows, cols = linear_sum_assignment(D)
    phi = np.empty(X.shape[0], np.int64)
    phi[rows] = cols
    diff = X - Y[phi]
    dist = np.sqrt((diff * diff).sum(1))
    grad = np.where(dist[:, None] > 0, diff / np.where(dist > 0, dist, 1.0)[:, None], 0.0)
    return float(dist.sum()), phi, grad
