"""Shared test helpers: run a workload through the FP64 oracle and through
the CUDA library on the same seeded FP32 inputs."""
import numpy as np

import oracle


def oracle_params(w, particle_collision=1, shovel_on=1, clip=0, gravity=None, grad_scale=0):
    return oracle.Params(res=tuple(w.res), dx=w.dx, dt=w.dt, gravity=tuple(w.gravity if gravity is None else gravity),
                         bound=w.bound, E=w.E, nu=w.nu, rho=w.rho, phi_deg=w.phi_deg, vol=w.vol, friction=w.friction,
                         particle_collision=particle_collision, shovel_half=tuple(w.shovel_half), shovel_on=shovel_on,
                         clip_grads=clip, grad_scale=grad_scale)


def oracle_actions(w):
    t = w.traj
    if t.theta is not None:
        acts, T, jac = oracle.skill_actions(t.theta, t.v_lin, t.v_ang, t.substeps_per_action * w.dt,
                                            unrounded=t.unrounded)
        return acts, jac
    return np.asarray(t.actions, np.float64), None


def oracle_poses(w, nsub):
    acts, _ = oracle_actions(w)
    return oracle.pose_table(w.traj.start_pose, acts, w.traj.substeps_per_action, w.dt, nsub)


def initial_state(x0):
    n = x0.shape[0]
    return (np.asarray(x0, np.float64), np.zeros((n, 3)), np.zeros((n, 9)), np.tile(np.eye(3).ravel(), (n, 1)))


def oracle_rollout(w, nsub, **kw):
    p = oracle_params(w, **kw)
    x, v, C, F = initial_state(w.x0)
    status, s = oracle.rollout(p, x, v, C, F, oracle_poses(w, nsub))
    assert status == 0, status
    return s


def rel_err(a, b, floor_frac=1e-3):
    """Per-component |a - b| / max(|b|, floor_frac * max|b|)."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    floor = floor_frac * max(np.abs(b).max(), 1e-300)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)
