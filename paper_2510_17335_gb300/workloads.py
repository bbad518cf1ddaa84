"""Seeded synthetic workloads for the MLS-MPM sand substep.

This module holds the input recipes only: particle beds, material points,
shovel geometry and trajectory specifications. It contains none of the
method's arithmetic (no constitutive model, no transfer, no skill mapping), so
both the FP64 oracle tests and the CUDA path may draw their inputs from it.

Every bed is a lattice at spacing dx/2 (eight particles per cell) with uniform
jitter, drawn with ``numpy.random.default_rng(seed)`` in FP64 and rounded to
FP32; both sides read the same FP32 arrays. Beds rest on the floor at
y = bound*dx and are centred in x and z. The paper fills its container with a
fixed particle density (Sec. III-A, initial state: 0.28 x 0.28 x 0.07 m at
5e6 particles per m^3); ``paper_bed`` reproduces that recipe.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 2510173350


@dataclass
class Trajectory:
    """Shovel motion: either skill parameters (mapped by Algorithm 2 inside
    the library) or a scripted list of per-step displacements."""
    start_pose: Sequence[float]              # tip x, y, z and tilt psi
    substeps_per_action: int
    theta: Optional[Sequence[float]] = None  # 6 skill parameters
    v_lin: float = 0.0
    v_ang: float = 0.0
    actions: Optional[np.ndarray] = None     # scripted: [T, 6] in the simulator frame
    unrounded: bool = False                  # skill: phases 1 and 4 by real-valued step counts


@dataclass
class Workload:
    name: str
    res: Sequence[int]
    dx: float
    dt: float
    n_substeps: int
    E: float
    nu: float
    rho: float
    phi_deg: float
    vol: float
    x0: np.ndarray                           # [N, 3] float32
    traj: Trajectory
    shovel_half: Sequence[float] = (0.01, 0.075, 0.1)
    bound: int = 3
    gravity: Sequence[float] = (0.0, -9.8, 0.0)
    friction: float = 0.5
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x0.shape[0])


def lattice_bed(seed: int, cells: Sequence[int], origin: Sequence[float], dx: float,
                per_axis: int = 2, jitter: float = 0.25) -> np.ndarray:
    """Particles on a lattice of spacing dx/per_axis filling `cells`, jittered
    uniformly by +-jitter*spacing per axis; FP64 draw rounded to FP32."""
    rng = np.random.default_rng(seed)
    h = dx / per_axis
    nx, ny, nz = (int(c) * per_axis for c in cells)
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    p = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    p = (p + 0.5) * h + np.asarray(origin, dtype=np.float64)
    p += rng.uniform(-jitter * h, jitter * h, size=p.shape)
    return p.astype(np.float32)


def paper_bed(seed: int = SEED_BASE, density: float = 5e6, size=(0.28, 0.07, 0.28),
              origin=(0.0, 0.0, 0.0)) -> tuple[np.ndarray, float]:
    """The paper's initial body: a box filled with particles at a fixed number
    density (Sec. III-A), count = box volume x density, positions uniform in
    the box. Returns positions (y up) and the per-particle volume (box volume
    over the count)."""
    box = float(np.prod(size))
    n = int(round(box * density))
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(size) + np.asarray(origin)
    return p.astype(np.float32), box / n


def _centred_bed(seed, res, dx, cells, bound=3):
    R = res[0]
    ox = 0.5 * (R * dx - cells[0] * dx)
    oz = 0.5 * (res[2] * dx - cells[2] * dx)
    oy = bound * dx
    return lattice_bed(seed, cells, (ox, oy, oz), dx), (ox, oy, oz)


def insert_push_actions(n_actions_each: int, depth: float, push: float) -> np.ndarray:
    """Scripted straight insertion (down y) then push (+x)."""
    a = np.zeros((2 * n_actions_each, 6))
    a[:n_actions_each, 1] = -depth / n_actions_each
    a[n_actions_each:, 0] = push / n_actions_each
    return a


def sysid_actions(scale: float, steps_per_segment: int) -> np.ndarray:
    """The paper's optimisation trajectory for system identification
    (Sec. IV-B): +0.09 m in x, -0.05 m insert (down), -0.12 m in x, +0.12 m
    lift, scaled by `scale` and split evenly over `steps_per_segment` global
    steps per segment. Simulator frame: y is up."""
    segs = [(0, 0.09), (1, -0.05), (0, -0.12), (1, 0.12)]
    a = np.zeros((4 * steps_per_segment, 6))
    for s, (ax, d) in enumerate(segs):
        a[s * steps_per_segment:(s + 1) * steps_per_segment, ax] = scale * d / steps_per_segment
    return a


DEMO_THETA = (0.5, 0.2, 0.8, 0.0, -0.5, 1.0)   # Sec. III-C demonstration constants + lift


def cfg_small(seed: int = SEED_BASE + 1) -> Workload:
    """8,000 particles (20^3 lattice at dx/2), 32^3 grid, dt 1e-4, 200
    substeps, E 1e5, nu 0.3, rho 1500, phi 30 deg, box shovel 0.2 x 0.02 x
    0.15 inserted 0.10 m then pushed 0.10 m in x."""
    res, dx = (32, 32, 32), 1.0 / 32
    cells = (10, 10, 10)
    x0, (ox, oy, oz) = _centred_bed(seed, res, dx, cells)
    top = oy + cells[1] * dx
    traj = Trajectory(start_pose=(0.40, top + 0.01, 0.5, 0.0), substeps_per_action=20,
                      actions=insert_push_actions(5, 0.10, 0.10))
    return Workload("bed8k_grid32", res, dx, 1e-4, 200, 1e5, 0.3, 1500.0, 30.0, dx ** 3 / 8, x0, traj)


def cfg_1m(seed: int = SEED_BASE + 2) -> Workload:
    """1,048,576 particles at 8 per cell in a 64 x 32 x 64-cell bed, 128^3
    grid, dt 5e-5, E 3e5, nu 0.25, rho 1800, phi 35 deg, digging skill with
    the demonstration parameters, v_l 2.5 m/s, v_w 25 rad/s, 20 substeps per
    action."""
    res, dx = (128, 128, 128), 1.0 / 128
    cells = (64, 32, 64)
    x0, (ox, oy, oz) = _centred_bed(seed, res, dx, cells)
    top = oy + cells[1] * dx
    traj = Trajectory(start_pose=(ox + 0.25 * cells[0] * dx, top + 0.01, 0.5, 0.0), substeps_per_action=20,
                      theta=DEMO_THETA, v_lin=2.5, v_ang=25.0)
    return Workload("bed1m_grid128", res, dx, 5e-5, 2000, 3e5, 0.25, 1800.0, 35.0, dx ** 3 / 8, x0, traj)


def cfg_250k(seed: int = SEED_BASE + 3) -> Workload:
    """250,000 particles (50 x 25 x 25 cells at 8 per cell), 96^3 grid, dt
    5e-5, 1,000 substeps; ground-truth E 1.5e5, nu 0.3, rho 1600, phi 30 deg;
    skill with 10 substeps per action, v_l 5 m/s, v_w 50 rad/s."""
    res, dx = (96, 96, 96), 1.0 / 96
    cells = (50, 25, 25)
    x0, (ox, oy, oz) = _centred_bed(seed, res, dx, cells)
    top = oy + cells[1] * dx
    traj = Trajectory(start_pose=(ox + 0.25 * cells[0] * dx, top + 0.01, 0.5, 0.0), substeps_per_action=10,
                      theta=DEMO_THETA, v_lin=5.0, v_ang=50.0)
    w = Workload("bed250k_grid96", res, dx, 5e-5, 1000, 1.5e5, 0.3, 1600.0, 30.0, dx ** 3 / 8, x0, traj)
    w.extra["start_material"] = (1.8e5, 0.36, 1920.0, 36.0)
    w.extra["checkpoint_every"] = 50
    return w


def batch_uneven(n_inst: int = 64, seed: int = SEED_BASE + 4, n_lo: float = 2e4, n_hi: float = 2e5,
                 r_lo: int = 64, r_hi: int = 96, n_substeps: int = 500) -> List[Workload]:
    """Uneven instances: particle counts log-uniform in [n_lo, n_hi], beds of
    a x b x a cells with b = round(0.375 a) at 8 per cell, grids log-uniform
    in [r_lo, r_hi] (rounded to a multiple of 4), materials uniform in
    E [5e4, 5e5], nu [0.2, 0.4], phi [25, 40] deg, rho [1200, 2200]; the
    paper's system-identification trajectory scaled to each bed and paced at
    about 0.5 m/s."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n_target = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        R = int(round(np.exp(rng.uniform(np.log(r_lo), np.log(r_hi))) / 4.0)) * 4
        a = max(4, int(round((n_target / 3.0) ** (1.0 / 3.0))))
        b = max(2, int(round(0.375 * a)))
        a = min(a, R - 12)
        b = min(b, R - 16)
        dx = 1.0 / R
        x0, (ox, oy, oz) = _centred_bed(seed * 131 + i, (R, R, R), dx, (a, b, a))
        top = oy + b * dx
        E = rng.uniform(5e4, 5e5)
        nu = rng.uniform(0.2, 0.4)
        phi = rng.uniform(25.0, 40.0)
        rho = rng.uniform(1200.0, 2200.0)
        scale = a * dx / 0.28
        # ~0.5 m/s along the first segment (10 substeps of 5e-5 s per step)
        steps = max(1, int(round(0.09 * scale / (0.5 * 10 * 5e-5))))
        traj = Trajectory(start_pose=(ox + 0.25 * a * dx, top + 0.01, 0.5, 0.0), substeps_per_action=10,
                          actions=sysid_actions(scale, steps))
        out.append(Workload(f"inst{i}_n{x0.shape[0]}_grid{R}", (R, R, R), dx, 5e-5, n_substeps, E, nu, rho, phi,
                            dx ** 3 / 8, x0, traj))
    return out


def cfg_sysid(seed: int = SEED_BASE + 5, n_substeps: int = 1500) -> Workload:
    """The batched system-identification workload's bed: 98,304 particles
    (32 x 12 x 32 cells at 8 per cell) on a 64^3 grid, dt 5e-5; the shovel tip
    starts at the bed surface, a quarter along x, and is scripted to insert
    then push, each by 0.05 m per 1,500 substeps (about 1.3 m/s). Hidden
    material E 1.2e5, nu 0.3, rho 1600, phi 32 deg (inside the ranges of
    Sec. IV-B)."""
    res, dx = (64, 64, 64), 1.0 / 64
    cells = (32, 12, 32)
    x0, (ox, oy, oz) = _centred_bed(seed, res, dx, cells)
    top = oy + cells[1] * dx
    half = max(1, n_substeps // 20)                 # actions of 10 substeps per phase
    d = 0.05 * n_substeps / 1500.0
    traj = Trajectory(start_pose=(ox + 0.25 * cells[0] * dx, top, 0.5, 0.0), substeps_per_action=10,
                      actions=insert_push_actions(half, d, d))
    return Workload(f"sysid_n{x0.shape[0]}_grid64", res, dx, 5e-5, n_substeps, 1.2e5, 0.3, 1600.0, 32.0,
                    dx ** 3 / 8, x0, traj)


def tiny(seed: int, n_side: int = 3, res: int = 12, jitter: float = 0.25) -> np.ndarray:
    """A small cube of n_side^3 particles in the middle of a res^3 grid."""
    dx = 1.0 / res
    c = res // 2 - n_side // 4 - 1
    return lattice_bed(seed, (max(1, n_side // 2),) * 3, (c * dx,) * 3, dx,
                       per_axis=2 if n_side > 1 else 1, jitter=jitter)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def strained_F(rng: np.random.Generator, n: int, log_strain_scale: float = 0.02,
               mean_log_strain: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """Deformation gradients R1 diag(exp(e)) R2 with random rotations and
    log stretches e ~ mean + scale * N(0, 1)."""
    out = np.empty((n, 3, 3))
    for i in range(n):
        e = np.asarray(mean_log_strain) + log_strain_scale * rng.normal(size=3)
        out[i] = random_rotation(rng) @ np.diag(np.exp(e)) @ random_rotation(rng)
    return out
