"""Thin ctypes binding of libmpm_gb300.so (include/mpm.h).

Functions carry the C names and do argument marshalling only: numpy arrays
are passed as host pointers, torch CUDA tensors as device pointers. Every
step of the simulation runs in the library's CUDA kernels; there is no CPU
path. ``lib()`` raises if the library is missing or cannot be loaded.

``Simulation`` is a small convenience owner of one handle (creation from a
list of workloads, state and gradient accessors).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpm_gb300.so")

MPM_OK = 0
PROFILE_KERNELS = 12    # MPM_PROFILE_KERNELS of the header
ERRORS = {
    -1: "MPM_ERR_INVALID_ARG", -2: "MPM_ERR_OOM", -3: "MPM_ERR_CUDA", -4: "MPM_ERR_OUT_OF_DOMAIN",
    -5: "MPM_ERR_NON_FINITE", -6: "MPM_ERR_NO_RECORD", -7: "MPM_ERR_TIMEOUT", -8: "MPM_ERR_NO_DEVICE",
}


class MpmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().mpm_error_string(code).decode() if _lib is not None else ERRORS.get(code, "?")
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


class mpm_material(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("rho", ctypes.c_double),
                ("phi_deg", ctypes.c_double)]


class mpm_config(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int * 3), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("gravity", ctypes.c_double * 3), ("bound", ctypes.c_int), ("particle_volume", ctypes.c_double),
                ("friction", ctypes.c_double), ("particle_collision", ctypes.c_int),
                ("shovel_half", ctypes.c_double * 3), ("shovel_on", ctypes.c_int)]


class mpm_options(ctypes.Structure):
    _fields_ = [("checkpoint_every", ctypes.c_int), ("clip_grads", ctypes.c_int), ("clip_value", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("sort_every", ctypes.c_int), ("tile_scatter", ctypes.c_int),
                ("cuda_graphs", ctypes.c_int), ("grad_scale", ctypes.c_int), ("oom_star", ctypes.c_double),
                ("grad_delta", ctypes.c_double), ("fuse_adjoint", ctypes.c_int)]


class mpm_skill(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double * 6), ("v_lin", ctypes.c_double), ("v_ang", ctypes.c_double),
                ("substeps_per_action", ctypes.c_int), ("start_pose", ctypes.c_double * 4),
                ("unrounded_T", ctypes.c_int)]


class mpm_info_t(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int), ("n_particles", ctypes.c_int64), ("substep", ctypes.c_int64),
                ("recorded", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("fp64_fallbacks", ctypes.c_int64), ("graph_launches", ctypes.c_int64)]


class mpm_obs_grid(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 2), ("size", ctypes.c_double), ("res", ctypes.c_int),
                ("tap", ctypes.c_double)]


def make_obs_grid(center_xz, size: float = 0.24, res: int = 40, tap: float = 0.0) -> mpm_obs_grid:
    """Observation / height-map square (Sec. III-A): res x res pixels of side
    size in the (x, z) plane centred at center_xz; tap is the height-map
    splat offset."""
    g = mpm_obs_grid()
    g.center[0], g.center[1] = float(center_xz[0]), float(center_xz[1])
    g.size, g.res, g.tap = float(size), int(res), float(tap)
    return g


_vp, _dp, _fp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int
_lib = None

EXPORTS = {
    "mpm_create": (_ip, [_ip, ctypes.POINTER(mpm_config), ctypes.POINTER(mpm_material), ctypes.POINTER(ctypes.c_int64),
                         _fp, ctypes.POINTER(mpm_options), ctypes.POINTER(_vp)]),
    "mpm_set_material": (_ip, [_vp, _ip, ctypes.POINTER(mpm_material)]),
    "mpm_set_shovel_actions": (_ip, [_vp, _ip, _dp, _ip, _dp, _ip]),
    "mpm_set_shovel_trajectory": (_ip, [_vp, _ip, ctypes.POINTER(mpm_skill)]),
    "mpm_num_actions": (_ip, [_vp, _ip]),
    "mpm_reset": (_ip, [_vp]),
    "mpm_set_state": (_ip, [_vp, _fp, _fp, _fp, _fp, _ip]),
    "mpm_get_state": (_ip, [_vp, _fp, _fp, _fp, _fp, _ip]),
    "mpm_forward": (_ip, [_vp, _ip, _ip]),
    "mpm_loss_mse": (_ip, [_vp, _fp, _dp, _fp, _ip]),
    "mpm_backward": (_ip, [_vp, _fp, _fp, _ip, _dp, _dp]),
    "mpm_get_state_grad": (_ip, [_vp, _fp, _fp, _fp, _fp, _ip]),
    "mpm_get_action_grad": (_ip, [_vp, _ip, _dp, _dp]),
    "mpm_set_stream": (_ip, [_vp, _vp]),
    "mpm_synchronize": (_ip, [_vp]),
    "mpm_get_info": (_ip, [_vp, ctypes.POINTER(mpm_info_t)]),
    "mpm_grid_mass": (_ip, [_vp, _dp]),
    "mpm_set_substep": (_ip, [_vp, ctypes.c_int64]),
    "mpm_autotune": (_ip, [_vp, _ip, ctypes.POINTER(ctypes.c_int)]),
    "mpm_set_launch_shape": (_ip, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "mpm_record_bytes": (_ip, [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)]),
    "mpm_get_launch_shape": (_ip, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "mpm_profile": (_ip, [_vp, _ip]),
    "mpm_profile_read": (_ip, [_vp, _ip, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "mpm_kernel_name": (ctypes.c_char_p, [_ip]),
    "mpm_loss_mse_noalloc": (_ip, [_fp, _fp, ctypes.c_int64, _fp, _dp, _vp]),
    "mpm_surface_observation": (_ip, [_vp, ctypes.POINTER(mpm_obs_grid), _fp, ctypes.POINTER(ctypes.c_int), _ip]),
    "mpm_height_map": (_ip, [_vp, ctypes.POINTER(mpm_obs_grid), _fp, _ip]),
    "mpm_loss_hmd": (_ip, [_vp, ctypes.POINTER(mpm_obs_grid), _fp, _dp, _fp, _ip]),
    "mpm_loss_emd": (_ip, [_vp, ctypes.POINTER(mpm_obs_grid), _fp, ctypes.POINTER(ctypes.c_int), _dp, _fp, _ip]),
    "mpm_line_search": (_ip, [_vp, _ip, ctypes.POINTER(mpm_material), ctypes.POINTER(mpm_skill), _ip,
                              ctypes.POINTER(mpm_obs_grid), _fp, _ip, _dp, ctypes.POINTER(ctypes.c_int)]),
    "mpm_destroy": (None, [_vp]),
    "mpm_error_string": (ctypes.c_char_p, [_ip]),
    "mpm_version": (_ip, []),
}


def lib():
    """Load libmpm_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2510_17335_gb300.build` "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code: int, where: str) -> None:
    if code != MPM_OK:
        raise MpmError(code, where)


# ---------------------------------------------------------------------------
# pointer marshalling
# ---------------------------------------------------------------------------
def _ptr(a, device: bool):
    """(pointer, keepalive) for a float32 numpy array (host) or torch tensor (device)."""
    if a is None:
        return None, None
    if device:
        import torch
        assert isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr.ctypes.data_as(ctypes.c_void_p), arr


def _is_device(*arrays) -> bool:
    for a in arrays:
        if a is not None and hasattr(a, "is_cuda"):
            return bool(a.is_cuda)
    return False


def loss_mse_noalloc(x, target, dL_dx=None, stream_ptr: int = 0) -> float:
    """mpm_loss_mse_noalloc on device tensors x, target [n, 3] (float32);
    writes dL/dx into dL_dx if given; returns the loss."""
    import torch
    # the C entry point reads and writes n * 3 floats of every array it is
    # given: check the shapes and that all arrays live on one CUDA device
    # before anything is launched
    tensors = [("x", x), ("target", target)] + ([("dL_dx", dL_dx)] if dL_dx is not None else [])
    for name, t in tensors:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"loss_mse_noalloc: {name} must be a torch tensor")
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"loss_mse_noalloc: {name} must be contiguous float32")
    if x.dim() != 2 or x.shape[1] != 3:
        raise ValueError(f"loss_mse_noalloc: x must be [n, 3], got {tuple(x.shape)}")
    for name, t in tensors[1:]:
        if t.shape != x.shape:
            raise ValueError(f"loss_mse_noalloc: {name} has shape {tuple(t.shape)}, x has {tuple(x.shape)}")
    if not all(t.is_cuda for _, t in tensors):
        raise ValueError("loss_mse_noalloc: every array must be a CUDA tensor")
    if len({t.device for _, t in tensors}) != 1:
        raise ValueError("loss_mse_noalloc: every array must be on the same device")
    L = ctypes.c_double()
    with torch.cuda.device(x.device):
        xp, _ = _ptr(x, True)
        tp, _ = _ptr(target, True)
        gp, _ = _ptr(dL_dx, True) if dL_dx is not None else (None, None)
        check(lib().mpm_loss_mse_noalloc(xp, tp, int(x.shape[0]), gp, ctypes.byref(L),
                                         ctypes.c_void_p(stream_ptr)), "mpm_loss_mse_noalloc")
    return L.value


def record_bytes(n_particles: int, n_nodes: int) -> tuple[int, int]:
    """mpm_record_bytes: (bytes of one state slot, bytes of one recorded
    substep's slot) for n_particles particles on n_nodes grid nodes."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    check(lib().mpm_record_bytes(int(n_particles), int(n_nodes), ctypes.byref(a), ctypes.byref(b)),
          "mpm_record_bytes")
    return a.value, b.value


def blocked_nodes(res) -> int:
    """Grid nodes of one instance as the library lays them out (4x4x4 blocks)."""
    return int(np.prod([-(-int(r) // 4) * 4 for r in res]))


def best_interval(n_substeps: int, k_max: int) -> int:
    """The checkpoint interval K <= k_max that recomputes least. The backward
    reverses the last segment from its record and recomputes every earlier
    segment once from its checkpoint, so n_substeps minus the last segment's
    length (S - K (ceil(S / K) - 1)) substeps are recomputed; among the K
    with the longest last segment, the largest."""
    S = int(n_substeps)
    best, best_last = 1, 0
    for K in range(1, int(k_max) + 1):
        last = S - K * (-(-S // K) - 1)
        if last >= best_last:
            best, best_last = K, last
    return best


def checkpoint_interval(n_substeps: int, n_particles: int, n_nodes: int, free_bytes: int,
                        reserve: int | None = None) -> int:
    """The checkpoint interval for a recorded rollout of n_substeps on
    n_particles particles and n_nodes grid nodes (all instances): the K that
    recomputes least (best_interval) among those whose recording fits in
    free_bytes less a reserve: the segment's K + 1 state slots and K substep
    slots (mpm_record_bytes) and one state slot per segment's checkpoint.
    The reserve (default: the larger of 8 GiB and a sixteenth of free_bytes)
    is left for the handle's working buffers and the caller's."""
    S = int(n_substeps)
    state, sub = record_bytes(n_particles, n_nodes)
    if reserve is None:
        reserve = max(8 << 30, int(free_bytes) // 16)
    budget = int(free_bytes) - int(reserve)
    k_max = 1
    for K in range(1, S + 1):
        if (K + 1) * state + K * sub + (-(-S // K)) * state <= budget:
            k_max = K
    return best_interval(S, k_max)


def make_config(res, dx, dt, particle_volume, gravity=(0.0, -9.8, 0.0), bound=3, friction=0.5,
                particle_collision=1, shovel_half=(0.01, 0.075, 0.1), shovel_on=1) -> mpm_config:
    c = mpm_config()
    c.res[:] = [int(r) for r in res]
    c.dx, c.dt = float(dx), float(dt)
    c.gravity[:] = [float(g) for g in gravity]
    c.bound = int(bound)
    c.particle_volume = float(particle_volume)
    c.friction = float(friction)
    c.particle_collision = int(particle_collision)
    c.shovel_half[:] = [float(h) for h in shovel_half]
    c.shovel_on = int(shovel_on)
    return c


def make_skill(theta, v_lin, v_ang, substeps_per_action, start_pose, unrounded_T=False) -> mpm_skill:
    """Skill parameters (Sec. III-B, Algorithm 2); unrounded_T selects the
    alternative mapping that divides phases 1 and 4 by real-valued step counts."""
    s = mpm_skill()
    s.theta[:] = [float(t) for t in theta]
    s.v_lin, s.v_ang, s.substeps_per_action = float(v_lin), float(v_ang), int(substeps_per_action)
    s.start_pose[:] = [float(p) for p in start_pose]
    s.unrounded_T = int(bool(unrounded_T))
    return s


def make_options(checkpoint_every=50, clip_grads=0, clip_value=1e4, sigma_min=1e-4, sort_every=0,
                 tile_scatter=0, cuda_graphs=1, grad_scale=0, oom_star=4.0, grad_delta=1e-6,
                 fuse_adjoint=1) -> mpm_options:
    o = mpm_options()
    o.checkpoint_every, o.clip_grads, o.clip_value = int(checkpoint_every), int(clip_grads), float(clip_value)
    o.sigma_min, o.sort_every, o.tile_scatter = float(sigma_min), int(sort_every), int(tile_scatter)
    o.cuda_graphs = int(cuda_graphs)
    o.grad_scale, o.oom_star, o.grad_delta = int(grad_scale), float(oom_star), float(grad_delta)
    o.fuse_adjoint = int(fuse_adjoint)
    return o


class Simulation:
    """Owner of one mpm_handle (a batch of instances)."""

    def __init__(self, configs: Sequence[mpm_config], materials: Sequence[Sequence[float]],
                 positions: Sequence[np.ndarray], options: Optional[mpm_options] = None):
        L = lib()
        n = len(configs)
        self.n_inst = n
        self.counts = [int(np.asarray(p).reshape(-1, 3).shape[0]) for p in positions]
        self.n = int(sum(self.counts))
        cfg_arr = (mpm_config * n)(*configs)
        mat_arr = (mpm_material * n)(*[mpm_material(*map(float, m)) for m in materials])
        cnt = (ctypes.c_int64 * n)(*self.counts)
        x0 = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float32).reshape(-1, 3) for p in positions])
                                  if self.n else np.zeros((0, 3), np.float32))
        h = ctypes.c_void_p()
        check(L.mpm_create(n, cfg_arr, mat_arr, cnt, x0.ctypes.data_as(ctypes.c_void_p),
                           ctypes.byref(options) if options is not None else None, ctypes.byref(h)), "mpm_create")
        self.h = h
        self.n_actions = [0] * n

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib().mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- setup ------------------------------------------------------------
    def set_stream(self, stream_ptr: int):
        check(lib().mpm_set_stream(self.h, ctypes.c_void_p(stream_ptr)), "mpm_set_stream")

    def set_material(self, inst: int, material: Sequence[float]):
        m = mpm_material(*map(float, material))
        check(lib().mpm_set_material(self.h, inst, ctypes.byref(m)), "mpm_set_material")

    def set_actions(self, inst: int, start_pose, actions, substeps_per_action: int):
        a = np.ascontiguousarray(np.asarray(actions, np.float64).reshape(-1, 6))
        sp = np.ascontiguousarray(np.asarray(start_pose, np.float64).reshape(4))
        check(lib().mpm_set_shovel_actions(self.h, inst, sp.ctypes.data_as(_dp), a.shape[0], a.ctypes.data_as(_dp),
                                           int(substeps_per_action)), "mpm_set_shovel_actions")
        self.n_actions[inst] = a.shape[0]

    def set_skill(self, inst: int, theta, v_lin, v_ang, substeps_per_action, start_pose, unrounded_T=False):
        s = make_skill(theta, v_lin, v_ang, substeps_per_action, start_pose, unrounded_T)
        check(lib().mpm_set_shovel_trajectory(self.h, inst, ctypes.byref(s)), "mpm_set_shovel_trajectory")
        self.n_actions[inst] = lib().mpm_num_actions(self.h, inst)

    # -- simulation -------------------------------------------------------
    def reset(self):
        check(lib().mpm_reset(self.h), "mpm_reset")

    def forward(self, n_substeps: int, record: bool = False):
        check(lib().mpm_forward(self.h, int(n_substeps), int(bool(record))), "mpm_forward")

    def set_state(self, x, v=None, C=None, F=None):
        dev = _is_device(x, v, C, F)
        ps = [_ptr(a, dev) for a in (x, v, C, F)]
        check(lib().mpm_set_state(self.h, *[p for p, _ in ps], int(dev)), "mpm_set_state")

    def get_state(self, device_out: Optional[dict] = None) -> dict:
        """Host numpy copies of x, v, C, F (external order) unless device
        tensors are given in device_out (keys x, v, C, F)."""
        if device_out is not None:
            ps = [_ptr(device_out.get(k), True) for k in ("x", "v", "C", "F")]
            check(lib().mpm_get_state(self.h, *[p for p, _ in ps], 1), "mpm_get_state")
            return device_out
        out = {"x": np.empty((self.n, 3), np.float32), "v": np.empty((self.n, 3), np.float32),
               "C": np.empty((self.n, 3, 3), np.float32), "F": np.empty((self.n, 3, 3), np.float32)}
        check(lib().mpm_get_state(self.h, *[out[k].ctypes.data_as(ctypes.c_void_p) for k in ("x", "v", "C", "F")], 0),
              "mpm_get_state")
        return out

    def loss_mse(self, target, want_grad: bool = True, grad_out=None):
        dev = _is_device(target)
        L = np.zeros(self.n_inst, np.float64)
        tp, tk = _ptr(target, dev)
        if dev:
            gp, gk = _ptr(grad_out, True) if want_grad else (None, None)
            check(lib().mpm_loss_mse(self.h, tp, L.ctypes.data_as(_dp), gp, 1), "mpm_loss_mse")
            return L, grad_out
        g = np.empty((self.n, 3), np.float32) if want_grad else None
        check(lib().mpm_loss_mse(self.h, tp, L.ctypes.data_as(_dp),
                                 g.ctypes.data_as(ctypes.c_void_p) if g is not None else None, 0), "mpm_loss_mse")
        return L, g

    def backward(self, dL_dx=None, dL_dv=None):
        dev = _is_device(dL_dx, dL_dv)
        gx, kx = _ptr(dL_dx, dev)
        gv, kv = _ptr(dL_dv, dev)
        gm = np.zeros((self.n_inst, 4), np.float64)
        gt = np.zeros((self.n_inst, 6), np.float64)
        check(lib().mpm_backward(self.h, gx, gv, int(dev), gm.ctypes.data_as(_dp), gt.ctypes.data_as(_dp)),
              "mpm_backward")
        return gm, gt

    def state_grad(self) -> dict:
        out = {"x": np.empty((self.n, 3), np.float32), "v": np.empty((self.n, 3), np.float32),
               "C": np.empty((self.n, 3, 3), np.float32), "F": np.empty((self.n, 3, 3), np.float32)}
        check(lib().mpm_get_state_grad(self.h, *[out[k].ctypes.data_as(ctypes.c_void_p) for k in ("x", "v", "C", "F")],
                                       0), "mpm_get_state_grad")
        return out

    def action_grad(self, inst: int):
        na = lib().mpm_num_actions(self.h, inst)
        ga = np.zeros((max(na, 1), 6), np.float64)
        gs = np.zeros(4, np.float64)
        check(lib().mpm_get_action_grad(self.h, inst, ga.ctypes.data_as(_dp), gs.ctypes.data_as(_dp)),
              "mpm_get_action_grad")
        return ga[:na], gs

    def synchronize(self):
        check(lib().mpm_synchronize(self.h), "mpm_synchronize")

    def autotune(self, trial_substeps: int = 20) -> dict:
        """mpm_autotune: the chosen sort interval and register caps."""
        c = (ctypes.c_int * 2)()
        check(lib().mpm_autotune(self.h, int(trial_substeps), c), "mpm_autotune")
        return {"tile_scatter": c[0], "sort_every": c[1], "launch_shape": self.launch_shape()}

    def launch_shape(self) -> dict:
        """Register caps (minimum resident CTAs per SM) of k_p2g, k_g2p and the fused adjoint."""
        c = (ctypes.c_int * 3)()
        check(lib().mpm_get_launch_shape(self.h, c), "mpm_get_launch_shape")
        return {"p2g": c[0], "g2p": c[1], "fused": c[2]}

    def set_launch_shape(self, p2g: int, g2p: int, fused: int):
        c = (ctypes.c_int * 3)(int(p2g), int(g2p), int(fused))
        check(lib().mpm_set_launch_shape(self.h, c), "mpm_set_launch_shape")

    def set_substep(self, s: int):
        check(lib().mpm_set_substep(self.h, int(s)), "mpm_set_substep")

    def profile(self, enable: bool):
        check(lib().mpm_profile(self.h, int(bool(enable))), "mpm_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total device ms, launches)} for every kernel."""
        out = {}
        for k in range(PROFILE_KERNELS):
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            check(lib().mpm_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)), "mpm_profile_read")
            out[lib().mpm_kernel_name(k).decode()] = (ms.value, n.value)
        return out

    def grid_mass(self) -> np.ndarray:
        out = np.zeros(self.n_inst, np.float64)
        check(lib().mpm_grid_mass(self.h, out.ctypes.data_as(_dp)), "mpm_grid_mass")
        return out

    def _grids(self, grids):
        if isinstance(grids, mpm_obs_grid):
            grids = [grids] * self.n_inst
        assert len(grids) == self.n_inst
        return (mpm_obs_grid * self.n_inst)(*grids)

    def surface_observation(self, grids):
        """(points [n_inst, res*res, 3] with NaN for empty pixels, counts [n_inst])."""
        ga = self._grids(grids)
        npix = ga[0].res * ga[0].res
        pts = np.empty((self.n_inst, npix, 3), np.float32)
        cnt = (ctypes.c_int * self.n_inst)()
        check(lib().mpm_surface_observation(self.h, ga, pts.ctypes.data_as(ctypes.c_void_p), cnt, 0),
              "mpm_surface_observation")
        return pts, np.array(cnt[:], np.int64)

    def height_map(self, grids) -> np.ndarray:
        """[n_inst, res, res] height maps."""
        ga = self._grids(grids)
        res = ga[0].res
        out = np.empty((self.n_inst, res, res), np.float32)
        check(lib().mpm_height_map(self.h, ga, out.ctypes.data_as(ctypes.c_void_p), 0), "mpm_height_map")
        return out

    def loss_hmd(self, grids, target_maps, want_grad: bool = True):
        """(loss [n_inst] (FP64), dL/dx [n, 3] or None)."""
        ga = self._grids(grids)
        tm = np.ascontiguousarray(target_maps, np.float32)
        assert tm.size == self.n_inst * ga[0].res * ga[0].res
        L = np.zeros(self.n_inst, np.float64)
        g = np.empty((self.n, 3), np.float32) if want_grad else None
        check(lib().mpm_loss_hmd(self.h, ga, tm.ctypes.data_as(ctypes.c_void_p), L.ctypes.data_as(_dp),
                                 g.ctypes.data_as(ctypes.c_void_p) if g is not None else None, 0), "mpm_loss_hmd")
        return L, g

    def loss_emd(self, grids, targets, want_grad: bool = True):
        """Earth Mover's distance of the observation to target clouds (Eq. (1)):
        targets is a list of [m_i, 3] arrays (m_i <= res^2). Returns (loss [n_inst]
        (FP64), dL/dx [n, 3] or None)."""
        ga = self._grids(grids)
        npix = ga[0].res * ga[0].res
        tg = np.full((self.n_inst, npix, 3), np.nan, np.float32)
        nt = (ctypes.c_int * self.n_inst)()
        for i, t in enumerate(targets):
            t = np.asarray(t, np.float32).reshape(-1, 3)
            assert t.shape[0] <= npix
            tg[i, :t.shape[0]] = t
            nt[i] = t.shape[0]
        L = np.zeros(self.n_inst, np.float64)
        g = np.empty((self.n, 3), np.float32) if want_grad else None
        check(lib().mpm_loss_emd(self.h, ga, tg.ctypes.data_as(ctypes.c_void_p), nt, L.ctypes.data_as(_dp),
                                 g.ctypes.data_as(ctypes.c_void_p) if g is not None else None, 0), "mpm_loss_emd")
        return L, g

    def line_search(self, n_substeps: int, grids, target_maps, materials=None, skills=None):
        """Batched line search (Sec. III-F): candidate k runs as instance k
        with materials[k] / skills[k]; returns (best k, losses)."""
        n_cand = len(materials) if materials is not None else len(skills)
        ga = self._grids(grids)
        tm = np.ascontiguousarray(target_maps, np.float32)
        mats = (mpm_material * n_cand)(*[mpm_material(*map(float, m)) for m in materials]) if materials else None
        sk = (mpm_skill * n_cand)(*skills) if skills else None
        L = np.zeros(n_cand, np.float64)
        best = ctypes.c_int()
        check(lib().mpm_line_search(self.h, n_cand, mats, sk, int(n_substeps), ga, tm.ctypes.data_as(ctypes.c_void_p),
                                    0, L.ctypes.data_as(_dp), ctypes.byref(best)), "mpm_line_search")
        return int(best.value), L

    def info(self) -> dict:
        i = mpm_info_t()
        check(lib().mpm_get_info(self.h, ctypes.byref(i)), "mpm_get_info")
        return {k: getattr(i, k) for k, _ in mpm_info_t._fields_}


def simulation_from_workloads(workloads, options: Optional[mpm_options] = None, particle_collision: int = 1,
                              shovel_on: int = 1, gravity=None) -> Simulation:
    """One handle holding every workload of the list as an instance, with
    its material and trajectory set."""
    cfgs, mats, xs = [], [], []
    for w in workloads:
        cfgs.append(make_config(w.res, w.dx, w.dt, w.vol, gravity=w.gravity if gravity is None else gravity,
                                bound=w.bound, friction=w.friction, particle_collision=particle_collision,
                                shovel_half=w.shovel_half, shovel_on=shovel_on))
        mats.append((w.E, w.nu, w.rho, w.phi_deg))
        xs.append(w.x0)
    sim = Simulation(cfgs, mats, xs, options)
    for i, w in enumerate(workloads):
        t = w.traj
        if t.theta is not None:
            sim.set_skill(i, t.theta, t.v_lin, t.v_ang, t.substeps_per_action, t.start_pose,
                          unrounded_T=getattr(t, "unrounded", False))
        elif t.actions is not None:
            sim.set_actions(i, t.start_pose, t.actions, t.substeps_per_action)
    return sim
