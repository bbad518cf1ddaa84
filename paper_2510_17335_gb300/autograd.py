"""torch.autograd.Function over the C ABI.

``rollout(sim, materials, thetas, n_substeps, skills)`` sets each instance's
material (E, nu, rho, phi_deg) and digging skill theta, runs a recorded
forward of ``n_substeps`` from the handle's creation state, and returns the
final particle positions as a CUDA tensor [N, 3] (external order). Its
backward calls ``mpm_backward`` with the incoming dL/dx and returns
dL/d(materials) [n_inst, 4] and dL/d(thetas) [n_inst, 6]. All arithmetic runs
in the library's kernels; this module only moves pointers.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import torch

from . import mpm


@dataclass
class SkillSetup:
    """Fixed (non-differentiated) part of an instance's skill."""
    v_lin: float
    v_ang: float
    substeps_per_action: int
    start_pose: Sequence[float]


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, materials, thetas, sim, n_substeps, skills):
        mats = materials.detach().double().cpu().numpy()
        ths = thetas.detach().double().cpu().numpy()
        for i in range(sim.n_inst):
            sim.set_material(i, mats[i])
            s = skills[i]
            sim.set_skill(i, ths[i], s.v_lin, s.v_ang, s.substeps_per_action, s.start_pose)
        sim.reset()
        sim.set_stream(torch.cuda.current_stream().cuda_stream)
        sim.forward(int(n_substeps), record=True)
        x = torch.empty((sim.n, 3), device="cuda", dtype=torch.float32)
        sim.get_state(device_out={"x": x})
        ctx.sim = sim
        ctx.mat = (materials.device, materials.dtype)
        ctx.th = (thetas.device, thetas.dtype)
        return x

    @staticmethod
    def backward(ctx, gx):
        gm, gt = ctx.sim.backward(dL_dx=gx.contiguous().float())
        # the FP64 sums of the library, in each input's device and dtype
        gmt = torch.from_numpy(gm).to(device=ctx.mat[0], dtype=ctx.mat[1])
        gtt = torch.from_numpy(gt).to(device=ctx.th[0], dtype=ctx.th[1])
        return gmt, gtt, None, None, None


def rollout(sim: "mpm.Simulation", materials: torch.Tensor, thetas: torch.Tensor, n_substeps: int,
            skills: Sequence[SkillSetup]) -> torch.Tensor:
    """Differentiable rollout; see the module docstring."""
    return _Rollout.apply(materials, thetas, sim, n_substeps, skills)
