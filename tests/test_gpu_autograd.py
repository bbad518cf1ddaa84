"""The torch.autograd.Function over the C ABI (paper_2510_17335_gb300.autograd):
a torch loss of the rollout's final positions gets, through rollout(), the
material and skill-parameter gradients of the oracle's FP64 adjoint, for two
batched instances with their own materials, in the dtype of its inputs."""
import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

from _common import initial_state, oracle_actions, oracle_params, oracle_poses, rel_err

pytestmark = pytest.mark.gpu
BAR = 2e-2   # gradient bar of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    mpm.lib()


def _skill_bed(material):
    """A 3,200-particle bed dug by the skill (the bed of the library's own
    theta-gradient test) with the given material."""
    res, dx = 32, 1.0 / 32
    x0 = W.lattice_bed(31, (10, 5, 8), (11 * dx, 3 * dx, 12 * dx), dx)
    top = 8 * dx
    traj = W.Trajectory((13.5 * dx, top - 0.005, 16 * dx, 0.0), 4, theta=(0.4, 0.3, 0.55, 0.2, -0.2, 0.5),
                        v_lin=25.0, v_ang=250.0)
    E, nu, rho, phi = material
    return W.Workload("skill", (res,) * 3, dx, 1e-4, 40, E, nu, rho, phi, dx ** 3 / 8, x0, traj,
                      shovel_half=(0.02, 0.06, 0.1))


def _oracle(w, nsub, gx):
    p = oracle_params(w)
    st, g = oracle.rollout_adjoint(p, *initial_state(w.x0), oracle_poses(w, nsub), gx=gx)
    assert st == 0
    acts, jac = oracle_actions(w)
    ga = oracle.pose_table_adjoint(acts.shape[0], w.traj.substeps_per_action, w.dt, g["poses"])
    return g["material"], np.einsum("tk,tkj->j", ga, jac)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_rollout_gradient_through_torch_matches_the_oracle(dtype):
    import torch

    from paper_2510_17335_gb300 import autograd

    dt = getattr(torch, dtype)
    ws = [_skill_bed((1e5, 0.3, 1500.0, 30.0)), _skill_bed((1.3e5, 0.28, 1600.0, 33.0))]
    nsub = 40
    skills = [autograd.SkillSetup(w.traj.v_lin, w.traj.v_ang, w.traj.substeps_per_action, w.traj.start_pose)
              for w in ws]
    mats = torch.tensor([[w.E, w.nu, w.rho, w.phi_deg] for w in ws], dtype=dt, device="cuda", requires_grad=True)
    ths = torch.tensor([list(w.traj.theta) for w in ws], dtype=dt, device="cuda", requires_grad=True)
    # a coherent loss direction, like the MSE gradient of a shifted target
    rng = np.random.default_rng(7)
    n = ws[0].n
    seed = np.concatenate([(np.array([1.0, -0.5, 0.3]) + 0.1 * rng.normal(size=(n, 3))) / n for _ in ws])
    with mpm.simulation_from_workloads(ws, mpm.make_options(checkpoint_every=10)) as sim:
        x = autograd.rollout(sim, mats, ths, nsub, skills)
        assert x.shape == (2 * n, 3) and x.is_cuda
        s = torch.from_numpy(seed.astype(np.float32)).cuda()
        loss = 3.0 * (x * s).sum()            # dL/dx = 3 seed
        loss.backward()
    assert mats.grad.dtype == dt and ths.grad.dtype == dt
    for i, w in enumerate(ws):
        gm_ref, gt_ref = _oracle(w, nsub, 3.0 * seed[i * n:(i + 1) * n])
        gm, gt = mats.grad[i].double().cpu().numpy(), ths.grad[i].double().cpu().numpy()
        print(f"instance {i}: material {gm} oracle {gm_ref}; theta {gt} oracle {gt_ref}")
        assert rel_err(gm, gm_ref).max() < BAR
        assert rel_err(gt, gt_ref).max() < BAR
