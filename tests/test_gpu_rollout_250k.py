"""The differentiable-rollout workload at its full size: 250,000 particles on
a 96^3 grid, the digging skill, checkpoints every 50 substeps, the MSE of the
final positions against a target cloud made with the hidden material, and
the gradient with respect to (E, nu, rho, phi) at a start material 20% off,
against central finite differences of the same FP32 simulation with a
relative step of 1e-4, within 5% plus the differences' own noise (the
spread of repeated evaluations over the step). (The FP64 oracle is far too
slow at this size; it is pinned to finite differences on small inputs.)"""
import numpy as np
import pytest

from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NSUB = 400      # 0.02 s: the shovel descends into the bed
BAR = 5e-2      # FP32 central differences of a 250k-particle, 400-substep loss


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    mpm.lib()


def test_material_gradient_against_central_differences_at_250k():
    w = W.cfg_250k()
    truth = (w.E, w.nu, w.rho, w.phi_deg)
    start = np.array(w.extra["start_material"], np.float64)
    opts = mpm.make_options(checkpoint_every=w.extra["checkpoint_every"])
    with mpm.simulation_from_workloads([w], opts) as sim:
        sim.set_material(0, truth)
        sim.forward(NSUB)
        target = sim.get_state()["x"]

        def loss(m):
            sim.reset()
            sim.set_material(0, m)
            sim.forward(NSUB)
            L, _ = sim.loss_mse(target, want_grad=False)
            return float(L[0])

        sim.reset()
        sim.set_material(0, start)
        sim.forward(NSUB, record=True)
        L0, g = sim.loss_mse(target)
        gm, _ = sim.backward(dL_dx=g)
        fd, h = np.zeros(4), 1e-4 * start
        for k in range(4):
            mp, mm = start.copy(), start.copy()
            mp[k] += h[k]
            mm[k] -= h[k]
            fd[k] = (loss(mp) - loss(mm)) / (2 * h[k])
        # the float atomics make repeated evaluations differ slightly: that
        # spread, divided by the step, bounds the differences' own error
        reps = [loss(start) for _ in range(4)]
        spread = max(reps) - min(reps)
    assert np.isclose(np.mean(reps), L0[0], rtol=1e-6)
    noise = spread / h
    print("loss", L0[0], "spread", spread, "adjoint", gm[0], "central FD", fd, "FD noise", noise)
    assert L0[0] > 0 and np.abs(fd).max() > 0
    assert np.all(np.abs(gm[0] - fd) <= BAR * np.abs(fd) + noise), (gm[0], fd, noise)
    # the check has teeth: for E, nu and rho the differences stand well above their noise
    assert all(noise[k] < 0.1 * abs(fd[k]) for k in (0, 1, 2)), (fd, noise)
    # the scale invariance of E and rho holds for the adjoint at this size too
    assert abs(start[0] * gm[0, 0] + start[2] * gm[0, 2]) <= 1e-4 * abs(start[0] * gm[0, 0])
