"""The allocation-free MSE entry point (mpm_loss_mse_noalloc) against the
handle-based mpm_loss_mse, through the C ABI, on two calls in a row.

The entry point exists for callers that cannot allocate device memory
(their GPU memory is owned by another allocator, or an allocation's implicit
synchronisation is not allowed where they run); its scratch is a fixed
device array inside the library. The loss is accumulated in FP64 on both
sides in a different order: tolerance 1e-12 relative; dL/dx is the same
FP32 expression on both sides: bit-equal."""
import numpy as np
import pytest

from paper_2510_17335_gb300 import mpm
from paper_2510_17335_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_loss_matches_handle_loss_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_17335_gb300 import build
    build.build()
    w = W.cfg_small()
    n = w.n
    with mpm.simulation_from_workloads([w]) as sim:
        for call in range(2):
            sim.forward(5)
            x = torch.empty((n, 3), device="cuda", dtype=torch.float32)
            sim.get_state(device_out={"x": x})
            torch.cuda.synchronize()
            shift = torch.tensor([0.003, -0.002, 0.001 * (call + 1)], device="cuda")
            target = (torch.from_numpy(w.x0).cuda() + shift).contiguous()
            g_ref = torch.empty((n, 3), device="cuda", dtype=torch.float32)
            L_ref, _ = sim.loss_mse(target, grad_out=g_ref)
            g = torch.full((n, 3), float("nan"), device="cuda", dtype=torch.float32)
            L = mpm.loss_mse_noalloc(x, target, g)
            torch.cuda.synchronize()
            assert np.isclose(L, L_ref[0], rtol=1e-12, atol=0), (call, L, L_ref[0])
            assert torch.equal(g, g_ref), call
    # sizes beyond the stated maximum are rejected before anything runs
    import ctypes
    big = torch.zeros((1, 3), device="cuda")
    out = ctypes.c_double(123.0)
    rc = mpm.lib().mpm_loss_mse_noalloc(ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                                        4194304 + 1, None, ctypes.byref(out), None)
    assert rc == -1 and out.value == 123.0
