"""CPU check of the CUDA library's constitutive arithmetic: the device
functions the kernels call (SVD on F^T F - I, Drucker-Prager return, SVK
stress, and the vector-Jacobian-product adjoint), compiled for the host,
against the FP64 oracle. The FP64 instantiation must agree to 1e-7 relative; the
FP32 instantiation (what the kernels run) to FP32 accuracy."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2510_17335_gb300.workloads import random_rotation

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host_math", "cuda_math_host.cu")
SO = os.path.join(ROOT, "_build", "libmpm_hostmath.so")
DEPS = [SRC] + [os.path.join(ROOT, "paper_2510_17335_gb300", "csrc", f) for f in ("mpm_device.cuh", "mpm_types.h")]


@pytest.fixture(scope="module")
def hm():
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if not os.path.exists(SO) or any(os.path.getmtime(d) > os.path.getmtime(SO) for d in DEPS):
        subprocess.run(["nvcc", "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
                        "-shared", "-o", SO, SRC], check=True)
    L = ctypes.CDLL(SO)
    dp = ctypes.POINTER(ctypes.c_double)
    L.hm_constitutive_adjoint.argtypes = ([ctypes.c_int, dp] + [ctypes.c_double] * 4 + [dp] * 6 +
                                          [ctypes.POINTER(ctypes.c_int)])
    return L


def _call(L, fp64, Ft, mu, lam, alpha, gFn, gtau):
    d = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    Fn, tau, gFt, gp = np.zeros(9), np.zeros(9), np.zeros(9), np.zeros(3)
    k = ctypes.c_int()
    Ftc, gFc, gtc = [np.ascontiguousarray(a, np.float64).ravel() for a in (Ft, gFn, gtau)]
    L.hm_constitutive_adjoint(fp64, d(Ftc), mu, lam, alpha, 1e-4, d(gFc), d(gtc), d(Fn), d(tau), d(gFt), d(gp),
                              ctypes.byref(k))
    return Fn.reshape(3, 3), tau.reshape(3, 3), gFt.reshape(3, 3), gp, k.value


CASES = [[0.03, 0.01, 0.02], [-0.010, -0.012, -0.008], [0.03, -0.06, 0.0], [0.02, 0.02, -0.08],
         [-0.01, -0.01, -0.012], [0.05, -0.12, 0.01], [-0.002, -0.0021, -0.0019], [1e-6, -2e-6, 5e-7]]


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("mat", [(1e5, 0.3, 30.0), (3e5, 0.25, 35.0), (5e4, 0.4, 15.0)])
def test_kernel_constitutive_matches_oracle(hm, ci, mat):
    rng = np.random.default_rng(100 * ci + int(mat[2]))
    mu, lam, alpha = oracle.material(*mat)
    eps = np.array(CASES[ci])
    Ft = random_rotation(rng) @ np.diag(np.exp(eps)) @ random_rotation(rng)
    gFn, gtau = rng.normal(size=(3, 3)), rng.normal(size=(3, 3)) / mu
    for fp64, tol in ((1, 1e-7), (0, 2e-4)):
        # the FP32 kernel sees the FP32-rounded inputs: so does the oracle here
        F_in = Ft if fp64 else Ft.astype(np.float32).astype(np.float64)
        gF_in = gFn if fp64 else gFn.astype(np.float32).astype(np.float64)
        gt_in = gtau if fp64 else gtau.astype(np.float32).astype(np.float64)
        Fn_o, tau_o, info = oracle.constitutive(F_in, mu, lam, alpha)
        gFt_o, gm_o, gl_o, ga_o = oracle.constitutive_adjoint(F_in, mu, lam, alpha, gF_in, gt_in)
        Fn, tau, gFt, gp, kase = _call(hm, fp64, F_in, mu, lam, alpha, gF_in, gt_in)
        assert kase == int(info[0])
        assert np.allclose(Fn, Fn_o, rtol=0, atol=tol * 10)
        assert np.allclose(tau, tau_o, rtol=0, atol=tol * 10 * max(1.0, np.abs(tau_o).max()))
        sc = max(np.abs(gFt_o).max(), 1e-30)
        assert np.allclose(gFt, gFt_o, rtol=0, atol=tol * sc), (fp64, gFt, gFt_o)
        for a, b in zip(gp, (gm_o, gl_o, ga_o)):
            assert abs(a - b) <= tol * max(abs(b), 1e-6 * max(abs(gm_o), abs(gl_o), abs(ga_o), 1e-30)), (fp64, gp,
                                                                                                          (gm_o, gl_o, ga_o))
