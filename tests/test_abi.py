"""CPU checks of the C-ABI library: it builds, loads, exports every entry
point that include/mpm.h declares (and the binding names no other), and
rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2510_17335_gb300 import build as libbuild
from paper_2510_17335_gb300 import mpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return mpm.lib()


def declared():
    hdr = open(os.path.join(ROOT, "include", "mpm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return set(re.findall(r"\b(mpm_[a-z_0-9]+)\s*\(", hdr))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert names == set(mpm.EXPORTS), names ^ set(mpm.EXPORTS)


def test_error_strings_and_version(L):
    assert L.mpm_version() == 1
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert len(L.mpm_error_string(code)) > 0
    assert L.mpm_error_string(-99) == b"unknown error"


def _create(L, cfg, mat, x, opts=None):
    h = ctypes.c_void_p()
    n = np.asarray(x, np.float32).reshape(-1, 3)
    cnt = (ctypes.c_int64 * 1)(n.shape[0])
    return L.mpm_create(1, (mpm.mpm_config * 1)(cfg), (mpm.mpm_material * 1)(mpm.mpm_material(*mat)), cnt,
                        n.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts) if opts else None, ctypes.byref(h))


def test_invalid_arguments_are_rejected(L):
    dx = 1.0 / 16
    good = mpm.make_config((16, 16, 16), dx, 1e-4, dx ** 3 / 8)
    x = np.array([[0.5, 0.5, 0.5]], np.float32)
    mat = (1e5, 0.3, 1500.0, 30.0)
    assert _create(L, good, (1e5, 0.5, 1500.0, 30.0), x) == -1          # nu = 0.5
    assert _create(L, good, (-1.0, 0.3, 1500.0, 30.0), x) == -1         # E < 0
    assert _create(L, good, (1e5, 0.3, 1500.0, 95.0), x) == -1          # phi > 90
    bad = mpm.make_config((16, 16, 16), dx, 0.0, dx ** 3 / 8)
    assert _create(L, bad, mat, x) == -1                                # dt = 0
    bad = mpm.make_config((4, 16, 16), dx, 1e-4, dx ** 3 / 8)
    assert _create(L, bad, mat, x) == -1                                # res too small
    assert _create(L, good, mat, np.array([[0.5, 0.5, 0.97]], np.float32)) == -4   # outside [dx, (res-2) dx)
    assert _create(L, good, mat, np.array([[0.5, 0.01, 0.5]], np.float32)) == -4
    assert _create(L, good, mat, np.array([[0.5, np.nan, 0.5]], np.float32)) == -1
    assert _create(L, good, mat, x, mpm.make_options(checkpoint_every=0)) == -1
    assert _create(L, good, mat, x, mpm.make_options(grad_scale=3)) == -1            # no such regulariser
    assert _create(L, good, mat, x, mpm.make_options(grad_scale=1, clip_grads=1)) == -1   # one at a time
    assert _create(L, good, mat, x, mpm.make_options(grad_scale=2, grad_delta=0.0)) == -1
    h = ctypes.c_void_p()
    assert L.mpm_create(0, None, None, None, None, None, ctypes.byref(h)) == -1
    # NULL handles
    assert L.mpm_forward(None, 1, 0) == -1
    assert L.mpm_backward(None, None, None, 0, None, None) == -1
    assert L.mpm_reset(None) == -1
    L.mpm_destroy(None)


def test_profile_kernel_table_matches_header(L):
    hdr = open(os.path.join(ROOT, "include", "mpm.h")).read()
    n = int(re.search(r"#define MPM_PROFILE_KERNELS (\d+)", hdr).group(1))
    assert n == mpm.PROFILE_KERNELS
    names = [L.mpm_kernel_name(k).decode() for k in range(n)]
    assert all(names) and len(set(names)) == n
    assert L.mpm_kernel_name(n) == b"" and L.mpm_kernel_name(-1) == b""
    # every id the header lists in its profile comment names the same kernel
    for k, name in re.findall(r"(\d+) (k_[a-z0-9_]+)", hdr):
        if int(k) < n:
            assert names[int(k)] == name, (k, name)


def test_noalloc_wrapper_rejects_bad_arrays_before_launch(monkeypatch):
    """The Python wrapper of mpm_loss_mse_noalloc checks shapes, dtypes and
    devices before it reaches the library: a short target or gradient
    buffer would otherwise be read or written past its end on the GPU."""
    import torch

    def no_lib():
        raise AssertionError("the library must not be reached")

    monkeypatch.setattr(mpm, "lib", no_lib)
    x = torch.zeros((8, 3))
    with pytest.raises(ValueError, match="target has shape"):
        mpm.loss_mse_noalloc(x, torch.zeros((7, 3)))
    with pytest.raises(ValueError, match="dL_dx has shape"):
        mpm.loss_mse_noalloc(x, torch.zeros((8, 3)), torch.zeros((4, 3)))
    with pytest.raises(ValueError, match=r"x must be \[n, 3\]"):
        mpm.loss_mse_noalloc(torch.zeros((8, 2)), torch.zeros((8, 2)))
    with pytest.raises(ValueError, match="x must be"):
        mpm.loss_mse_noalloc(torch.zeros(24), torch.zeros(24))
    with pytest.raises(ValueError, match="float32"):
        mpm.loss_mse_noalloc(x.double(), torch.zeros((8, 3)))
    with pytest.raises(TypeError):
        mpm.loss_mse_noalloc(np.zeros((8, 3), np.float32), torch.zeros((8, 3)))
    # right shapes, but host tensors: rejected as well
    with pytest.raises(ValueError, match="CUDA tensor"):
        mpm.loss_mse_noalloc(x, torch.zeros((8, 3)), torch.zeros((8, 3)))


def test_record_bytes_follow_the_layout(L):
    """mpm_record_bytes (host only): a state slot holds x, v, C, F (96 B a
    particle); a substep slot the SVD record (U and V as quaternions, the
    singular values and sigma^2 - 1: 56 B a particle), the accumulators and
    velocities (32 B a node) and the touched-block flags and list."""
    state, sub = mpm.record_bytes(1_048_576, 128 ** 3)
    assert state == 96 * 1_048_576
    blocks = 128 ** 3 // 64
    assert sub == 56 * 1_048_576 + 32 * 128 ** 3 + 4 * (2 * (blocks + 1) + 1)
    assert mpm.blocked_nodes((97, 64, 65)) == 100 * 64 * 68
    a, b = ctypes.c_int64(), ctypes.c_int64()
    assert L.mpm_record_bytes(-1, 10, ctypes.byref(a), ctypes.byref(b)) == -1
