"""GB300-native (sm_103a) MLS-MPM sand/soil substep and its adjoint.

The compute path is a C-ABI shared library (``libmpm_gb300.so``, built from
``csrc/``); ``mpm`` is its thin ctypes binding and ``autograd`` wraps it in a
``torch.autograd.Function``. ``workloads`` holds the seeded input recipes.
Importing this package does not load the CUDA library; ``mpm.lib()`` does,
and raises if the library has not been built.
"""
__all__ = ["mpm", "workloads"]
