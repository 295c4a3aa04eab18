"""GB300-native CTU-MHD patch integrator (sm_103a CUDA behind a C ABI).

`ctu` is the ctypes binding of libctu.so (include/ctu.h); `workloads`
builds the seeded synthetic inputs; `_build` compiles the library.
"""
from . import workloads  # noqa: F401

__all__ = ["ctu", "workloads"]
