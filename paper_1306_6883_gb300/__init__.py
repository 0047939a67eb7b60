"""GB300 (sm_103a) implementation of the unsplit piecewise-linear CTU step of the compressible solver
of "pyro: a teaching code for computational astrophysical hydrodynamics" (paper §3.2).

The computation lives in libhydro.so (CUDA kernels behind the C ABI of include/hydro.h); `hydro` is its
ctypes binding and `solver.Solver` a convenience wrapper that lets PyTorch own the device buffers.
"""
from . import hydro  # noqa: F401
