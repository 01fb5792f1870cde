"""GB300 (sm_103a) library for adjoint-based optimal control of jump-diffusion processes.

Evaluates the Monte Carlo reduced cost J(u) of a controlled SDE with compound-Poisson
jumps and its exact discrete-adjoint gradient (discretize-then-optimize, after
"Adjoint-based optimal control of jump-diffusion processes", arXiv 2505.04328), and
minimizes it by projected gradient descent with the Armijo rule.  All numerics run in
the CUDA library libjd.so (C ABI: include/jd.h); this package only marshals arguments.
"""
from .binding import (ABI_SYMBOLS, UNIT_PATHS, JdError, JdProblem, JdServer, combine_units,  # noqa: F401
                      footprint, launch_count, lib, library_path, profile_enable, profile_read)

__all__ = ["JdProblem", "JdServer", "JdError", "footprint", "combine_units", "UNIT_PATHS", "lib", "library_path",
           "launch_count", "ABI_SYMBOLS", "build"]


def build(verbose: bool = False) -> str:
    """Compile libjd.so for sm_103a (nvcc required)."""
    from . import _build
    return _build.build(verbose=verbose)
