"""GB300 implementation of the contour-integral Helmholtz solver (arXiv 1811.12378):
the shifted 7-point stencil, the polynomial fixed-point scheme at every contour node, the
FCI preconditioner (Algorithm 1) and flexible GMRES, as CUDA kernels behind the C ABI of
include/hz.h.  ``hz`` is the Python binding (argument marshalling only)."""
from .hz import (HZ_DISC_FD7, HZ_DISC_SPECTRAL, HZ_C128, HZ_MIXED_C64, HZ_MIXED_C64_FCI32, HZ_MIXED_C64_FF, HZ_LIMIT_SWEEPS_C64,
                 HZ_LIMIT_Z_C64, HZ_LIMIT_CASE_TWO, EXPORTS, PROF_KRYLOV, PROF_POLY, PROF_STENCIL, HzError,
                 Problem, SolveStats, launch_count, library_path, load, plan, solve_batched,
                 Net, NET_CONVS, flatten_params, unflatten_params, init_params, conv3d,
                 conv3d_backward)

__all__ = ["HZ_DISC_FD7", "HZ_DISC_SPECTRAL", "HZ_C128", "HZ_MIXED_C64", "HZ_MIXED_C64_FCI32", "HZ_MIXED_C64_FF",
           "HZ_LIMIT_SWEEPS_C64", "HZ_LIMIT_Z_C64", "HZ_LIMIT_CASE_TWO", "EXPORTS", "PROF_KRYLOV", "PROF_POLY", "PROF_STENCIL",
           "HzError", "Problem", "SolveStats",
           "launch_count", "library_path", "load", "plan", "solve_batched",
           "Net", "NET_CONVS", "flatten_params", "unflatten_params", "init_params", "conv3d",
           "conv3d_backward"]
