"""B300-native (sm_103a) matrix-free staggered-grid Stokes solver: multigrid-preconditioned FGMRES.

The compute path is libpyro.so (CUDA kernels + C ABI, include/pyro.h); this package is its thin
Python binding plus the autograd wrapper and the continuous-batching solve server.
"""
from .pyro import (Stokes, Markers, LATTICE_NODES, LATTICE_CELLS, LATTICE_VX, LATTICE_VY, ADVECT_EULER, ADVECT_HEUN,
                   ADVECT_RK4, ADVECT_TAYLOR, PyroError, PyroOpts, PyroBC, PyroStats, default_opts, make_bc, footprint, lib,
                   load_library, EXPORTED, FREE_SLIP, NO_SLIP, PERIODIC, VELOCITY, PREC_FP64, PREC_MIXED,
                   ETA_ARITH, ETA_GEOM, PYRO_OK, PYRO_W_NOT_CONVERGED, ACCEL_FGMRES, ACCEL_GCR, ACCEL_ANDERSON, SMOOTH_RBGS, SMOOTH_JACOBI,
                   SMOOTH_RAS, SMOOTH_MIXED, fp64_fma_rate, residual_noalloc)

__all__ = ["Stokes", "Markers", "LATTICE_NODES", "LATTICE_CELLS", "LATTICE_VX", "LATTICE_VY", "ADVECT_EULER",
           "ADVECT_HEUN", "ADVECT_RK4", "ADVECT_TAYLOR", "PyroError", "PyroOpts", "PyroBC", "PyroStats", "default_opts", "make_bc", "footprint", "lib",
           "load_library", "EXPORTED", "FREE_SLIP", "NO_SLIP", "PERIODIC", "VELOCITY", "PREC_FP64", "PREC_MIXED",
           "ETA_ARITH", "ETA_GEOM", "PYRO_OK", "PYRO_W_NOT_CONVERGED", "ACCEL_FGMRES", "ACCEL_GCR",
           "ACCEL_ANDERSON", "SMOOTH_RBGS", "SMOOTH_JACOBI", "SMOOTH_RAS",
           "SMOOTH_MIXED", "fp64_fma_rate", "residual_noalloc"]
