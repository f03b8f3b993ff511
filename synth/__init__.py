"""Seeded synthetic inputs for the Stokes workloads (shared by the oracle tests, the GPU tests and the bench).

This package only draws random numbers and paints material fields; it contains none of the
solver's arithmetic (no stencils, no transfer operators, no Krylov steps).
"""
from .fields import (Fields, sample_lattice_to_fields, sinker, random_field_log10,
                     random_inclusions_density, grf_config, layered_config, serving_request,
                     adjoint_member, random_vectors)

__all__ = ["Fields", "sample_lattice_to_fields", "sinker", "random_field_log10",
           "random_inclusions_density", "grf_config", "layered_config", "serving_request",
           "adjoint_member", "random_vectors"]
