"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package holds no arithmetic of the time step itself: it only builds the
grid spacing, the initial prognostic fields, the (given, steady) mass fluxes
and the time step length that both implementations take as inputs.
"""
from .fields import (  # noqa: F401
    CONFIGS, SEED_BASE, DX, DY, Case, make_dz, make_case, make_config_case,
    make_ensemble_cases, ensemble_sizes, DAMPING, make_boundary_data,
    ACOUSTIC, make_acoustic_state, halo_periodic, halo_strips, extend_fluxes, split_extent,
    subdomain, make_open_boundary, HEVI, make_hevi_state,
)
