"""Seeded synthetic galaxy particle sets (the inputs of the QUMOND path).

Both the CUDA path and the CPU oracle are fed from here; nothing in this
package computes any part of the method itself (no deposit, no solve, no
source, no force).  All randomness comes from numpy's PCG64 generator seeded
by the caller, so a seed fixes every particle bit for bit.

Units: pc, Msun.
"""
from .galaxies import (  # noqa: F401
    Particles,
    kuzmin_disk,
    exponential_disk,
    hernquist_bulge,
    two_component_disk,
    large_galaxy,
    fit_sweep_parameters,
    SweepGalaxy,
)
