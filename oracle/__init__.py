"""FP64 CPU oracle of the QUMOND particle-mesh path (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  It is
the plain, slow reference the CUDA path is checked against; the two share no
code.  The arithmetic lives in ``qumond_oracle.c`` (plain C, FP64, natural
grid layout); this module only marshals numpy arrays and strings the C steps
together in the order of Section 2 of the paper (``pipeline``).
"""
from .core import (  # noqa: F401
    build,
    lib_path,
    cic_deposit,
    rho_from_fixed,
    relax_rbgs,
    residual,
    interior_sumsq,
    restrict_fw,
    prolong,
    coarsest,
    vcycle,
    fmg,
    solve,
    source,
    boundary_fill,
    forces,
    rotation_curve,
    chi2,
    rotation_curve_algebraic,
    sigma_z,
    far_field,
    Box,
    pipeline,
    grid_index,
)
