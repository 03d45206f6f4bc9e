"""GB300-native QUMOND particle-mesh hot path (Angus et al., arXiv:1201.3185).

Importing the package loads libqumond.so (built by ``build.build()``); it
raises ImportError if the library is missing.  There is no CPU fallback.
"""
from .qumond import (  # noqa: F401
    Context,
    Guess,
    NotConverged,
    QumondError,
    SolveStats,
    default_params,
    QUMOND_PREC_FP64,
    QUMOND_PREC_MIXED,
    QUMOND_PREC_MIXED_FIXED,
    QUMOND_BC_ZERO,
    QUMOND_BC_GIVEN,
    QUMOND_BC_MULTIPOLE,
    EXPORTED,
)
from .pipeline import Pipeline, PipelineResult, run_lanes  # noqa: F401
from .sweep import FitSweep, SweepResult, autotune, tune_workers  # noqa: F401
