"""H²-matrix Galerkin single-layer product and GMRES on one GB300 GPU.

The compute path lives in ``libh2.so`` (CUDA kernels for sm_103a behind the
C ABI of ``include/h2.h``); this package only marshals arguments.
"""
from ._lib import (H2_F32, H2_F64, EXPORTED, PHASES, Batch, GcaMatrix, H2Error, H2Matrix, HelmholtzMatrix, Plan,  # noqa: F401
                   ProductGraph, Server,
                   colmajor, library_path, load)
from ._build import build as build_library  # noqa: F401
