"""Plain FP64 CPU oracle for the H²-matrix Galerkin single-layer product.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and
the CPU-baseline leg of the benchmark, never by the library.  The arithmetic
lives in ``h2oracle.c`` (plain C, FP64); this module compiles it with gcc and
wraps it with ctypes.  See ``h2oracle.c`` for the paper passages each step
follows and for the readings taken where the paper is silent.
"""
from .oracle import (Oracle, HelmholtzOracle, GcaOracle, build_library, gauss01, pair_quad,  # noqa: F401
                     green_rule, aca, KIND_LAPLACE, KIND_POLY, KIND_HELM_COS, KIND_HELM_SIN)
