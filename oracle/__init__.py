"""Plain FP64 CPU oracle of weighted-quadrature assembly.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline legs of bench.py. The CUDA library never imports or links it,
and it imports nothing from the CUDA library.
"""
from .wq_oracle import (Direction, Oracle3D, bspline_all, cardinal_bspline, coefficients,
                        exact_integrals, galerkin_dense, quadrature_points, wq_rule, COEF_LM)
from .wq_oracle_c import build_oracle, rows_c

__all__ = ["Direction", "Oracle3D", "bspline_all", "cardinal_bspline", "coefficients",
           "exact_integrals", "galerkin_dense", "quadrature_points", "wq_rule", "COEF_LM",
           "build_oracle", "rows_c"]
