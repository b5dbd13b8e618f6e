"""Mixed-precision iterative refinement, step by step -- TEST INFRASTRUCTURE.

The algorithm (classical iterative refinement, Wilkinson 1963; Moler 1967):

    x_0 = solve_f32(A, d)
    repeat for k = 0, 1, ...:
        r_k = d - A x_k                 (fp64)
        delta_k = solve_f32(A, r_k)     (binary32 elimination)
        x_{k+1} = x_k + delta_k         (fp64)
    until ||delta_k||_inf <= tol * ||x_{k+1}||_inf or k reaches max_iters.

solve_f32 rounds its matrix and right-hand side to binary32 and runs the
Thomas recurrences in binary32 (``oracle.thomas_f32``).  When it converges
the result is A^{-1} d to fp64 accuracy, so the tests compare it -- and the
GPU refinement -- against the fp64 Thomas solution.
"""
from __future__ import annotations

import numpy as np

from . import residual, thomas_f32


def refine(a, b, c, d, tol=1e-12, max_iters=10):
    """Returns (x, iterations, converged)."""
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    x = thomas_f32(a, b, c, d).astype(np.float64)
    for k in range(1, max_iters + 1):
        r = residual(a, b, c, d, x)
        delta = thomas_f32(a, b, c, r).astype(np.float64)
        x = x + delta
        xn = float(np.max(np.abs(x))) if x.size else 0.0
        dn = float(np.max(np.abs(delta))) if delta.size else 0.0
        if dn <= tol * xn:
            return x, k, True
    return x, max_iters, False
