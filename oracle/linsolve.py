"""Linear solves for the implicit stages (oracle; test infrastructure only).

The paper does not name its linear solver. Each implicit Euler stage of
Algorithms 1 and 2 solves (diag(m) + dtau K) x = b with K symmetric positive
definite (K = -(A + B_env), Sec. 2), so the reading taken here is the
textbook Jacobi-preconditioned conjugate gradient method, stopped when
||r||_2 <= rtol ||b||_2, with a dense Cholesky solve as an exact alternative
for small systems.

Parity: pinned by tests/test_oracle_stepper.py (PCG agrees with a dense
Cholesky solve to the requested tolerance).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pcg(apply_A, b, x0, dinv, rtol=1e-12, max_iter=2000):
    """Jacobi-preconditioned CG. Returns (x, iterations, converged)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_A(x)
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    bnorm = float(np.linalg.norm(b))
    it = 0
    while it < max_iter:
        if float(np.linalg.norm(r)) <= rtol * bnorm:
            return x, it, True
        Ap = apply_A(p)
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        z = dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, float(np.linalg.norm(r)) <= rtol * bnorm


def dense_solve(A_dense, b):
    """Cholesky solve of a small SPD system."""
    c, low = sla.cho_factor(A_dense)
    return sla.cho_solve((c, low), b)
