"""Extreme eigenvalues and the condition-number estimate of the global and the condensed
matrices (test infrastructure only).

Sec. 4 (Fig. ConditionNumber) approximates the L2 condition number of a system matrix by
the ratio of the moduli of its largest and smallest eigenvalues.  The oracle takes that
definition literally on small systems: every eigenvalue of the dense matrix (numpy's
eigvals, a library primitive used as one step), then the two extremes by modulus.
"""
from __future__ import annotations

import numpy as np


def extreme_eigenvalues(M: np.ndarray):
    """(eigenvalue of largest modulus, eigenvalue of smallest modulus, ratio of the moduli)."""
    ev = np.linalg.eigvals(np.asarray(M, dtype=np.float64))
    lmax = ev[np.argmax(np.abs(ev))]
    lmin = ev[np.argmin(np.abs(ev))]
    return complex(lmax), complex(lmin), float(np.abs(lmax) / np.abs(lmin))


def condition_estimates(A, n: int, N: int):
    """The estimate for the global Jacobian A (scipy sparse or dense) and for its condensed
    matrix S = A_bb - A_bi A_ii^-1 A_ib (Sec. 2.2): {'A': (...), 'S': (...)}."""
    from .linalg import condensed_operator
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    S = condensed_operator(A, n, N).dense_S()
    return {"A": extreme_eigenvalues(Ad), "S": extreme_eigenvalues(S)}
