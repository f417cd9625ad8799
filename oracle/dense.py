"""Dense cross-checks for tiny problems (oracle; test infrastructure only).

Builds the skew matrix Q of eq. (19) explicitly and solves (I + Q) u = omega
with a dense LU, independently of the block eliminations of Section IV.
"""

from __future__ import annotations

import numpy as np

from .conic import ConicData


def Q_matrix(cd: ConicData) -> np.ndarray:
    """Q = [0 -A^T c; A 0 -b; -c^T b^T 0] (eq. (19))."""
    A = cd.A.toarray()
    m, nx = A.shape
    n = nx + m + 1
    Q = np.zeros((n, n))
    Q[:nx, nx:nx + m] = -A.T
    Q[:nx, -1] = cd.c
    Q[nx:nx + m, :nx] = A
    Q[nx:nx + m, -1] = -cd.b
    Q[-1, :nx] = -cd.c
    Q[-1, nx:nx + m] = cd.b
    return Q


def affine_dense(cd: ConicData, omega: np.ndarray) -> np.ndarray:
    Q = Q_matrix(cd)
    return np.linalg.solve(np.eye(Q.shape[0]) + Q, omega)
