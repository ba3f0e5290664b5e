"""The plain definition of the three outputs, through a Householder QR of A^*.

Test infrastructure only (see ``oracle/__init__.py``).

For a full-rank m x n matrix A (m <= n), Section 1 lists the outputs: the
projection Zb of b onto the null space of A (Eq. 1: Zb = b - A^*(AA^*)^{-1}Ab),
the projection onto the row space, and the minimiser h of ||A^* h - b||
(Remark 4.1). With the Householder QR A^* = Q R (Q n x m with orthonormal
columns, R m x m upper triangular; Golub & Van Loan Ch. 5, the decomposition the
paper uses throughout Section 5) these are

    row(b)  = Q Q^* b,      Zb = b - Q Q^* b,      h = R^{-1} Q^* b.

Right-hand sides are stored as rows: B is k x n, row j is the j-th vector.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = ["householder_qr", "qr_factor", "project", "null_project", "row_project", "lstsq"]


def householder_qr(M: np.ndarray):
    """Textbook Householder QR of a tall p x q matrix (p >= q), Golub & Van Loan Alg. 5.2.1.

    Returns (V, beta, R): column j of V is the Householder vector v_j (zero above
    row j), H_j = I - beta_j v_j v_j^*, and H_{q-1}...H_0 M = [R; 0].
    Slow and plain; used to cross-check the library QR at small sizes.
    """
    M = np.array(M, dtype=np.float64, copy=True)
    p, q = M.shape
    if p < q:
        raise ValueError("householder_qr needs a tall matrix")
    V = np.zeros((p, q))
    beta = np.zeros(q)
    for j in range(q):
        x = M[j:, j].copy()
        nx = np.linalg.norm(x)
        if nx == 0.0:
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x
        v[0] -= alpha
        vv = v @ v
        b = 2.0 / vv
        M[j:, j:] -= b * np.outer(v, v @ M[j:, j:])
        M[j + 1:, j] = 0.0
        V[j:, j] = v
        beta[j] = b
    return V, beta, np.triu(M[:q, :q])


def householder_apply_qt(V, beta, X):
    """Q^* X for the Q of ``householder_qr`` (X is p x k)."""
    X = np.array(X, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        v = V[j:, j]
        X[j:] -= beta[j] * np.outer(v, v @ X[j:])
    return X


def householder_apply_q(V, beta, X):
    """Q X for the Q of ``householder_qr`` (X is p x k)."""
    X = np.array(X, dtype=np.float64, copy=True)
    for j in range(V.shape[1] - 1, -1, -1):
        v = V[j:, j]
        X[j:] -= beta[j] * np.outer(v, v @ X[j:])
    return X


def qr_factor(A: np.ndarray):
    """Reduced Householder QR of A^* through LAPACK (dgeqrf/dorgqr): returns (Q, R)."""
    A = np.asarray(A, dtype=np.float64)
    q, r = np.linalg.qr(A.T, mode="reduced")
    return q, r


def project(A: np.ndarray, B: np.ndarray, factors=None):
    """All three outputs for right-hand sides B (k x n rows).

    Returns (Z, ROW, H): Z and ROW are k x n (null-space and row-space
    projections), H is k x m (least-squares solutions, one per row).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.atleast_2d(np.asarray(B, dtype=np.float64))
    q, r = qr_factor(A) if factors is None else factors
    y = B @ q                      # (Q^* b)^T for every row b of B
    row = y @ q.T                  # (Q Q^* b)^T
    z = B - row
    h = sla.solve_triangular(r, y.T, lower=False).T
    return z, row, h


def null_project(A, B):
    return project(A, B)[0]


def row_project(A, B):
    return project(A, B)[1]


def lstsq(A, B):
    return project(A, B)[2]
