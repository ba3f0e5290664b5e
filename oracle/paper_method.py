"""The algorithm of Section 4, step by step, in float64.

Test infrastructure only (see ``oracle/__init__.py``).

Notation follows Section 4. A is m x n with m <= l <= n, G is n x l.

Preconditioner (Eqs. 12-13):
  1. S = A G (Eq. 12), m x l.
  2. Pivoted QR of S^*: S^* = Q R Pi (Eq. 13), Q l x m orthonormal columns, R m x m
     upper triangular, Pi an m x m permutation. Then P = Pi^* R^*.
Y (Eqs. 14-16):
  1. P^- = Pi^* R^{-1} (Eq. 15).
  2. Column k of X (k = 1..m): c = P^- e_k; d = A^* c; e = A d; f = Pi e;
     solve R^* x = f. (X = P^{-1} A A^* (P^*)^{-1}.)
  3. Y = X^{-1} (Eq. 16).
Apply to b, seven steps:
  c = A b; d = Pi c; solve R^* e = d; f = Y e; solve R g = f; h = Pi^* g;
  b~ = A^* h. Then Zb = b - b~ (null space), b~ is the row-space projection and
  h solves min ||A^* h - b|| (Remark 4.1).
Refinement (Remark 4.3): the paper refines h as in Dahlquist & Bjorck Sec. 5.7.3
and reprojects the projection, without spelling out the update. This oracle reads
it as: s = b - A^* h0, r = A s, dh = (steps 2-6 applied to r), h1 = h0 + dh,
Zb = s - A^* dh, which refines h and reprojects Zb in one pass.

Permutation convention: the pivoted QR returns ``perm`` with
S^*[:, perm] = Q R, i.e. position j holds original column perm[j]. Then
(Pi x)[j] = x[perm[j]] (a gather) and Pi^* scatters back.

Readings where the paper is silent: the pivoting rule is Businger-Golub (largest
remaining column norm, lowest index on ties, norms recomputed each step); the
inverse in Eq. 16 is LAPACK's LU-based inverse; reflectors use
alpha = -sign(x_1) ||x||.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

__all__ = [
    "sketch", "pivoted_qr", "Preconditioner", "precondition", "gram_columns",
    "apply_seven_steps", "refine", "project",
]


def sketch(A: np.ndarray, G: np.ndarray) -> np.ndarray:
    """S = A G (Eq. 12). The paper forms it one column of G at a time to avoid
    storing G; the product is the same (a library matmul)."""
    return np.asarray(A, np.float64) @ np.asarray(G, np.float64)


def pivoted_qr(M: np.ndarray):
    """Businger-Golub column-pivoted Householder QR of a p x q matrix M (p >= q).

    Returns (Q, R, perm) with M[:, perm] = Q R, Q p x q with orthonormal columns,
    R q x q upper triangular with non-increasing |R_kk|.
    """
    M = np.array(M, dtype=np.float64, copy=True)
    p, q = M.shape
    if p < q:
        raise ValueError("pivoted_qr needs p >= q")
    perm = np.arange(q)
    V = np.zeros((p, q))
    beta = np.zeros(q)
    for j in range(q):
        norms = np.einsum("ij,ij->j", M[j:, j:], M[j:, j:])
        piv = j + int(np.argmax(norms))          # argmax returns the lowest index on ties
        if piv != j:
            M[:, [j, piv]] = M[:, [piv, j]]
            perm[[j, piv]] = perm[[piv, j]]
        x = M[j:, j].copy()
        nx = np.linalg.norm(x)
        if nx == 0.0:
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x
        v[0] -= alpha
        b = 2.0 / (v @ v)
        M[j:, j:] -= b * np.outer(v, v @ M[j:, j:])
        M[j + 1:, j] = 0.0
        V[j:, j] = v
        beta[j] = b
    R = np.triu(M[:q, :q])
    Q = np.eye(p, q)
    for j in range(q - 1, -1, -1):
        v = V[j:, j]
        Q[j:] -= beta[j] * np.outer(v, v @ Q[j:])
    return Q, R, perm


@dataclasses.dataclass
class Preconditioner:
    """R, Pi (as perm) and Y of Section 4, plus the intermediates for testing."""
    R: np.ndarray
    perm: np.ndarray
    Y: np.ndarray
    X: np.ndarray
    S: np.ndarray
    Q: np.ndarray

    def pinv_columns(self) -> np.ndarray:
        """P^- = Pi^* R^{-1} (Eq. 15)."""
        m = self.R.shape[0]
        rinv = sla.solve_triangular(self.R, np.eye(m), lower=False)
        out = np.empty_like(rinv)
        out[self.perm, :] = rinv          # Pi^* scatters rows back
        return out


def gram_columns(A: np.ndarray, R: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """X = P^{-1} A A^* (P^*)^{-1}, built column by column with steps a-e of Section 4."""
    A = np.asarray(A, np.float64)
    m = R.shape[0]
    rinv = sla.solve_triangular(R, np.eye(m), lower=False)
    pminus = np.empty_like(rinv)
    pminus[perm, :] = rinv
    X = np.empty((m, m))
    for k in range(m):
        c = pminus[:, k]                              # a. k-th column of P^-
        d = A.T @ c                                   # b. d = A^* c
        e = A @ d                                     # c. e = A d
        f = e[perm]                                   # d. f = Pi e
        X[:, k] = sla.solve_triangular(R.T, f, lower=True)  # e. solve R^* x = f
    return X


def precondition(A: np.ndarray, G: np.ndarray) -> Preconditioner:
    """R, Pi and Y from A and the test matrix G (Eqs. 12-16)."""
    S = sketch(A, G)
    Q, R, perm = pivoted_qr(S.T)
    X = gram_columns(A, R, perm)
    Y = np.linalg.inv(X)
    return Preconditioner(R=R, perm=perm, Y=Y, X=X, S=S, Q=Q)


def _middle(pc: Preconditioner, C: np.ndarray) -> np.ndarray:
    """Steps 2-6 on columns c (m x k): d = Pi c; R^* e = d; f = Y e; R g = f; h = Pi^* g."""
    d = C[pc.perm, :]
    e = sla.solve_triangular(pc.R.T, d, lower=True)
    f = pc.Y @ e
    g = sla.solve_triangular(pc.R, f, lower=False)
    h = np.empty_like(g)
    h[pc.perm, :] = g
    return h


def apply_seven_steps(A: np.ndarray, pc: Preconditioner, B: np.ndarray):
    """The seven-step apply for right-hand sides B (k x n rows).

    Returns (Z, ROW, H) with Z = B - B~ (k x n), ROW = B~ (k x n), H (k x m)."""
    A = np.asarray(A, np.float64)
    B = np.atleast_2d(np.asarray(B, np.float64))
    C = A @ B.T                       # 1. c = A b
    H = _middle(pc, C)                # 2.-6.
    ROW = (A.T @ H).T                 # 7. b~ = A^* h
    return B - ROW, ROW, H.T


def refine(A: np.ndarray, pc: Preconditioner, B: np.ndarray, H0: np.ndarray, passes: int = 1):
    """Refinement of Remark 4.3 in float64 (reading stated in the module docstring).

    Returns (Z, ROW, H) after ``passes`` refinement passes starting from H0 (k x m)."""
    A = np.asarray(A, np.float64)
    B = np.atleast_2d(np.asarray(B, np.float64))
    H = np.array(H0, dtype=np.float64, copy=True).T          # m x k
    S = B.T - A.T @ H                                         # s = b - A^* h0  (n x k)
    for _ in range(passes):
        r = A @ S                                             # r = A s
        dH = _middle(pc, r)                                   # dh
        H = H + dH                                            # h1 = h0 + dh
        S = S - A.T @ dH                                      # Zb = s - A^* dh
    Z = S.T
    return Z, B - Z, H.T


def project(A, G, B, refine_passes: int = 0):
    """Precondition with G, then apply (and optionally refine) for B."""
    pc = precondition(A, G)
    Z, ROW, H = apply_seven_steps(A, pc, B)
    if refine_passes:
        Z, ROW, H = refine(A, pc, B, H, refine_passes)
    return Z, ROW, H, pc
