"""Exact projections for the paper's test family (Eqs. 20-21), at any condition number.

Test infrastructure only (see ``oracle/__init__.py``).

A = U [B | B | ... | B] V with B (m x m) invertible and U, V permutations
(Section 5). For any y, A^* y = V^* [B^* U^* y; ...; B^* U^* y], and B^* U^* is
onto R^m, so the row space of A is V^* applied to the "repeated block" vectors
[w; w; ...; w], w in R^m. Hence, writing c = V b split into q = n/m blocks
c_1..c_q of length m and cbar = (c_1 + ... + c_q)/q:

    row(b) = V^* [cbar; ...; cbar],   Zb = b - row(b),
    h      = U B^{-*} cbar            (the least-squares solution, Remark 4.1).

Only the invertibility of the stored B is used, so row(b) and Zb are exact for
the stored float64 matrix whatever kappa is (up to the rounding of the block
average). h needs a solve with B, whose eigenvalues are
lambda_p = d + 16 sin^4(pi p / m), p = 0..m-1 (B is symmetric circulant, Eq. 20);
it is computed with the FFT and is accurate to about eps * kappa.

Permutations follow ``workloads.paper_test_matrix``: A[i, pv[c]] = C[pu[i], c],
C = [B|...|B].
"""
from __future__ import annotations

import numpy as np

__all__ = ["project", "apply_A", "kappa_of_B", "eigenvalues_B"]


def eigenvalues_B(m: int, d: float) -> np.ndarray:
    """Eigenvalues of the circulant B of Eq. 20: d + 16 sin^4(pi p / m)."""
    p = np.arange(m)
    return d + 16.0 * np.sin(np.pi * p / m) ** 4


def kappa_of_B(m: int, d: float) -> float:
    """Condition number of B; equals (16 + d)/d for even m (Section 5)."""
    lam = eigenvalues_B(m, d)
    return float(lam.max() / lam.min())


def project(Bblock: np.ndarray, pu: np.ndarray, pv: np.ndarray, Brhs: np.ndarray):
    """(Z, ROW, H) for right-hand sides Brhs (k x n rows)."""
    Brhs = np.atleast_2d(np.asarray(Brhs, np.float64))
    m = Bblock.shape[0]
    k, n = Brhs.shape
    q = n // m
    # c = V b: entry c of [B|...|B]-space reads b at column pv[c] of A.
    c = Brhs[:, pv]                                   # k x n
    cbar = c.reshape(k, q, m).mean(axis=1)            # k x m
    rowc = np.tile(cbar, (1, q))                      # k x n, in C-column order
    row = np.empty_like(Brhs)
    row[:, pv] = rowc                                 # back to A's columns: V^*
    z = Brhs - row
    # h = U B^{-*} cbar; B is symmetric circulant: solve in Fourier space.
    col0 = Bblock[:, 0]
    lam = np.fft.fft(col0)
    w = np.real(np.fft.ifft(np.fft.fft(cbar, axis=1) / lam[None, :], axis=1))  # k x m, B^{-1} cbar
    # A^* h = V^* C^* U^* h; with (U^* h)[pu[i]] = h[i]:  U^* h = w  =>  h[i] = w[pu[i]].
    h = w[:, pu]
    return z, row, h


def apply_A(Bblock: np.ndarray, pu: np.ndarray, pv: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """A z for the rows z of Z (k x n), accumulated in double-double (TwoSum and Dekker's
    TwoProduct) and rounded once: with A[i, pv[c]] = C[pu[i], c], C = [B|...|B],
    (A z)_i = sum_t B[pu[i], t] y_t where y_t = sum_q z[pv[q m + t]] sums the q = n/m
    blocks. O(n k + m^2 k) instead of the dense m n k; Section 5's delta = ||A z||."""
    from .exact import _dd_sum_rows, two_prod, two_sum
    Z = np.atleast_2d(np.asarray(Z, np.float64))
    m = Bblock.shape[0]
    k, n = Z.shape
    q = n // m
    blocks = Z[:, pv].reshape(k, q, m).transpose(0, 2, 1)          # k x m x q
    yh, yl = _dd_sum_rows(blocks, np.zeros_like(blocks))            # k x m, y = yh + yl
    Bp = np.asarray(Bblock, np.float64)[pu, :]                      # row i of A's block: B[pu[i], :]
    p, e = two_prod(Bp[None, :, :], yh[:, None, :])                 # k x m x m
    e = e + Bp[None, :, :] * yl[:, None, :]
    hi, lo = _dd_sum_rows(p, e)
    s, t = two_sum(hi, lo)
    return s + t

