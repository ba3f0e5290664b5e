"""The exact projection of the stored float64 matrix, to float64 rounding.

Test infrastructure only (see ``oracle/__init__.py``).

Remark 5.1 explains why a float64 computation of Zb is accurate only to about
eps * kappa(A): any backward-stable method computes the projection of a matrix
perturbed at the level eps * ||A||. To measure how close a result is to the
projection of the matrix actually stored, this module runs the refinement of
Remark 4.3 with residuals accumulated in double-double arithmetic (the classical
form of iterative refinement, Dahlquist & Bjorck Sec. 5.7.3), keeping h as an
unevaluated sum h_hi + h_lo:

    h_0 = R^{-1} Q^* b                      (Householder QR A^* = Q R, float64)
    repeat:  s = b - A^*(h_hi + h_lo)       (double-double)
             r = A s                        (double-double, rounded)
             dh = R^{-1} R^{-*} r           (corrected seminormal equations)
             h_hi + h_lo += dh              (double-double)
    Zb = b - A^*(h_hi + h_lo)               (double-double, rounded)

The fixed point satisfies A Zb = 0 to double-double accuracy, so the result is the
exact projection of the stored A rounded to float64, independent of kappa as long
as the correction contracts (eps * kappa(A) well below 1).

Double-double building blocks: TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct
with Veltkamp/Dekker splitting (Dekker, Numer. Math. 18, 1971).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = ["two_sum", "two_prod", "dd_matvec", "exact_project", "exact_residual"]

_SPLITTER = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    """s + e == a + b exactly, s = fl(a + b)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def _split(a):
    c = _SPLITTER * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    """p + e == a * b exactly, p = fl(a * b) (no FMA needed)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _dd_sum_rows(h, l):
    """Pairwise double-double reduction along the last axis of (h + l)."""
    while h.shape[-1] > 1:
        if h.shape[-1] % 2:
            pad = [(0, 0)] * (h.ndim - 1) + [(0, 1)]
            h = np.pad(h, pad)
            l = np.pad(l, pad)
        s, e = two_sum(h[..., 0::2], h[..., 1::2])
        e = e + (l[..., 0::2] + l[..., 1::2])
        h, l = two_sum(s, e)
    return h[..., 0], l[..., 0]


def dd_matvec(M: np.ndarray, xh: np.ndarray, xl: np.ndarray | None = None, block: int = 64):
    """(hi, lo) with hi + lo = M (xh + xl) to double-double accuracy."""
    M = np.asarray(M, np.float64)
    xh = np.asarray(xh, np.float64)
    rows = M.shape[0]
    hi = np.empty(rows)
    lo = np.empty(rows)
    for r0 in range(0, rows, block):
        blk = M[r0:r0 + block]
        p, e = two_prod(blk, xh[None, :])
        if xl is not None:
            e = e + blk * xl[None, :]
        h, l = _dd_sum_rows(p, e)
        hi[r0:r0 + block] = h
        lo[r0:r0 + block] = l
    return hi, lo


def _residual(A, AT, b, hh, hl):
    """(s_hi, s_lo) = b - A^*(hh + hl) in double-double."""
    th, tl = dd_matvec(AT, hh, hl)
    s1, e1 = two_sum(b, -th)
    return two_sum(s1, e1 - tl)


def exact_project(A: np.ndarray, B: np.ndarray, passes: int = 12, factors=None, return_info=False,
                  stop_rel: float = 2.0 ** -70):
    """Exact (Z, ROW, H) for right-hand sides B (k x n rows), rounded to float64.

    Refinement stops once the correction is below ``stop_rel`` times max|h| (checked
    after at least two passes), or after ``passes`` passes; ``return_info`` adds
    the max-norm of the last correction relative to h (the convergence evidence).
    """
    A = np.ascontiguousarray(np.asarray(A, np.float64))
    AT = np.ascontiguousarray(A.T)
    B = np.atleast_2d(np.asarray(B, np.float64))
    if factors is None:
        Q, R = np.linalg.qr(AT, mode="reduced")
    else:
        Q, R = factors
    k, n = B.shape
    m = A.shape[0]
    Z = np.empty((k, n))
    ROW = np.empty((k, n))
    H = np.empty((k, m))
    last = 0.0
    rel = 0.0
    for j in range(k):
        b = B[j]
        hh = sla.solve_triangular(R, Q.T @ b, lower=False)
        hl = np.zeros(m)
        for it in range(passes):
            sh, sl = _residual(A, AT, b, hh, hl)
            rh, rl = dd_matvec(A, sh, sl)
            r = rh + rl
            d = sla.solve_triangular(R, sla.solve_triangular(R.T, r, lower=True), lower=False)
            hh, e = two_sum(hh, d)
            hh, hl = two_sum(hh, hl + e)
            nh = np.max(np.abs(hh))
            rel = float(np.max(np.abs(d)) / nh) if nh > 0 else 0.0
            if it >= 1 and rel <= stop_rel:
                break
        last = max(last, rel)
        sh, sl = _residual(A, AT, b, hh, hl)
        Z[j] = sh + sl
        th, tl = dd_matvec(AT, hh, hl)
        ROW[j] = th + tl
        H[j] = hh + hl
    if return_info:
        return Z, ROW, H, last
    return Z, ROW, H


def exact_residual(A: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """||A z|| for each row z of Z, with A z accumulated in double-double."""
    A = np.asarray(A, np.float64)
    Z = np.atleast_2d(np.asarray(Z, np.float64))
    out = np.empty(Z.shape[0])
    for j in range(Z.shape[0]):
        h, l = dd_matvec(A, Z[j])
        out[j] = np.linalg.norm(h + l)
    return out
