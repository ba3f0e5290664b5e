"""Error measures used to report results.

Test infrastructure only (see ``oracle/__init__.py``).

Section 5 (the table headings) measures a computed projection z of a unit b by
  delta   = ||A z||            (how well A annihilates the projection), and
  epsilon = ||z - Z z||        (idempotence: z against its own projection),
each the maximum over the right-hand sides, and reports both divided by kappa.
For comparison against a reference the relative error per right-hand side is
||z - z_ref|| / ||z_ref||, reported as the maximum over the rows.
"""
from __future__ import annotations

import numpy as np

__all__ = ["rel_err_rows", "max_rel_err", "delta", "normalised_residual"]


def rel_err_rows(X: np.ndarray, Xref: np.ndarray) -> np.ndarray:
    X = np.atleast_2d(np.asarray(X, np.float64))
    Xref = np.atleast_2d(np.asarray(Xref, np.float64))
    num = np.linalg.norm(X - Xref, axis=1)
    den = np.linalg.norm(Xref, axis=1)
    den = np.where(den == 0, 1.0, den)
    return num / den


def max_rel_err(X, Xref) -> float:
    return float(np.max(rel_err_rows(X, Xref)))


def delta(A: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """||A z|| for each row z (float64 products)."""
    return np.linalg.norm(np.atleast_2d(Z) @ np.asarray(A, np.float64).T, axis=1)


def normalised_residual(A: np.ndarray, Z: np.ndarray, B: np.ndarray, normA: float | None = None) -> float:
    """max over rows of ||A z|| / (||A||_2 ||b||)."""
    A = np.asarray(A, np.float64)
    if normA is None:
        normA = float(np.linalg.norm(A, 2))
    nb = np.linalg.norm(np.atleast_2d(B), axis=1)
    return float(np.max(delta(A, Z) / (normA * np.where(nb == 0, 1.0, nb))))
