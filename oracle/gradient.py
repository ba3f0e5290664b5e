"""Gradient of the null-space projection (the adjoint of Eq. 1), from the plain definition.

Test infrastructure only (see ``oracle/__init__.py``).

The paper does not differentiate the projection; this follows from Eq. 1. For a full-rank
A with P = A^*(AA^*)^{-1} (so that Z = I - P A and P^* b = h, the least-squares solution of
Remark 4.1), differentiating (AA^*)^{-1} gives

    dZ = -(Z dA^* P^* + P dA Z).

Hence for L = sum_j <g_j, Z b_j> (B, G: k x n, one right-hand side per row)

    dL/dB = Z G                          (rows Z g_j; Z is symmetric),
    dL/dA = -(H^* (Z G) + W^* (Z B)),    H = lstsq(B), W = lstsq(G)  (rows h_j, w_j).

Every quantity here comes from ``oracle.reference`` (Householder QR of A^*).
"""
from __future__ import annotations

import numpy as np

from . import reference

__all__ = ["loss", "grad"]


def loss(A: np.ndarray, B: np.ndarray, G: np.ndarray) -> float:
    """L = sum_j <g_j, Z b_j>."""
    Z = reference.null_project(A, B)
    return float(np.sum(np.asarray(G, np.float64) * Z))


def grad(A: np.ndarray, B: np.ndarray, G: np.ndarray):
    """(dL/dA, dL/dB) for L = sum_j <g_j, Z b_j>."""
    A = np.asarray(A, np.float64)
    Z, _, H = reference.project(A, B)
    Y, _, W = reference.project(A, G)
    return -(H.T @ Y + W.T @ Z), Y
