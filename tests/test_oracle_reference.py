"""Pins for oracle.reference (the Householder-QR definition of Zb, row(b), h)."""
import mpmath as mp
import numpy as np
import pytest

import workloads
from oracle import metrics, reference

EPS = np.finfo(np.float64).eps


def mp_project(A, B, dps=60):
    """Brute force in 60-digit arithmetic: h = (A A^*)^{-1} A b, row = A^* h, Z = b - row (Eq. 1)."""
    with mp.workdps(dps):
        Am = mp.matrix(A.tolist())
        G = Am * Am.T
        Z, ROW, H = [], [], []
        for b in np.atleast_2d(B):
            bm = mp.matrix(b.tolist())
            h = mp.lu_solve(G, Am * bm)
            row = Am.T * h
            ROW.append([float(x) for x in row])
            Z.append([float(x) for x in (bm - row)])
            H.append([float(x) for x in h])
    return np.array(Z), np.array(ROW), np.array(H)


def test_textbook_householder_matches_lapack():
    A = workloads.haar_spectrum_matrix(7, 40, 1e-3, 3)
    V, beta, R = reference.householder_qr(A.T)
    q, r = reference.qr_factor(A)
    # same R up to the signs of its rows
    s = np.sign(np.diag(R)) * np.sign(np.diag(r))
    np.testing.assert_allclose(R, s[:, None] * r, rtol=0, atol=1e-13)
    B = workloads.rhs(3, 40, 4)
    y = reference.householder_apply_qt(V, beta, B.T)
    y[7:] = 0.0
    row = reference.householder_apply_q(V, beta, y).T
    np.testing.assert_allclose(row, reference.row_project(A, B), atol=1e-13)


@pytest.mark.parametrize("m,n,kappa", [(4, 12, 1e2), (6, 20, 1e4), (8, 32, 1e6)])
def test_against_extended_precision_brute_force(m, n, kappa):
    A = workloads.haar_spectrum_matrix(m, n, 1.0 / kappa, 10 + m)
    B = workloads.rhs(3, n, 20 + m)
    Z, ROW, H = reference.project(A, B)
    Zm, ROWm, Hm = mp_project(A, B)
    # float64 Householder is accurate to about eps * kappa (Remark 5.1)
    tol = 50 * EPS * kappa
    assert metrics.max_rel_err(Z, Zm) < tol
    assert metrics.max_rel_err(ROW, ROWm) < tol
    assert metrics.max_rel_err(H, Hm) < 50 * EPS * kappa ** 2


def test_square_matrix_has_trivial_null_space():
    A = workloads.haar_spectrum_matrix(9, 9, 1e-2, 5)
    B = workloads.rhs(2, 9, 6)
    Z, ROW, H = reference.project(A, B)
    assert np.max(np.abs(Z)) < 1e-12
    np.testing.assert_allclose(H, np.linalg.solve(A.T, B.T).T, rtol=1e-10, atol=1e-12)


def test_diagonal_block_matrix_zeroes_leading_coordinates():
    m, n = 5, 17
    A = np.zeros((m, n))
    A[np.arange(m), np.arange(m)] = [3.0, -1e-6, 2.5, 1e3, 0.25]
    B = workloads.rhs(3, n, 7)
    Z, ROW, H = reference.project(A, B)
    np.testing.assert_array_equal(Z[:, :m], 0.0 * Z[:, :m])
    np.testing.assert_allclose(Z[:, m:], B[:, m:], rtol=0, atol=1e-15)
    np.testing.assert_allclose(H, B[:, :m] / np.diag(A)[:m][None, :], rtol=1e-14)


def test_orthonormal_rows_closed_form():
    rng = np.random.default_rng(8)
    A = workloads.haar_orthonormal(rng, 30, 6).T       # 6 x 30 with orthonormal rows
    B = workloads.rhs(4, 30, 9)
    Z, ROW, H = reference.project(A, B)
    np.testing.assert_allclose(Z, B - (B @ A.T) @ A, atol=1e-14)
    np.testing.assert_allclose(H, B @ A.T, atol=1e-14)


def test_left_multiplication_leaves_projection_unchanged():
    A = workloads.haar_spectrum_matrix(6, 40, 1e-2, 12)
    M = np.random.default_rng(1).standard_normal((6, 6)) + 3 * np.eye(6)
    B = workloads.rhs(3, 40, 13)
    Z1 = reference.null_project(A, B)
    Z2 = reference.null_project(M @ A, B)
    np.testing.assert_allclose(Z1, Z2, atol=1e-12)


def test_projector_invariants():
    # Section 1: ZZ = Z, Z^* = Z, AZ = 0
    A = workloads.haar_spectrum_matrix(10, 60, 1e-4, 14)
    B = workloads.rhs(5, 60, 15)
    C = workloads.rhs(5, 60, 16)
    Z = reference.null_project(A, B)
    ZZ = reference.null_project(A, Z)
    assert metrics.max_rel_err(ZZ, Z) < 1e-13
    assert np.max(metrics.delta(A, Z)) < 1e-13 * np.linalg.norm(B)
    ZC = reference.null_project(A, C)
    np.testing.assert_allclose(np.sum(Z * C, axis=1), np.sum(B * ZC, axis=1), rtol=1e-12, atol=1e-12)
    H = reference.lstsq(A, B)
    # normal equations of min ||A^* h - b||: A (b - A^* h) = 0
    res = (B - H @ A) @ A.T
    assert np.max(np.abs(res)) < 1e-12
