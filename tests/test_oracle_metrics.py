"""Pins for oracle.metrics (the error measures every parity test reads).

Hand-computed 2 x 3 cases: each value below was worked out on paper from the
definitions (per-row 2-norms; Section 5's delta = ||A z||; the normalised residual
||A z|| / (||A||_2 ||b||)), so an axis, transpose or normalisation slip fails them."""
import numpy as np
import pytest

from oracle import metrics

X = np.array([[1.0, 2.0, 2.0], [0.0, 3.0, 4.0]])
XREF = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 5.0]])
A = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])      # ||A||_2 = 2
Z = np.array([[3.0, 4.0, 5.0], [0.0, 0.0, 7.0]])
B = np.array([[1.0, 2.0, 2.0], [0.0, 0.0, 1.0]])      # row norms 3 and 1


def test_rel_err_rows_hand_case():
    # row 0: ||(0, 0, -1)|| / ||(1, 2, 3)|| = 1/sqrt(14); row 1: ||(0, 3, -1)|| / 5 = sqrt(10)/5
    e = metrics.rel_err_rows(X, XREF)
    assert e.shape == (2,)
    np.testing.assert_allclose(e, [1 / np.sqrt(14.0), np.sqrt(10.0) / 5.0], rtol=1e-15)
    assert metrics.max_rel_err(X, XREF) == pytest.approx(np.sqrt(10.0) / 5.0, rel=1e-15)
    # a zero reference row is measured absolutely
    np.testing.assert_allclose(metrics.rel_err_rows([[0.0, 3.0, 4.0]], [[0.0, 0.0, 0.0]]), [5.0])
    # one vector is one row
    assert metrics.max_rel_err([1.0, 2.0, 2.0], [1.0, 2.0, 3.0]) == pytest.approx(1 / np.sqrt(14.0), rel=1e-15)


def test_delta_hand_case():
    # A z_0 = (3, 8): ||.|| = sqrt(73); A z_1 = (0, 0)
    np.testing.assert_allclose(metrics.delta(A, Z), [np.sqrt(73.0), 0.0], rtol=1e-15)


def test_normalised_residual_hand_case():
    # max(sqrt(73) / (2 * 3), 0 / (2 * 1)) with ||A||_2 = 2 from the SVD
    assert metrics.normalised_residual(A, Z, B) == pytest.approx(np.sqrt(73.0) / 6.0, rel=1e-14)
    # a given ||A|| replaces the SVD's
    assert metrics.normalised_residual(A, Z, B, normA=1.0) == pytest.approx(np.sqrt(73.0) / 3.0, rel=1e-15)


def test_planted_axis_mistake_is_caught():
    """Column norms in place of row norms give different numbers on the hand case."""
    wrong = np.linalg.norm(X - XREF, axis=0) / np.linalg.norm(XREF, axis=0)
    assert not np.allclose(np.max(wrong), metrics.max_rel_err(X, XREF))
