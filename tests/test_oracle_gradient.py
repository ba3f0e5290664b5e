"""Pins for oracle.gradient (the adjoint of Eq. 1).

Central finite differences of the plain definition (oracle.reference) along random unit
directions, on a well-conditioned A (sigma over [1e-2, 1]) so that the difference quotient
is in its linear regime; the exact invariants dL/dA A^* = 0 (Z(MA) = Z(A) for every
invertible M, so no change of A inside its row space moves L) and <dL/dB, c> = <G, Z c>;
and a planted dropped term that the differences catch."""
import numpy as np
import pytest

import workloads
from oracle import gradient, reference


def _case(m=6, n=40, k=3, seed=11):
    A = workloads.haar_spectrum_matrix(m, n, 1e-2, seed)
    B = workloads.rhs(k, n, seed + 1)
    G = workloads.rhs(k, n, seed + 2)
    return A, B, G


def _fd_dir(f, X, E, h):
    return (f(X + h * E) - f(X - h * E)) / (2 * h)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_gradient_matches_central_differences(seed):
    A, B, G = _case(seed=seed)
    dA, dB = gradient.grad(A, B, G)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        E = rng.standard_normal(A.shape)
        E /= np.linalg.norm(E)
        fd = _fd_dir(lambda X: gradient.loss(X, B, G), A, E, 1e-6)
        assert abs(fd - np.sum(dA * E)) <= 1e-7 * max(1.0, abs(fd))
        F = rng.standard_normal(B.shape)
        F /= np.linalg.norm(F)
        fdb = _fd_dir(lambda X: gradient.loss(A, X, G), B, F, 1e-6)
        assert abs(fdb - np.sum(dB * F)) <= 1e-8 * max(1.0, abs(fdb))


def test_gradient_invariants():
    A, B, G = _case(m=8, n=50, k=4, seed=21)
    dA, dB = gradient.grad(A, B, G)
    # row-space moves of A leave Z unchanged: dL/dA A^* = 0
    assert np.linalg.norm(dA @ A.T) <= 1e-12 * np.linalg.norm(dA) * np.linalg.norm(A)
    # dL/dB = Z G and Z is a symmetric projector: <Z g, c> = <g, Z c>, Z(Z g) = Z g
    C = workloads.rhs(4, 50, 22)
    np.testing.assert_allclose(np.sum(dB * C), np.sum(G * reference.null_project(A, C)), rtol=1e-12)
    np.testing.assert_allclose(reference.null_project(A, dB), dB, atol=1e-13)


def test_planted_dropped_term_is_caught():
    """Without the w z^* term (only h (Z g)^*) the gradient misses the differences."""
    A, B, G = _case(seed=31)
    Z, _, H = reference.project(A, B)
    Y, _, W = reference.project(A, G)
    wrong = -(H.T @ Y)
    E = np.random.default_rng(3).standard_normal(A.shape)
    E /= np.linalg.norm(E)
    fd = _fd_dir(lambda X: gradient.loss(X, B, G), A, E, 1e-6)
    assert abs(fd - np.sum(wrong * E)) > 1e-3 * max(1.0, abs(fd))
