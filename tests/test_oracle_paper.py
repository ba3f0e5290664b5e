"""Pins for oracle.paper_method (the algorithm of Section 4) and oracle.theory."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import closed_form, exact, metrics, paper_method, philox, theory

EPS = np.finfo(np.float64).eps


def test_pivoted_qr_properties_and_scipy_agreement():
    M = np.random.default_rng(2).standard_normal((30, 12)) * np.logspace(0, -6, 12)[None, :]
    Q, R, perm = paper_method.pivoted_qr(M)
    np.testing.assert_allclose(M[:, perm], Q @ R, atol=1e-14)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-14)
    assert np.all(np.tril(R, -1) == 0)
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:])
    # column pivoting makes each row diagonally dominant: |R_kk| >= |R_kj|
    assert np.all(d[:, None] >= np.abs(np.triu(R)) - 1e-15)
    Qs, Rs, ps = sla.qr(M, mode="economic", pivoting=True)
    np.testing.assert_array_equal(perm, ps)
    np.testing.assert_allclose(np.abs(R), np.abs(Rs), atol=1e-13)


def _setup(m=12, n=96, kappa=1e6, l=None, seed=4, dist="uniform"):
    A, U, sig, V = workloads.haar_spectrum_matrix(m, n, 1.0 / kappa, seed, return_factors=True)
    l = 4 * m if l is None else l
    G = philox.omega(seed + 50, n, l, dist)
    return A, V, G


def test_gram_columns_equal_preconditioned_gram():
    A, V, G = _setup()
    pc = paper_method.precondition(A, G)
    W = sla.solve_triangular(pc.R.T, A[pc.perm], lower=True)     # P^{-1} A = R^{-*} Pi A
    np.testing.assert_allclose(pc.X, W @ W.T, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(pc.X, pc.X.T, rtol=1e-9, atol=1e-9)
    ev = np.linalg.eigvalsh(0.5 * (pc.X + pc.X.T))
    assert ev.min() > 0
    sv = np.linalg.svd(W, compute_uv=False)
    assert abs(ev.max() / ev.min() / (sv[0] / sv[-1]) ** 2 - 1) < 1e-6
    # P = Pi^* R^*, P^- = Pi^* R^{-1} = (P^*)^{-1} (Eq. 15)
    P = np.empty_like(pc.R)
    P[pc.perm, :] = pc.R.T
    np.testing.assert_allclose(pc.pinv_columns(), np.linalg.inv(P.T), rtol=1e-8, atol=1e-8)
    # S^* = Q R Pi (Eq. 13)
    np.testing.assert_allclose(pc.S.T[:, pc.perm], pc.Q @ pc.R, atol=1e-12 * np.abs(pc.S).max())


def test_lemma_2_4_condition_number_equality():
    # kappa(P^{-1} A) = kappa(V^* G) for any factorisation A G = P Q^*
    A, V, G = _setup(m=10, n=80, kappa=1e3)
    pc = paper_method.precondition(A, G)
    W = sla.solve_triangular(pc.R.T, A[pc.perm], lower=True)
    s1 = np.linalg.svd(W, compute_uv=False)
    s2 = np.linalg.svd(V.T @ G, compute_uv=False)
    assert abs((s1[0] / s1[-1]) / (s2[0] / s2[-1]) - 1) < 1e-9


def test_observation_3_2_statistical_bound():
    # l - m = 4, Gaussian G: kappa(P^{-1}A) <= 10 l except with probability 1e-4 per draw.
    m, n = 6, 60
    l = m + 4
    worst = 0.0
    for seed in range(120):
        A = workloads.haar_spectrum_matrix(m, n, 1e-6, 1000 + seed)
        G = np.random.default_rng(5000 + seed).standard_normal((n, l))
        pc = paper_method.precondition(A, G)
        W = sla.solve_triangular(pc.R.T, A[pc.perm], lower=True)
        s = np.linalg.svd(W, compute_uv=False)
        worst = max(worst, s[0] / s[-1])
    assert worst <= 10 * l


def test_seven_step_apply_matches_exact_within_floor():
    A, V, G = _setup(m=12, n=96, kappa=1e6)
    B = workloads.rhs(4, 96, 33)
    Z, ROW, H, pc = paper_method.project(A, G, B)
    Zx, ROWx, Hx = exact.exact_project(A, B)
    assert metrics.max_rel_err(Z, Zx) < 100 * EPS * 1e6
    assert metrics.max_rel_err(ROW, ROWx) < 100 * EPS * 1e6
    assert metrics.max_rel_err(H, Hx) < 100 * EPS * 1e12
    np.testing.assert_allclose(Z + ROW, B, atol=1e-14)


def test_result_independent_of_sketch_seed_and_size():
    A, V, G = _setup(m=8, n=64, kappa=1e4)
    B = workloads.rhs(3, 64, 34)
    Z1 = paper_method.project(A, G, B)[0]
    Z2 = paper_method.project(A, philox.omega(999, 64, 8 + 4, "rademacher"), B)[0]
    assert metrics.max_rel_err(Z1, Z2) < 100 * EPS * 1e4


def _refine_case():
    A, V, G = _setup(m=12, n=120, kappa=1e9, seed=6)
    B = workloads.rhs(3, 120, 35)
    Z0, _, H0, pc = paper_method.project(A, G, B)
    Zx, _, Hx = exact.exact_project(A, B)
    return A, B, Z0, H0, pc, Zx


def _refine_pin(A, B, Z0, H0, pc, Zx, refine):
    """One pass of Remark 4.3 must (i) cut ||A z|| by at least 1e4 (the unrefined
    residual is about eps * kappa^2 / kappa relative to |A||b|; one pass with float64
    residuals leaves about eps), (ii) lower the error against the exact projection, and
    (iii) keep Z + ROW = B."""
    Z1, ROW1, H1 = refine(A, pc, B, H0, passes=1)
    r0 = np.max(exact.exact_residual(A, Z0))
    r1 = np.max(exact.exact_residual(A, Z1))
    e0 = metrics.max_rel_err(Z0, Zx)
    e1 = metrics.max_rel_err(Z1, Zx)
    return r1 <= 1e-4 * r0 and e1 < e0 and np.allclose(Z1 + ROW1, B, atol=1e-13), (r0, r1, e0, e1)


def test_refinement_contracts_the_residual():
    A, B, Z0, H0, pc, Zx = _refine_case()
    ok, vals = _refine_pin(A, B, Z0, H0, pc, Zx, paper_method.refine)
    assert ok, vals
    assert vals[0] > 1e-9          # the case really starts well above float64 rounding


def test_refinement_planted_mistakes_fail_the_pin():
    """A refine that returns its input, one that skips the update of s, and one that
    forgets to add dh to h each fail the same pin."""
    A, B, Z0, H0, pc, Zx = _refine_case()

    def noop(A_, pc_, B_, H0_, passes=1):
        return Z0, B_ - Z0, H0_

    def no_s_update(A_, pc_, B_, H0_, passes=1):
        H = np.array(H0_, copy=True).T
        S = B_.T - A_.T @ H
        for _ in range(passes):
            H = H + paper_method._middle(pc_, A_ @ S)
        return S.T, B_ - S.T, H.T

    def s_from_stale_h(A_, pc_, B_, H0_, passes=1):
        H = np.array(H0_, copy=True).T
        S = B_.T - A_.T @ H
        for _ in range(passes):
            dH = paper_method._middle(pc_, A_ @ S)
            S = B_.T - A_.T @ H            # h never moves: s is recomputed from h0
        return S.T, B_ - S.T, H.T

    for wrong in (noop, no_s_update, s_from_stale_h):
        ok, vals = _refine_pin(A, B, Z0, H0, pc, Zx, wrong)
        assert not ok, (wrong.__name__, vals)


def test_closed_form_family_and_planted_permutation_mistake(monkeypatch):
    A, Bb, pu, pv = workloads.paper_test_matrix(10, 200, 1e8, 3, return_parts=True)
    G = philox.omega(77, 200, 14)
    B = workloads.rhs(3, 200, 36)
    Zc, ROWc, Hc = closed_form.project(Bb, pu, pv, B)
    Z, ROW, H, pc = paper_method.project(A, G, B)
    assert metrics.max_rel_err(Z, Zc) < 1e-7          # eps * kappa
    # Planted mistake: Pi applied as a scatter instead of a gather in step 2.
    orig = paper_method._middle

    def wrong_middle(pc_, C):
        d = np.empty_like(C)
        d[pc_.perm, :] = C
        e = sla.solve_triangular(pc_.R.T, d, lower=True)
        g = sla.solve_triangular(pc_.R, pc_.Y @ e, lower=False)
        h = np.empty_like(g)
        h[pc_.perm, :] = g
        return h

    monkeypatch.setattr(paper_method, "_middle", wrong_middle)
    Zw = paper_method.project(A, G, B)[0]
    monkeypatch.setattr(paper_method, "_middle", orig)
    assert metrics.max_rel_err(Zw, Zc) > 1e-3


def test_observation_3_2_golden(golden_dir):
    with open(os.path.join(golden_dir, "observation_3_2.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        a = case["alpha_squared"] ** 0.5
        b = case["beta"]
        for m in (2, 10, 100, 4000):
            l = m + g["l_minus_m"]
            assert theory.kappa_bound(l, a, b) <= case["kappa_over_l"] * l
            p_simple = theory.pi_zero_simple(l, m, a, b)
            assert 1.0 - p_simple <= case["failure_probability"]
            # Eq. 10 is a lower bound for Eq. 5
            assert theory.pi_zero(l, m, a, b) >= p_simple - 1e-15


def test_theory_planted_mistake_is_caught():
    # A dropped exponent in Eq. 4 (power 1 instead of l-m+1) breaks the golden claim.
    l, m, b = 104, 100, 3.0
    j = l - m + 1
    wrong = np.e / (j * b) / np.sqrt(2 * np.pi * j)
    assert wrong > 1e-4 >= theory.fail_minus(l, m, b) + theory.fail_plus(l - m + 2, 2.0)


def test_test_family_condition_number_golden(golden_dir):
    with open(os.path.join(golden_dir, "test_family_kappa.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        d = 16.0 / (case["kappa"] - 1.0)
        k = closed_form.kappa_of_B(case["m"], d)
        assert abs(k / case["kappa"] - 1) < 1e-9
        assert abs(k - (16 + d) / d) <= 1e-9 * k
    # the dense build of the family has that condition number (small case)
    A = workloads.paper_test_matrix(12, 48, 1e6, 2)
    s = np.linalg.svd(A, compute_uv=False)
    assert abs(s[0] / s[-1] / 1e6 - 1) < 1e-6
