"""Pins for oracle.exact (the exact projection of the stored float64 matrix)."""
import numpy as np
import pytest

import workloads
from oracle import closed_form, exact, metrics, reference
from tests.test_oracle_reference import mp_project


def test_two_sum_two_prod_are_error_free():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000)
    b = rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000)
    from fractions import Fraction
    s, e = exact.two_sum(a, b)
    p, f = exact.two_prod(a, b)
    for i in range(0, 1000, 37):
        assert Fraction(s[i]) + Fraction(e[i]) == Fraction(a[i]) + Fraction(b[i])
        assert Fraction(p[i]) + Fraction(f[i]) == Fraction(a[i]) * Fraction(b[i])


def test_dd_matvec_matches_exact_rational_dot():
    from fractions import Fraction
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, 257)) * 10.0 ** rng.integers(-6, 6, (3, 257))
    x = rng.standard_normal(257)
    hi, lo = exact.dd_matvec(M, x)
    for i in range(3):
        ref = sum(Fraction(M[i, j]) * Fraction(x[j]) for j in range(257))
        err = abs(Fraction(hi[i]) + Fraction(lo[i]) - ref)
        scale = sum(abs(Fraction(M[i, j]) * Fraction(x[j])) for j in range(257))
        assert err <= scale * Fraction(1, 2 ** 95)


@pytest.mark.parametrize("m,n,kappa,seed", [(6, 24, 1e8, 1), (8, 40, 1e12, 3), (16, 64, 1e10, 5)])
def test_matches_extended_precision_brute_force(m, n, kappa, seed):
    A = workloads.haar_spectrum_matrix(m, n, 1.0 / kappa, seed)
    B = workloads.rhs(2, n, 100 + seed)
    Z, ROW, H = exact.exact_project(A, B)
    Zm, ROWm, Hm = mp_project(A, B, dps=80)
    assert metrics.max_rel_err(Z, Zm) < 4e-16
    assert metrics.max_rel_err(ROW, ROWm) < 4e-16
    assert metrics.max_rel_err(H, Hm) < 1e-15


@pytest.mark.parametrize("kappa", [1e4, 1e10, 1e13])
def test_matches_closed_form_of_paper_family(kappa):
    A, Bb, pu, pv = workloads.paper_test_matrix(16, 256, kappa, 7, return_parts=True)
    B = workloads.rhs(3, 256, 8)
    Zc, ROWc, Hc = closed_form.project(Bb, pu, pv, B)
    Z, ROW, H = exact.exact_project(A, B)
    assert metrics.max_rel_err(Z, Zc) < 1e-15
    assert metrics.max_rel_err(ROW, ROWc) < 1e-15
    assert metrics.max_rel_err(H, Hc) < 100 * np.finfo(float).eps * kappa


def test_float64_householder_sits_at_the_eps_kappa_floor():
    # Remark 5.1: a float64 method is meaningful to about eps * kappa; the exact
    # oracle resolves errors well below that floor.
    A = workloads.haar_spectrum_matrix(32, 512, 1e-10, 9)
    B = workloads.rhs(2, 512, 10)
    Zx, _, _ = exact.exact_project(A, B)
    Zq = reference.null_project(A, B)
    e = metrics.max_rel_err(Zq, Zx)
    assert 1e-13 < e < 1e-5
    assert np.max(exact.exact_residual(A, Zx)) < 1e-15 * np.linalg.norm(B)


def test_planted_dropped_error_term_is_caught(monkeypatch):
    # A plausible mistake: TwoProduct without its error term (plain float64 products).
    monkeypatch.setattr(exact, "two_prod", lambda a, b: (a * b, np.zeros_like(a * b)))
    A = workloads.haar_spectrum_matrix(8, 40, 1e-12, 3)
    B = workloads.rhs(1, 40, 103)
    Z, _, _ = exact.exact_project(A, B)
    Zm, _, _ = mp_project(A, B, dps=80)
    assert metrics.max_rel_err(Z, Zm) > 1e-12


def test_paper_family_apply_matches_dense_double_double():
    """closed_form.apply_A (the family's structure, O(n)) against the dense matrix times z
    accumulated by oracle.exact.dd_matvec -- two independent routes to A z."""
    A, Bb, pu, pv = workloads.paper_test_matrix(8, 96, 1e8, 4, return_parts=True)
    Z = workloads.rhs(3, 96, 5)
    got = closed_form.apply_A(Bb, pu, pv, Z)
    for j in range(3):
        h, l = exact.dd_matvec(A, Z[j])
        np.testing.assert_allclose(got[j], h + l, rtol=1e-15, atol=1e-15 * np.abs(A).max() * np.abs(Z[j]).sum())
    # on the family's own null-space projection, A z vanishes to double-double accuracy
    Zc, _, _ = closed_form.project(Bb, pu, pv, Z)
    assert np.max(np.abs(closed_form.apply_A(Bb, pu, pv, Zc))) < 1e-13 * np.abs(A).max()
