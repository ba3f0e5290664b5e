"""GPU parity of the mixed form: digit-sliced tensor-core products (tcgen05) plus refinement.

The sketch test pins the sliced GEMM itself: with s digits of A and the exact digit planes
of G (one for the uniform entries, two for the Gaussian ones), S = A G must equal the exact
product up to the digit truncation bound plus float64 rounding of the result (and, for the
Gaussian entries, one 2^-12 step where the float32 transform may round either way). The
apply tests compare with the exact projection of the stored matrix (oracle.exact)."""
import numpy as np
import pytest

import workloads
from oracle import closed_form, exact, metrics, philox
from tests.gpu_common import EPS, assert_rows_close, fp64_tol, rt_module, to_dev, torch_cuda
from tests.test_gpu_fp64 import ambiguity_allowance

pytestmark = pytest.mark.gpu

# Tolerances of the mixed form: the target of 1e-10 relative error in Zb against the exact
# projection and 1e-12 in ||A Zb|| / (||A|| ||b||).
Z_TOL = 1e-10
RESID_TOL = 1e-12
# h = (A A^*)^{-1} A b: its error is the residual products' error (2^-72 relative to
# |A||s| with nine digits) amplified by ||(A A^*)^{-1} A||, about kappa, relative to |h|
# which is itself about kappa |b|: the refinement's fixed point is accurate to ~2^-72 kappa
H_TOL = 1e-10


def exact_sketch(A, G):
    S = np.empty((A.shape[0], G.shape[1]))
    for j in range(G.shape[1]):
        h, l = exact.dd_matvec(A, G[:, j])
        S[:, j] = h + l
    return S


@pytest.mark.parametrize("omega", ["uniform", "gaussian"])
@pytest.mark.parametrize("s", [1, 2, 4, 8, 10])
@pytest.mark.parametrize("m,n,l", [(64, 2048, 256), (37, 1000, 41)])
def test_sliced_sketch_is_exact_up_to_digit_truncation(m, n, l, s, omega):
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1e-6, 3)
    with rt.Projector(to_dev(torch, A), l_max=l, k_max=1, mode="mixed", sketch_slices=s, omega=omega) as P:
        S = P.sketch(seed=77, l=l).cpu().numpy()
    G = philox.omega(77, n, l, omega)
    Sx = exact_sketch(A, G)
    e = np.frexp(np.max(np.abs(A), axis=1))[1]            # |A_i,:| < 2^{e_i}
    # dropped digits of A (below 2^{e_i - 8s} per entry) times |G| (< 1 uniform, < 5.78
    # Gaussian), and for the two-digit Gaussian plane the dropped pair (s-1, 1), below
    # 2^{e_i + 3 - 8s} per entry: at most 16 n 2^{e_i - 8s} per output in all
    per_entry = 1.0 if omega == "uniform" else 16.0
    amb = ambiguity_allowance(A, 77, n, l, omega)
    bound = n * per_entry * np.ldexp(1.0, e - 8 * s)[:, None] + 2 * EPS * np.abs(Sx) + amb
    assert np.all(np.abs(S - Sx) <= bound)
    if s >= 8:
        # eight digits exceed float64: the result is the exact product, rounded
        assert np.all(np.abs(S - Sx) <= 4 * EPS * (np.abs(A) @ np.abs(G)) + amb)


def _mixed(rt, torch, A, l, k, **kw):
    return rt.Projector(to_dev(torch, A), l_max=l, k_max=k, mode="mixed", **kw)


@pytest.mark.parametrize("m,n,l,k,kappa", [
    (64, 2048, 256, 16, 1e8),       # the small dense configuration
    (64, 2048, 256, 16, 10.0),
    (37, 1000, 41, 3, 1e5),         # ragged sizes, l = m + 4
    (5, 77, 19, 1, 1e3),            # tiny, one right-hand side
])
def test_apply_matches_exact_oracle(m, n, l, k, kappa):
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1.0 / kappa, 10 + m)
    B = workloads.rhs(k, n, 20 + m)
    Zx, ROWx, Hx = exact.exact_project(A, B)
    with _mixed(rt, torch, A, l, k) as P:
        P.precondition(seed=11, l=l)
        Z, ROW, H = P.project(to_dev(torch, B), null=True, row=True, lstsq=True)
        info = P.info()
    assert info["status"] == 0
    Z, ROW, H = Z.cpu().numpy(), ROW.cpu().numpy(), H.cpu().numpy()
    assert_rows_close(Z, Zx, Z_TOL, "Z")
    assert_rows_close(ROW, ROWx, Z_TOL * max(1.0, np.max(np.linalg.norm(Zx, axis=1) / np.linalg.norm(ROWx, axis=1))),
                      "ROW")
    assert_rows_close(H, Hx, H_TOL, "H")
    assert metrics.normalised_residual(A, Z, B) < RESID_TOL


def test_square_matrix():
    """m = n: the null space is {0}, so Z = 0 up to rounding of b against b~, and h solves
    A^* h = b (Section 1). l <= n forces l = m: the square sketch's kappa(V^* G) is heavy
    tailed (Observation 3.2 needs l - m of a few), so the preconditioner contracts less and
    the refinement runs to a tolerance."""
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(48, 48, 1e-3, 40)
    B = workloads.rhs(2, 48, 41)
    with _mixed(rt, torch, A, 48, 2, refine_passes=8, refine_tol=1e-15) as P:
        P.precondition(seed=1, l=48)
        Z, _, H = P.project(to_dev(torch, B), null=True, lstsq=True)
    assert np.max(np.abs(Z.cpu().numpy())) < 1e-13 * np.max(np.abs(B))
    Hx = np.linalg.solve(A.T, B.T).T
    assert_rows_close(H.cpu().numpy(), Hx, 1e3 * EPS * 1e3, "H")   # float64 solve: eps kappa


def test_rank_deficient_matrix_is_reported():
    """Two equal rows: A G is rank deficient and the pivoted QR's last pivot collapses
    (RTPROJ_ERANK), or the Gram matrix is singular (RTPROJ_ENOTSPD)."""
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(16, 200, 1e-2, 50)
    A[5] = A[3]
    with _mixed(rt, torch, A, 40, 2) as P:
        with pytest.raises(rt.RtprojError) as e:
            P.precondition(seed=1, l=40)
        assert e.value.code in (3, 4)


def test_refinement_beats_float64_and_unrefined():
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 64, 4096, 256, 4
    A = workloads.haar_spectrum_matrix(m, n, 1e-10, 60)
    B = workloads.rhs(k, n, 61)
    Zx, _, _ = exact.exact_project(A, B)
    errs = {}
    for name, kw in {"fp64": dict(mode="fp64"), "mixed0": dict(mode="mixed", refine_passes=0),
                     "mixed1": dict(mode="mixed", refine_passes=1), "mixed2": dict(mode="mixed", refine_passes=2)}.items():
        with rt.Projector(to_dev(torch, A), l_max=l, k_max=k, **kw) as P:
            P.precondition(seed=5, l=l)
            errs[name] = metrics.max_rel_err(P.null_project(to_dev(torch, B)).cpu().numpy(), Zx)
    assert errs["mixed1"] < Z_TOL and errs["mixed2"] < Z_TOL, errs
    assert errs["mixed1"] < errs["fp64"] / 10, errs
    assert errs["mixed1"] <= errs["mixed0"], errs


def test_paper_family_closed_form():
    torch = torch_cuda()
    rt = rt_module()
    A, Bb, pu, pv = workloads.paper_test_matrix(64, 4096, 1e10, 42, return_parts=True)
    B = workloads.rhs(4, 4096, 43)
    Zc, ROWc, _ = closed_form.project(Bb, pu, pv, B)
    with _mixed(rt, torch, A, 256, 4) as P:
        P.precondition(seed=2, l=256)
        Z = P.null_project(to_dev(torch, B)).cpu().numpy()
    assert metrics.max_rel_err(Z, Zc) < Z_TOL


def test_long_reduction_over_flat_rows():
    """The paper family at 40 x 10^6: W = P^{-1} A repeats each of its m distinct columns
    n/m times, so the diagonal of X = W W^* is a coherent sum of 10^6 squares near the row
    maximum -- the largest value the sliced product's fixed point has to hold (about
    2^{20+86-8D} for K = 10^6). The preconditioner must still factor and Z match the closed
    form."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l = 40, 10 ** 6, 44
    A, Bb, pu, pv = workloads.paper_test_matrix(m, n, 1e8, 5, return_parts=True)
    B = workloads.rhs(2, n, 6)
    Zc, _, _ = closed_form.project(Bb, pu, pv, B)
    with _mixed(rt, torch, A, l, 2, refine_passes=4, refine_tol=1e-12) as P:
        P.precondition(seed=7, l=l)
        Z = P.null_project(to_dev(torch, B)).cpu().numpy()
        inf = P.info()
    assert inf["status"] == 0 and inf["kappa_pre"] < 100, inf
    assert metrics.max_rel_err(Z, Zc) < Z_TOL


def test_alias_and_entry_points_agree():
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 24, 500, 60, 5
    A = workloads.haar_spectrum_matrix(m, n, 1e-3, 31)
    B = workloads.rhs(k, n, 32)
    with _mixed(rt, torch, A, l, k) as P:
        P.precondition(seed=3, l=l)
        Bt = to_dev(torch, B)
        Z, ROW, H = P.project(Bt, null=True, row=True, lstsq=True)
        np.testing.assert_array_equal(P.null_project(Bt).cpu().numpy(), Z.cpu().numpy())
        np.testing.assert_array_equal(P.row_project(Bt).cpu().numpy(), ROW.cpu().numpy())
        np.testing.assert_array_equal(P.lstsq(Bt).cpu().numpy(), H.cpu().numpy())
        P.null_project(Bt, out=Bt)
        np.testing.assert_array_equal(Bt.cpu().numpy(), Z.cpu().numpy())


@pytest.mark.parametrize("m,n,l,k", [(64, 2048, 256, 16), (37, 1000, 41, 3)])
def test_pipelined_and_synchronous_sliced_gemm_agree_bitwise(m, n, l, k, monkeypatch):
    """Both tensor-core kernels form exact level sums, so their results are identical bit
    for bit: the TMA-pipelined kernel (default) against the synchronous cp.async one
    (RTPROJ_SYNC_GEMM=1)."""
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1e-9, 70)
    B = workloads.rhs(k, n, 71)
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("RTPROJ_SYNC_GEMM", flag)
        with _mixed(rt, torch, A, l, k) as P:
            S = P.sketch(seed=5, l=l).cpu().numpy()
            P.precondition(seed=5, l=l)
            Z, ROW, H = P.project(to_dev(torch, B), null=True, row=True, lstsq=True)
            out[flag] = (S, Z.cpu().numpy(), ROW.cpu().numpy(), H.cpu().numpy())
    for a, b in zip(out["0"], out["1"]):
        np.testing.assert_array_equal(a, b)


def test_nonfinite_entry_of_a_is_reported_by_precondition():
    """A is sliced once, at create; a non-finite entry found there makes precondition
    return RTPROJ_ENONFINITE without reading A again."""
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(37, 1000, 1e-3, 5)
    A[11, 503] = np.inf
    with _mixed(rt, torch, A, 41, 2) as P:
        with pytest.raises(rt.RtprojError) as e:
            P.precondition(seed=1, l=41)
        assert e.value.code == 5


@pytest.mark.parametrize("m,n,l,form", [(64, 2048, 256, 1), (37, 1000, 41, 1), (512, 8192, 516, 1),
                                         (64, 2048, 256, 0), (37, 1000, 41, 0), (512, 8192, 516, 0),
                                         (2048, 8192, 4128, 0)])
def test_float_float_qr_is_a_valid_pivoted_qr(m, n, l, form):
    """The mixed form's float-float QRs (qr_form 0: the whole grid, columns in shared memory
    or, at 2048 x 4128, in global memory; 1: one cluster), checked by properties that do not
    depend on how near-ties between pivots resolve: R^* R equals the Gram matrix of the
    permuted S^* (S^* Pi = Q R with orthonormal Q) to float-float accuracy, R is upper
    triangular, and every diagonal entry dominates the trailing part of its row's columns
    (the column-pivoting property: |R_jj|^2 >= sum_{i >= j} R_ic^2 for c > j)."""
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1e-8, 80 + m)
    with _mixed(rt, torch, A, l, 1, qr_form=form) as P:
        S = P.sketch(seed=21, l=l).cpu().numpy()
        P.precondition(seed=21, l=l)
        R, perm, _ = P.export_state()
    assert sorted(perm) == list(range(m))
    assert np.all(np.tril(R, -1) == 0)
    Sp = S[perm]                                   # rows of S = columns of S^*, permuted
    G = Sp @ Sp.T
    assert np.max(np.abs(R.T @ R - G)) <= 32 * l * 2.0 ** -48 * np.max(np.abs(G))
    tail = np.cumsum((R ** 2)[::-1], axis=0)[::-1]          # tail[j, c] = sum_{i >= j} R_ic^2
    for j in range(m - 1):
        assert R[j, j] ** 2 >= (1 - 1e-6) * np.max(tail[j, j + 1:])


@pytest.mark.parametrize("form", [0, 1, 2])
def test_float_float_qr_hands_a_wide_range_to_the_float64_kernel(form):
    """Rows of A scaled by 2^0 .. 2^-100 (the row space, hence Z, is unchanged): the columns
    of S^* then span 2^100 in norm, their squares 2^200 -- beyond float-float's range -- so
    the float-float QR (grid or cluster) must hand the factorization to the float64 kernel,
    and the projection must still be that of the unscaled matrix."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 64, 2048, 256, 3
    A = workloads.haar_spectrum_matrix(m, n, 1e-3, 91)
    B = workloads.rhs(k, n, 92)
    Zx, _, _ = exact.exact_project(A, B)
    As = A * (2.0 ** (-100.0 * np.arange(m) / (m - 1)))[:, None]
    # R_mm / R_11 is about 2^-100 kappa^-1 here by construction, so the rank test is opened
    with _mixed(rt, torch, As, l, k, qr_form=form, refine_passes=4, refine_tol=1e-13, rank_tol=1e-300) as P:
        P.precondition(seed=93, l=l)
        Z = P.null_project(to_dev(torch, B)).cpu().numpy()
        assert P.info()["status"] == 0
    assert_rows_close(Z, Zx, Z_TOL, f"Z (qr_form={form})")


def test_qr_forms_give_the_same_projection():
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 64, 4096, 256, 4
    A = workloads.haar_spectrum_matrix(m, n, 1e-10, 85)
    B = workloads.rhs(k, n, 86)
    Zx, _, _ = exact.exact_project(A, B)
    for form in (0, 1, 2):
        with _mixed(rt, torch, A, l, k, qr_form=form) as P:
            P.precondition(seed=5, l=l)
            assert P.info()["kappa_R"] > 1e8                 # rank revealing: R_11 / R_mm ~ kappa
            assert_rows_close(P.null_project(to_dev(torch, B)).cpu().numpy(), Zx, Z_TOL, f"Z (qr_form={form})")
