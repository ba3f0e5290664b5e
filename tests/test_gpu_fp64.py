"""GPU parity of the plain float64 form (every kernel on the FP64 pipe) against the oracle.

All calls go through the C ABI (the ctypes binding); the oracle runs on the host."""
import numpy as np
import pytest

import workloads
from oracle import closed_form, exact, metrics, paper_method, philox
from tests.gpu_common import EPS, assert_rows_close, fp64_tol, rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _projector(rt, torch, A, l, k, **kw):
    return rt.Projector(to_dev(torch, A), l_max=l, k_max=k, mode="fp64", **kw)


def ambiguity_allowance(A, seed, n, l, dist):
    """|A| times one 2^-12 step on the Gaussian entries whose rounding a float32 transform
    may decide either way (oracle.philox.gaussian_ambiguous); zero for the exact maps."""
    if dist != "gaussian":
        return 0.0
    amb = philox.gaussian_ambiguous(seed, n, l)
    return np.abs(A) @ (amb / philox.GAUSS_GRID)


@pytest.mark.parametrize("dist", ["uniform", "rademacher", "gaussian"])
@pytest.mark.parametrize("m,n,l", [(64, 2048, 256), (37, 1000, 41), (5, 77, 19)])
def test_sketch_matches_oracle(m, n, l, dist):
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1e-6, 3)
    seed = (1 << 40) + 17
    with _projector(rt, torch, A, l, 1, omega=dist) as P:
        S = P.sketch(seed=seed, l=l).cpu().numpy()
    G = philox.omega(seed, n, l, dist)
    Sref = A @ G
    scale = np.abs(A) @ np.abs(G)
    assert np.all(np.abs(S - Sref) <= 4 * n * EPS * scale + ambiguity_allowance(A, seed, n, l, dist) + 1e-300)


@pytest.mark.parametrize("m,n,l", [(64, 2048, 256), (37, 1000, 41)])
def test_pivoted_qr_and_cholesky_match_oracle(m, n, l):
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1e-4, 4)
    with _projector(rt, torch, A, l, 1) as P:
        S = P.sketch(seed=9, l=l).cpu().numpy()
        P.precondition(seed=9, l=l)
        R, perm, L = P.export_state()
    Q, Rref, pref = paper_method.pivoted_qr(S.T)
    np.testing.assert_array_equal(perm, pref)
    d = np.abs(np.diag(Rref))
    assert np.all(np.abs(R - Rref) <= 1e-11 * d[:, None] + 1e-300)
    # Gram matrix X = P^{-1} A A^* P^{-*} from the GPU's own R and Pi, then Cholesky
    import scipy.linalg as sla
    W = sla.solve_triangular(R.T, A[perm], lower=True)
    Lref = np.linalg.cholesky(W @ W.T)
    assert np.max(np.abs(L - Lref)) <= 1e-10 * np.max(np.abs(Lref))


@pytest.mark.parametrize("m,n,l,k,kappa", [
    (64, 2048, 256, 16, 10.0),      # well conditioned: exposes any arithmetic slip
    (64, 2048, 256, 16, 1e8),       # the small dense configuration
    (37, 1000, 41, 3, 1e5),         # ragged sizes, l = m + 4
    (5, 77, 19, 1, 1e3),            # tiny, one right-hand side
])
def test_apply_matches_exact_oracle(m, n, l, k, kappa):
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(m, n, 1.0 / kappa, 10 + m)
    B = workloads.rhs(k, n, 20 + m)
    Zx, ROWx, Hx = exact.exact_project(A, B)
    with _projector(rt, torch, A, l, k) as P:
        P.precondition(seed=11, l=l)
        Z, ROW, H = P.project(to_dev(torch, B), null=True, row=True, lstsq=True)
        info = P.info()
    assert info["status"] == 0
    tol = fp64_tol(kappa)
    assert_rows_close(Z.cpu().numpy(), Zx, tol, "Z")
    assert_rows_close(ROW.cpu().numpy(), ROWx, tol * np.max(np.linalg.norm(Zx, axis=1) / np.linalg.norm(ROWx, axis=1)),
                      "ROW")
    # h's error lands near eps kappa too (measured 0.5 to 1.3 eps kappa at kappa = 1e8, 1e10)
    assert_rows_close(H.cpu().numpy(), Hx, 16 * tol, "H")


def test_separate_entry_points_agree_and_alias():
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 24, 500, 60, 5
    A = workloads.haar_spectrum_matrix(m, n, 1e-3, 31)
    B = workloads.rhs(k, n, 32)
    with _projector(rt, torch, A, l, k) as P:
        P.precondition(seed=3, l=l)
        Bt = to_dev(torch, B)
        Z, ROW, H = P.project(Bt, null=True, row=True, lstsq=True)
        np.testing.assert_array_equal(P.null_project(Bt).cpu().numpy(), Z.cpu().numpy())
        np.testing.assert_array_equal(P.row_project(Bt).cpu().numpy(), ROW.cpu().numpy())
        np.testing.assert_array_equal(P.lstsq(Bt).cpu().numpy(), H.cpu().numpy())
        P.null_project(Bt, out=Bt)                 # Z aliases B
        np.testing.assert_array_equal(Bt.cpu().numpy(), Z.cpu().numpy())


def test_square_matrix_and_paper_family():
    torch = torch_cuda()
    rt = rt_module()
    A = workloads.haar_spectrum_matrix(48, 48, 1e-3, 40)
    B = workloads.rhs(2, 48, 41)
    with _projector(rt, torch, A, 48, 2) as P:
        P.precondition(seed=1, l=48)
        Z, _, H = P.project(to_dev(torch, B), null=True, lstsq=True)
    assert np.max(np.abs(Z.cpu().numpy())) < 1e-9 * np.max(np.abs(B))
    np.testing.assert_allclose(H.cpu().numpy(), np.linalg.solve(A.T, B.T).T, rtol=1e-8, atol=1e-10)
    # the paper's test family (Eqs. 20-21): exact closed form at any kappa
    A, Bb, pu, pv = workloads.paper_test_matrix(64, 4096, 1e10, 42, return_parts=True)
    B = workloads.rhs(4, 4096, 43)
    Zc, ROWc, _ = closed_form.project(Bb, pu, pv, B)
    with _projector(rt, torch, A, 68, 4) as P:
        P.precondition(seed=2, l=68)
        Z = P.null_project(to_dev(torch, B)).cpu().numpy()
    assert metrics.max_rel_err(Z, Zc) < fp64_tol(1e10)


def test_status_codes():
    torch = torch_cuda()
    rt = rt_module()
    m, n = 16, 200
    A = workloads.haar_spectrum_matrix(m, n, 1e-2, 50)
    B = to_dev(torch, workloads.rhs(2, n, 51))
    P = _projector(rt, torch, A, 64, 2)
    with pytest.raises(rt.RtprojError) as e:
        P.null_project(B)
    assert e.value.code == 2                      # apply before precondition
    with pytest.raises(rt.RtprojError) as e:
        P.precondition(seed=1, l=m - 1)
    assert e.value.code == 1                      # l < m
    P.precondition(seed=1, l=40)
    B3 = to_dev(torch, workloads.rhs(3, n, 52))
    with pytest.raises(TypeError):
        P.null_project(B3)                        # k > k_max: the binding refuses it ...
    Zb = torch.empty_like(B3)
    L = rt.load_library()
    import ctypes
    assert L.rtproj_null_project(P._h, ctypes.c_void_p(B3.data_ptr()), n, 3, ctypes.c_void_p(Zb.data_ptr()),
                                 n) == 1          # ... and so does the C ABI (EINVAL)
    assert L.rtproj_null_project(P._h, ctypes.c_void_p(B3.data_ptr()), n - 1, 2, ctypes.c_void_p(Zb.data_ptr()),
                                 n) == 1          # ldb < n
    P.close()
    Ad = A.copy()
    Ad[5] = Ad[3]                                 # rank deficient
    P = _projector(rt, torch, Ad, 64, 2)
    with pytest.raises(rt.RtprojError) as e:
        P.precondition(seed=1, l=40)
    assert e.value.code in (3, 4)
    P.close()
    An = A.copy()
    An[2, 7] = np.nan
    P = _projector(rt, torch, An, 64, 2)
    with pytest.raises(rt.RtprojError) as e:
        P.precondition(seed=1, l=40)
    assert e.value.code == 5
    P.close()
