"""The sparse operator form (rtproj_create_sparse): the paper's Section 5 test matrix of
Eq. 21 in compressed sparse row form, and its sum with the rank-10 term of Eq. 22,
against the closed-form projection of the family (oracle.closed_form, exact for the stored
matrix at any kappa), the double-double oracle (oracle.exact) on the dense sum, and the
dense float64 form's sketch of the same matrix."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import closed_form, exact
from tests.gpu_common import EPS, assert_rows_close, rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _csr_dev(torch, rp, ci, v):
    return to_dev(torch, rp), to_dev(torch, ci), to_dev(torch, v)


def _unit_rhs(k, n, seed):
    B = workloads.rhs(k, n, seed)
    return B / np.linalg.norm(B, axis=1, keepdims=True)


@pytest.mark.parametrize("m,n,l,kappa", [(64, 4096, 68, 1e8), (64, 4096, 256, 1e12), (37, 1480, 41, 1e6),
                                         (200, 100000, 204, 1e10)])
def test_sparse_family_matches_closed_form(m, n, l, kappa):
    """Every product with A in the apply is summed in double-double, so refinement reaches
    the projection of the stored matrix to a few float64 roundings whatever kappa is:
    Z within 64 eps of the closed form (relative to ||b||, element-wise as well); h within
    eps kappa (the closed form's own accuracy for h); ||A z|| / ||b|| and the second
    projection's change at the same level."""
    torch = torch_cuda()
    rt = rt_module()
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, kappa, 7)
    B = _unit_rhs(8, n, 8)
    Zc, ROWc, Hc = closed_form.project(b, pu, pv, B)
    with rt.SparseProjector(*_csr_dev(torch, rp, ci, v), n, l_max=l, k_max=8, refine_passes=8,
                            refine_tol=1e-15) as P:
        P.precondition(seed=9, l=l)
        Z, ROW, H = P.project(to_dev(torch, B), null=True, row=True, lstsq=True)
        inf = P.info()
        ZZ = P.null_project(Z.clone()).cpu().numpy()
        Z, ROW, H = Z.cpu().numpy(), ROW.cpu().numpy(), H.cpu().numpy()
    assert inf["status"] == 0 and inf["passes"] >= 1, inf
    assert_rows_close(Z, Zc, 64 * EPS / np.min(np.linalg.norm(Zc, axis=1)), "Z")
    assert_rows_close(ROW, ROWc, 64 * EPS / np.min(np.linalg.norm(ROWc, axis=1)), "ROW")
    assert np.max(np.linalg.norm(H - Hc, axis=1) / np.linalg.norm(Hc, axis=1)) <= 16 * EPS * kappa
    delta = np.max(np.linalg.norm(closed_form.apply_A(b, pu, pv, Z), axis=1))
    assert delta <= 64 * EPS * np.linalg.norm(b, 2) * np.sqrt(n / m), delta
    assert np.max(np.linalg.norm(Z - ZZ, axis=1)) <= 64 * EPS


def test_sparse_low_rank_sum_matches_exact_oracle():
    """A = S + E F / sqrt(m n) (Eq. 22), the rank-10 part kept as factors: against the
    double-double oracle on the dense sum formed in float64 (which differs from the
    operator by one rounding per entry, so the bound is eps times the sum's condition
    number, floored at 1e3)."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, kappa = 64, 4096, 256, 1e4
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, kappa, 11)
    U, V = workloads.paper_low_rank(m, n, 12)
    A = workloads.paper_test_matrix(m, n, kappa, 11) + U @ V
    B = _unit_rhs(6, n, 13)
    Zx, ROWx, Hx = exact.exact_project(A, B)
    kap = np.linalg.cond(A)
    with rt.SparseProjector(*_csr_dev(torch, rp, ci, v), n, U=to_dev(torch, U), V=to_dev(torch, V), l_max=l,
                            k_max=6, refine_passes=6, refine_tol=1e-15) as P:
        P.precondition(seed=14, l=l)
        Z, _, H = P.project(to_dev(torch, B), null=True, lstsq=True)
        inf = P.info()
        Z, H = Z.cpu().numpy(), H.cpu().numpy()
    assert inf["status"] == 0, inf
    assert abs(inf["norm_A"] - np.linalg.norm(A)) <= 1e-13 * np.linalg.norm(A)
    assert_rows_close(Z, Zx, 64 * EPS * max(kap, 1e3), "Z")
    assert np.max(np.linalg.norm(H - Hx, axis=1) / np.linalg.norm(Hx, axis=1)) <= 64 * EPS * kap ** 2


@pytest.mark.parametrize("dist", ["uniform", "rademacher", "gaussian"])
def test_sparse_sketch_matches_dense_form(dist):
    """S = A G of the sparse form and of the dense float64 form of the same matrix (same
    seed, so the same G): equal to float64 rounding of the sums, entry by entry."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l = 40, 2000, 77
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, 1e6, 21)
    U, V = workloads.paper_low_rank(m, n, 22, r=3)
    A = workloads.paper_test_matrix(m, n, 1e6, 21) + U @ V
    with rt.SparseProjector(*_csr_dev(torch, rp, ci, v), n, U=to_dev(torch, U), V=to_dev(torch, V), l_max=l,
                            omega=dist) as P:
        Ss = P.sketch(23, l).cpu().numpy()
    with rt.Projector(to_dev(torch, A), l_max=l, mode="fp64", omega=dist) as P:
        Sd = P.sketch(23, l).cpu().numpy()
    G = rt.generate_omega(23, n, l, dist).cpu().numpy()
    bound = 64 * EPS * (np.abs(A) @ np.abs(G))
    assert np.all(np.abs(Ss - Sd) <= bound)


def test_sparse_unsorted_and_duplicate_entries():
    """Entries in any order within a row, and an entry given as two halves (exactly
    representable, so the stored matrix is unchanged): the same projection as the sorted
    matrix, to rounding."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, kappa = 32, 1024, 64, 1e6
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, kappa, 31)
    rng = np.random.default_rng(32)
    rows_ci, rows_v = [], []
    for i in range(m):
        c, x = ci[rp[i]:rp[i + 1]].copy(), v[rp[i]:rp[i + 1]].copy()
        p = rng.permutation(len(c))
        c, x = c[p], x[p]
        c = np.concatenate([c, c[:1]])            # split the first entry in two halves
        x = np.concatenate([x, x[:1] / 2])
        x[0] /= 2
        rows_ci.append(c)
        rows_v.append(x)
    rp2 = np.concatenate([[0], np.cumsum([len(c) for c in rows_ci])]).astype(np.int64)
    ci2, v2 = np.concatenate(rows_ci).astype(np.int32), np.concatenate(rows_v)
    B = _unit_rhs(4, n, 33)
    Zc, _, _ = closed_form.project(b, pu, pv, B)
    with rt.SparseProjector(*_csr_dev(torch, rp2, ci2, v2), n, l_max=l, k_max=4, refine_passes=8,
                            refine_tol=1e-15) as P:
        P.precondition(seed=34, l=l)
        Z = P.null_project(to_dev(torch, B)).cpu().numpy()
    assert_rows_close(Z, Zc, 64 * EPS / np.min(np.linalg.norm(Zc, axis=1)), "Z")


def test_sparse_invalid_inputs_are_refused():
    """Malformed row pointers, a column index out of range and a non-finite value are
    refused at create (RTPROJ_EINVAL, RTPROJ_EINVAL, RTPROJ_ENONFINITE); an empty row makes
    A rank deficient (RTPROJ_ERANK or RTPROJ_ENOTSPD at precondition); a sparse handle has
    no column scaling (RTPROJ_EUNSUPPORTED)."""
    torch = torch_cuda()
    rt = rt_module()
    m, n = 16, 256
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, 1e4, 41)
    bad_rp = rp.copy()
    bad_rp[5] = bad_rp[6] + 1                     # decreasing
    with pytest.raises(rt.RtprojError) as e:
        rt.SparseProjector(*_csr_dev(torch, bad_rp, ci, v), n)
    assert e.value.code == 1
    bad_ci = ci.copy()
    bad_ci[17] = n                                # out of range
    with pytest.raises(rt.RtprojError) as e:
        rt.SparseProjector(*_csr_dev(torch, rp, bad_ci, v), n)
    assert e.value.code == 1
    bad_v = v.copy()
    bad_v[3] = np.inf
    with pytest.raises(rt.RtprojError) as e:
        rt.SparseProjector(*_csr_dev(torch, rp, ci, bad_v), n)
    assert e.value.code == 5
    # row 3 emptied: its entries removed
    keep = np.ones(len(ci), bool)
    keep[rp[3]:rp[4]] = False
    rp3 = np.concatenate([[0], np.cumsum(np.diff(rp) * (np.arange(m) != 3))]).astype(np.int64)
    with rt.SparseProjector(*_csr_dev(torch, rp3, ci[keep], v[keep]), n, l_max=4 * m) as P:
        with pytest.raises(rt.RtprojError) as e:
            P.precondition(seed=42, l=4 * m)
        assert e.value.code in (3, 4)
        with pytest.raises(rt.RtprojError) as e:
            P.set_scaling(None)
        assert e.value.code == 9
    # the C ABI refuses float32 and column scaling for a sparse A
    L = rt.load_library()
    o = rt.make_opts("fp64")
    o.dtype = 1
    h = ctypes.c_void_p()
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda:0")
    rpd, cid, vd = _csr_dev(torch, rp, ci, v)
    assert L.rtproj_create_sparse(ctypes.byref(h), m, n, len(v), ctypes.c_void_p(rpd.data_ptr()),
                                  ctypes.c_void_p(cid.data_ptr()), ctypes.c_void_p(vd.data_ptr()), 0, None, None,
                                  m, 1, ctypes.c_void_p(ws.data_ptr()), 1 << 20, None, ctypes.byref(o)) == 9
