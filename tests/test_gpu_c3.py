"""Precision at scale: A 2048 x 262144 float64 (4.3 GB), sigma log-spaced over [1e-12, 1],
sketch size l = 2m + 32 = 4128, applies at k = 1, 16 and 256 right-hand sides.

At kappa = 1e12 the sketch needs six digits so that its own error (2^-48 relative) stays
below the smallest singular value (1e-12 relative), the rank test's threshold must sit below
1/kappa, the refinement's residual products need ten digits (2^-80 kappa ~ 1e-12), and the
correction contracts by about 2^-56 kappa per pass, so refinement runs to a tolerance
(Remark 4.3) instead of one fixed pass. The exact projection of a Haar matrix of
this size is out of the oracle's reach, so Z is checked against the closed form of the
paper's own family (Eqs. 20-21) at the same size and kappa (exact at any kappa), and on the
Haar matrix through ||A z|| accumulated in double-double (oracle.exact.exact_residual) on
sampled right-hand sides and idempotence Z(Zb) = Zb."""
import numpy as np
import pytest

import workloads
from oracle import closed_form, exact, metrics
from tests.gpu_common import assert_rows_close, rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

KEY = "dense_2048x262144"
# six sketch digits (2^-48 relative error, below sigma_min / sigma_max = 1e-12), a rank
# threshold below 1/kappa, ten residual digits, refinement to a tolerance
OPTS = dict(sketch_slices=6, resid_slices=10, refine_passes=4, refine_tol=1e-11, rank_tol=1e-14)
Z_TOL = 1e-10
RESID_TOL = 1e-12


def test_paper_family_at_c3_size_every_k():
    torch = torch_cuda()
    rt = rt_module()
    w = workloads.WORKLOADS[KEY]
    A, Bb, pu, pv = w.paper_family(return_parts=True)
    B = w.rhs()
    Zc, _, _ = closed_form.project(Bb, pu, pv, B[:16])
    with rt.Projector(to_dev(torch, A), l_max=w.l, k_max=w.k, **OPTS) as P:
        del A
        P.precondition(seed=w.seed_omega, l=w.l)
        Bt = to_dev(torch, B)
        for k in (1, 16, 256):
            Z = P.null_project(Bt[:k]).cpu().numpy()
            assert P.info()["status"] == 0
            kk = min(k, 16)
            assert_rows_close(Z[:kk], Zc[:kk], Z_TOL, f"Z (k={k})")


def test_haar_matrix_at_c3_size_every_k():
    torch = torch_cuda()
    rt = rt_module()
    w = workloads.WORKLOADS[KEY]
    A = w.matrix(device="cuda")
    B = w.rhs()
    with rt.Projector(to_dev(torch, A), l_max=w.l, k_max=w.k, **OPTS) as P:
        P.precondition(seed=w.seed_omega, l=w.l)
        Bt = to_dev(torch, B)
        out = {}
        for k in (1, 16, 256):
            out[k] = P.null_project(Bt[:k]).cpu().numpy()
            info = P.info()
            assert info["status"] == 0 and info["passes"] >= 1
        ZZ = P.null_project(to_dev(torch, out[16])).cpu().numpy()
    # one right-hand side gives the same projection whatever else is in the call
    for k in (16, 256):
        assert metrics.max_rel_err(out[k][:1], out[1]) < Z_TOL
    assert metrics.max_rel_err(ZZ, out[16]) < Z_TOL
    nb = np.linalg.norm(B, axis=1)
    for j in (0, 255):
        r = exact.exact_residual(A, out[256][j:j + 1])[0]
        assert r / nb[j] < RESID_TOL                       # ||A||_2 = sigma_1 = 1
