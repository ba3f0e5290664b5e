"""The C ABI's boundary features on the GPU: the test matrix G itself (step a1), the
bounded grid-exchange waits (RTPROJ_ETIMEOUT and recovery on the same handle), float32
inputs, ordering against a caller's stream, refinement to a tolerance (Remark 4.3), the
residual report, and Observation 3.2 on the GPU's own R and Pi."""
import ctypes

import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import exact, metrics, philox
from tests.gpu_common import EPS, assert_rows_close, rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

Z_TOL = 1e-10


@pytest.mark.parametrize("dist", ["uniform", "rademacher", "gaussian"])
def test_generated_omega_matches_oracle(dist):
    """Bit for bit, except for Gaussian entries the oracle marks as within float32's error
    of a rounding midpoint; those differ by at most one 2^-12 step."""
    torch = torch_cuda()
    rt = rt_module()
    seed, n, l = (3 << 33) + 5, 4101, 37                 # ragged: n not a multiple of 16
    G = rt.generate_omega(seed, n, l, dist).cpu().numpy()
    Gx = philox.omega(seed, n, l, dist)
    if dist != "gaussian":
        np.testing.assert_array_equal(G, Gx)
        return
    amb = philox.gaussian_ambiguous(seed, n, l)
    np.testing.assert_array_equal(G[~amb], Gx[~amb])
    d = np.abs(G[amb] - Gx[amb])
    assert np.all((d == 0) | (d == 1.0 / philox.GAUSS_GRID))
    assert amb.mean() < 0.01


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_spin_limit_expiry_is_reported_and_the_handle_recovers(mode):
    """A spin limit of one cycle makes the pivoted QR's grid exchange give up (the wait is a
    plain global-memory poll; every CTA returns): precondition reports RTPROJ_ETIMEOUT. After
    clearing the status and restoring the limit, the same handle preconditions and projects
    correctly."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 64, 2048, 256, 4
    A = workloads.haar_spectrum_matrix(m, n, 1e-6, 90)
    B = workloads.rhs(k, n, 91)
    with rt.Projector(to_dev(torch, A), l_max=l, k_max=k, mode=mode, spin_limit_cycles=1) as P:
        with pytest.raises(rt.RtprojError) as e:
            P.precondition(seed=3, l=l)
        assert e.value.code == 6                          # RTPROJ_ETIMEOUT
        P.clear_status()
        P.set_spin_limit(4_000_000_000)
        P.precondition(seed=3, l=l)
        Z = P.null_project(to_dev(torch, B)).cpu().numpy()
        assert P.info()["status"] == 0
    Zx, _, _ = exact.exact_project(A, B)
    tol = Z_TOL if mode == "mixed" else 1e-7
    assert_rows_close(Z, Zx, tol, "Z")


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_float32_inputs_and_outputs(mode):
    """float32 A and B are widened exactly; the result is the projection of the stored
    float32 matrix, rounded once to float32."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 32, 1500, 132, 5
    A32 = workloads.haar_spectrum_matrix(m, n, 1e-4, 92).astype(np.float32)
    B32 = workloads.rhs(k, n, 93).astype(np.float32)
    Zx, ROWx, Hx = exact.exact_project(A32.astype(np.float64), B32.astype(np.float64))
    with rt.Projector(torch.from_numpy(A32).cuda(), l_max=l, k_max=k, mode=mode) as P:
        P.precondition(seed=4, l=l)
        Z, ROW, H = P.project(torch.from_numpy(B32).cuda(), null=True, row=True, lstsq=True)
    assert Z.dtype == torch.float32 and ROW.dtype == torch.float32 and H.dtype == torch.float32
    # float32 rounding of the output (2^-24 relative per entry) dominates both forms here
    tol = 4 * 2.0 ** -24 * (1.0 if mode == "mixed" else 16.0)
    assert_rows_close(Z.cpu().numpy().astype(np.float64), Zx, tol, "Z")
    assert_rows_close(ROW.cpu().numpy().astype(np.float64), ROWx, tol * 4, "ROW")
    assert_rows_close(H.cpu().numpy().astype(np.float64), Hx, tol * (1.0 if mode == "mixed" else 1e4), "H")


def test_binding_orders_a_non_default_handle_stream():
    """The handle runs on its own stream; B is produced on the caller's stream just before
    the call and Z is read on the caller's stream right after it."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 32, 4096, 128, 8
    A = workloads.haar_spectrum_matrix(m, n, 1e-5, 94)
    B = workloads.rhs(k, n, 95)
    Zx, _, _ = exact.exact_project(A, B)
    side = torch.cuda.Stream()
    with rt.Projector(to_dev(torch, A), l_max=l, k_max=k, stream=side) as P:
        P.precondition(seed=5, l=l)
        for _ in range(3):
            Bt = torch.zeros((k, n), dtype=torch.float64, device="cuda")
            torch.cuda._sleep(2_000_000)                 # keep the caller's stream busy ...
            Bt.copy_(to_dev(torch, B))                   # ... so B is written late on it
            Z = P.null_project(Bt) * 1.0                  # consumed on the caller's stream
            del Bt
            assert_rows_close(Z.cpu().numpy(), Zx, Z_TOL, "Z")


def test_refinement_to_a_tolerance_and_the_residual_report():
    """refine_tol stops the refinement once every correction is small (Remark 4.3); the
    report gives the passes run, the residual ||A s|| / (||A||_F ||b||) that entered the last
    pass (checked against the oracle's) and the size of the last correction."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 64, 4096, 256, 4
    A = workloads.haar_spectrum_matrix(m, n, 1e-10, 96)
    B = workloads.rhs(k, n, 97)
    Zx, _, _ = exact.exact_project(A, B)
    At, Bt = to_dev(torch, A), to_dev(torch, B)
    infos = {}
    # the tolerance sits above the refinement's fixed point, ~2^-72 kappa in h (1e-12 here)
    for name, kw in {"fixed2": dict(refine_passes=2), "tol": dict(refine_passes=8, refine_tol=1e-9),
                     "none": dict(refine_passes=0)}.items():
        with rt.Projector(At, l_max=l, k_max=k, **kw) as P:
            P.precondition(seed=6, l=l)
            Z = P.null_project(Bt).cpu().numpy()
            infos[name] = (P.info(), metrics.max_rel_err(Z, Zx))
    inf2, e2 = infos["fixed2"]
    inft, et = infos["tol"]
    inf0, _ = infos["none"]
    assert inf2["passes"] == 2 and e2 < Z_TOL
    assert 1 <= inft["passes"] < 8 and inft["dh_rel"] <= 1e-9 and et < Z_TOL
    assert inf0["passes"] == 0 and inf0["resid_rel"] == 0.0
    # the first pass's residual is that of the unrefined projection s = b - A^* h0
    with rt.Projector(At, l_max=l, k_max=k, refine_passes=1) as P:
        P.precondition(seed=6, l=l)
        Z0 = P.project(Bt, null=True)[0]
        inf1 = P.info()
    with rt.Projector(At, l_max=l, k_max=k, refine_passes=0) as P:
        P.precondition(seed=6, l=l)
        S0 = P.null_project(Bt).cpu().numpy()
    ref = np.max(exact.exact_residual(A, S0) / (np.linalg.norm(A) * np.linalg.norm(B, axis=1)))
    assert abs(inf1["resid_rel"] / ref - 1) < 1e-6
    assert inf1["kappa_R"] > 1e8 and 1 <= inf1["kappa_pre"] < 1e3
    assert abs(inf1["norm_A"] / np.linalg.norm(A) - 1) < 1e-13


def test_observation_3_2_on_the_gpu_factorization():
    """l = m + 4, Gaussian G: kappa(P^{-1} A) from the GPU's R and Pi stays below 10 l for
    every one of 100 seeds (Observation 3.2: probability of failure below 1e-4 per draw)."""
    torch = torch_cuda()
    rt = rt_module()
    m, n = 24, 600
    l = m + 4
    A = workloads.haar_spectrum_matrix(m, n, 1e-6, 98)
    worst = 0.0
    with rt.Projector(to_dev(torch, A), l_max=l, k_max=1, mode="fp64", omega="gaussian") as P:
        for seed in range(100):
            P.precondition(seed=7000 + seed, l=l)
            R, perm, _ = P.export_state()
            W = sla.solve_triangular(R.T, A[perm], lower=True)      # P^{-1} A = R^{-*} Pi A
            s = np.linalg.svd(W, compute_uv=False)
            worst = max(worst, s[0] / s[-1])
    assert worst <= 10 * l, worst
