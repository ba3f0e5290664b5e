"""The projection layer's gradients on the GPU (NullProject: forward = rtproj_project,
backward = one more apply and rtproj_grad_A), against oracle.gradient (the same adjoint of
Eq. 1 on the Householder-QR definition), central finite differences of the GPU forward, and
the exact invariant dL/dA A^* = 0."""
import numpy as np
import pytest

import workloads
from oracle import gradient
from tests.gpu_common import rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _layer(torch, rt, A, B, G, mode, l):
    from paper_0912_1135_gb300.autograd import null_project
    At = to_dev(torch, A).requires_grad_(True)
    Bt = to_dev(torch, B).requires_grad_(True)
    Z = null_project(At, Bt, seed=5, l=l, mode=mode)
    (Z * to_dev(torch, G)).sum().backward()
    return Z.detach().cpu().numpy(), At.grad.cpu().numpy(), Bt.grad.cpu().numpy()


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_gradients_match_oracle_and_finite_differences(mode):
    """A well-conditioned copy (sigma over [1e-2, 1]): central differences with h = 1e-6 of
    the GPU forward along random unit directions agree with <dL/dA, E> to the differences'
    own accuracy (about 1e-9 relative to ||G|| ||Z|| / h plus h^2 / sigma_min^2)."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, k, l = 16, 512, 8, 64
    A = workloads.haar_spectrum_matrix(m, n, 1e-2, 70)
    B = workloads.rhs(k, n, 71)
    G = workloads.rhs(k, n, 72)
    Z, dA, dB = _layer(torch, rt, A, B, G, mode, l)
    dAx, dBx = gradient.grad(A, B, G)
    assert np.linalg.norm(dA - dAx) <= 1e-10 * np.linalg.norm(dAx)
    assert np.linalg.norm(dB - dBx) <= 1e-10 * np.linalg.norm(dBx)
    assert np.linalg.norm(dA @ A.T) <= 1e-10 * np.linalg.norm(dA) * np.linalg.norm(A)

    def L(X):
        with rt.Projector(to_dev(torch, X), l_max=l, k_max=k, mode=mode) as P:
            P.precondition(seed=5, l=l)
            return float(np.sum(G * P.null_project(to_dev(torch, B)).cpu().numpy()))

    rng = np.random.default_rng(73)
    h = 1e-6
    for _ in range(3):
        E = rng.standard_normal(A.shape)
        E /= np.linalg.norm(E)
        fd = (L(A + h * E) - L(A - h * E)) / (2 * h)
        scale = np.linalg.norm(G) * np.linalg.norm(Z)
        assert abs(fd - np.sum(dA * E)) <= 1e-9 * scale / h + 1e-3 * abs(fd)


def test_projection_layer_at_the_c5_configuration():
    """A 256 x 8192 float32 (sigma over [1e-6, 1]), a batch of 4096 right-hand sides:
    forward and backward through the layer against the float64 oracle gradient of the same
    stored float32 data. Outputs are float32, so the bound is float32 rounding of H, Z G, W
    and Z B (2^-24 relative each), summed over the 4096 terms of the rank-2k product: about
    sqrt(2k) 2^-24 relative to ||dL/dA|| for independent right-hand sides."""
    torch = torch_cuda()
    rt = rt_module()
    m, n, k = 256, 8192, 4096
    A = workloads.haar_spectrum_matrix(m, n, 1e-6, 80).astype(np.float32)
    B = workloads.rhs(k, n, 81, dtype=np.float32)
    G = workloads.rhs(k, n, 82, dtype=np.float32)
    Z, dA, dB = _layer(torch, rt, A, B, G, "mixed", 4 * m)
    assert dA.dtype == np.float32 and dB.dtype == np.float32
    dAx, dBx = gradient.grad(A.astype(np.float64), B.astype(np.float64), G.astype(np.float64))
    tol = 2 * np.sqrt(2 * k) * 2.0 ** -24
    assert np.linalg.norm(dA - dAx) <= tol * np.linalg.norm(dAx)
    assert np.linalg.norm(dB - dBx) <= 4 * 2.0 ** -24 * np.linalg.norm(dBx)
    A64 = A.astype(np.float64)
    assert np.linalg.norm(dA.astype(np.float64) @ A64.T) <= tol * np.linalg.norm(dAx) * np.linalg.norm(A64)
