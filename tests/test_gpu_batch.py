"""Batching: uneven instances in one CUDA-graph step, and one A under a sequence of
interior-point-style column scalings A diag(d_j).

Instances follow the batching configuration's recipe (m log-uniform, n = m times a
log-uniform factor in [4, 64], float32 data, sigma over [1e-4, 1], l = 2m + 32, 32
right-hand sides each) at a handful of sizes. The graph's replay must reproduce the eager
step bit for bit (the same kernels in the same order on the same inputs), and every
instance must match the exact projection of its stored float32 matrix to float32 rounding.
For the scalings, the oracle's input is A * d in float64 -- the same once-rounded products
the device forms -- and its exact projection."""
import numpy as np
import pytest

import workloads
from oracle import exact
from tests.gpu_common import assert_rows_close, rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_uneven_float32_instances_in_one_graph():
    torch = torch_cuda()
    rt_module()
    from paper_0912_1135_gb300.batch import Batch
    sizes = [(16, 64), (40, 400), (64, 4096), (100, 800), (33, 2112), (200, 1600)]
    k = 32
    As = [workloads.haar_spectrum_matrix(m, n, 1e-4, 1000 + i, dtype=np.float32) for i, (m, n) in enumerate(sizes)]
    Bs = [workloads.rhs(k, n, 2000 + i, dtype=np.float32) for i, (m, n) in enumerate(sizes)]
    At = [torch.from_numpy(A).cuda() for A in As]
    Bt = [torch.from_numpy(B).cuda() for B in Bs]
    Z1 = [torch.empty_like(B) for B in Bt]
    Z2 = [torch.full_like(B, float("nan")) for B in Bt]
    bt = Batch(At, [k] * len(sizes), [2 * m + 32 for m, _ in sizes], streams=4)
    seeds = [3000 + i for i in range(len(sizes))]
    bt.step(Bt, seeds, Z1)
    torch.cuda.synchronize()
    bt.capture(Bt, seeds, Z2)
    for Z in Z2:
        Z.fill_(float("nan"))
    bt.replay()
    torch.cuda.synchronize()
    assert bt.statuses() == [0] * len(sizes)
    bt.close()
    for i, (A, B) in enumerate(zip(As, Bs)):
        np.testing.assert_array_equal(Z2[i].cpu().numpy(), Z1[i].cpu().numpy())
        Zx, _, _ = exact.exact_project(A.astype(np.float64), B.astype(np.float64))
        assert_rows_close(Z1[i].cpu().numpy().astype(np.float64), Zx, 4 * 2.0 ** -24, f"Z (instance {i})")


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_interior_point_scalings(mode):
    torch = torch_cuda()
    rt = rt_module()
    m, n, l, k = 64, 4096, 160, 8
    A = workloads.haar_spectrum_matrix(m, n, 1e-3, 1100)
    rng = np.random.default_rng(1101)
    At = to_dev(torch, A)
    tol = 1e-10 if mode == "mixed" else 1e-6
    with rt.Projector(At, l_max=l, k_max=k, mode=mode, scalable=1, refine_passes=4, refine_tol=1e-12) as P:
        for j in range(3):
            d = 10.0 ** rng.uniform(-3, 3, n)                 # log-uniform scalings
            B = workloads.rhs(k, n, 1200 + j)
            P.set_scaling(to_dev(torch, d))
            P.precondition(seed=50 + j, l=l)
            Z = P.null_project(to_dev(torch, B)).cpu().numpy()
            assert P.info()["status"] == 0
            Zx, _, _ = exact.exact_project(A * d[None, :], B)
            assert_rows_close(Z, Zx, tol, f"Z (scaling {j})")
        P.set_scaling(None)                                   # back to A itself
        P.precondition(seed=60, l=l)
        B = workloads.rhs(k, n, 1300)
        Zx, _, _ = exact.exact_project(A, B)
        assert_rows_close(P.null_project(to_dev(torch, B)).cpu().numpy(), Zx, tol, "Z (unscaled)")
