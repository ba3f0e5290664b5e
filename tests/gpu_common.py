"""Helpers shared by the GPU tests (which call the library through its C ABI)."""
import numpy as np
import pytest

EPS = np.finfo(np.float64).eps


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rt_module():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0912_1135_gb300 as rt
    return rt


def to_dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def fp64_tol(kappa: float, m: int) -> float:
    """Relative error allowed for the plain float64 form against the exact projection.

    Remark 5.1: a float64 computation of Zb is meaningful to about eps * kappa. The
    computed products c = A b and A^* h carry errors of order eps * sqrt(n) |A||b|;
    amplified by the preconditioned solve they give ~ eps * kappa * sqrt(m) in Zb.
    A factor 64 covers the constants measured on the oracle."""
    return 64.0 * EPS * max(kappa, 10.0) * np.sqrt(m)
