"""Helpers shared by the GPU tests (which call the library through its C ABI)."""
import multiprocessing
import os
from concurrent.futures import ProcessPoolExecutor

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


def fp64_tol(kappa: float) -> float:
    """Relative error allowed for the plain float64 form against the exact projection.

    Remark 5.1: a float64 computation of Zb is meaningful only to about eps * kappa; the
    float64 form lands well inside that (2.8e-8 = 0.013 eps kappa at 512 x 65536,
    kappa = 1e10), so eps * kappa itself, floored at kappa = 1e3 for the well-conditioned
    cases where rounding of the products dominates, is the bound."""
    return EPS * max(kappa, 1e3)


def assert_rows_close(X, Xref, tol, what="Z"):
    """Per right-hand side (row): ||x - x_ref|| <= tol ||x_ref||, and entry by entry
    |x_i - x_ref,i| <= tol (|x_ref,i| + ||x_ref|| / sqrt(n)) so that an error confined to a
    few entries cannot hide inside the norm."""
    X = np.atleast_2d(np.asarray(X, np.float64))
    Xref = np.atleast_2d(np.asarray(Xref, np.float64))
    assert X.shape == Xref.shape, (what, X.shape, Xref.shape)
    nr = np.linalg.norm(Xref, axis=1)
    nr = np.where(nr == 0, 1.0, nr)
    rel = np.linalg.norm(X - Xref, axis=1) / nr
    assert np.max(rel) < tol, f"{what}: max relative error {np.max(rel):.3g} >= {tol:.3g}"
    scale = np.abs(Xref) + (nr / np.sqrt(X.shape[1]))[:, None]
    worst = np.max(np.abs(X - Xref) / scale)
    assert worst <= tol, f"{what}: element-wise error {worst:.3g} > {tol:.3g}"


def _exact_worker(args):
    key, rows = args
    try:
        from threadpoolctl import threadpool_limits
        lim = threadpool_limits(2)
    except Exception:
        lim = None
    import workloads
    from oracle import exact
    w = workloads.WORKLOADS[key]
    A = w.matrix()
    B = w.rhs()[rows]
    out = exact.exact_project(A, B)
    del lim
    return out


def exact_rows_parallel(key: str, rows, workers: int | None = None):
    """oracle.exact on the given right-hand sides of a named workload, one right-hand side
    per process (spawned, so that no worker inherits a CUDA context); each worker draws the
    workload's A and B from their seeds. Returns (Z, ROW, H) for those rows."""
    rows = list(rows)
    workers = workers or min(len(rows), max(1, (os.cpu_count() or 2) // 2))
    ctx = multiprocessing.get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        parts = list(ex.map(_exact_worker, [(key, [r]) for r in rows]))
    return tuple(np.concatenate([p[i] for p in parts], axis=0) for i in range(3))
