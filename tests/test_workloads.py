"""The seeded input generators (no arithmetic of the method): the compressed sparse row
form of the paper's Section 5 test matrix is the densified matrix, entry for entry."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("m,n", [(8, 64), (37, 1480), (6, 6), (64, 4096)])
def test_paper_test_csr_is_the_dense_matrix(m, n):
    A = workloads.paper_test_matrix(m, n, 1e8, 3)
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, 1e8, 3)
    assert rp.dtype == np.int64 and ci.dtype == np.int32 and v.dtype == np.float64
    assert rp[0] == 0 and rp[-1] == len(ci) == len(v) == 5 * n
    D = np.zeros((m, n))
    rows = np.repeat(np.arange(m), np.diff(rp))
    np.add.at(D, (rows, ci), v)
    assert np.array_equal(A, D)
    # five nonzeros per column (Section 5)
    assert np.all(np.bincount(ci, minlength=n) == 5)


def test_paper_low_rank_term():
    U, V = workloads.paper_low_rank(16, 256, 5)
    assert U.shape == (16, 10) and V.shape == (10, 256)
    E = np.random.default_rng(5).standard_normal((16, 10))
    assert np.array_equal(U, E / np.sqrt(16.0 * 256.0))
