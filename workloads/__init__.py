"""Seeded synthetic inputs shared by the oracle's tests, the GPU tests and bench.py.

This module holds no arithmetic of the projection method: it only draws test
matrices and right-hand sides. Everything is seeded and reproducible.

* ``haar_spectrum_matrix`` -- A = U diag(sigma) V^T with U (m x m) and V (n x m)
  Haar-distributed orthonormal factors and sigma log-spaced over
  [sigma_min, 1], so that kappa(A) = 1/sigma_min (the workloads of the
  dense-matrix benchmark configurations).
* ``paper_test_matrix`` -- the sparse test family of the paper's Section 5,
  Eqs. (20)-(21): A = U [B | B | ... | B] V with B the circulant
  pentadiagonal (1, -4, 6+d, -4, 1) and U, V uniformly random permutations,
  d = 16/(kappa-1) so that kappa(A) = kappa.
* ``rhs`` -- k right-hand sides with i.i.d. N(0,1) entries, stored as rows
  (k x n, each RHS contiguous).
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "haar_orthonormal",
    "haar_spectrum_matrix",
    "paper_test_matrix",
    "rhs",
    "log_spaced_sigma",
]


def haar_orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix with Haar-distributed orthonormal columns.

    QR of a Gaussian matrix with the columns multiplied by sign(diag R),
    which makes the distribution exactly Haar (Mezzadri, Notices AMS 2007).
    """
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def log_spaced_sigma(m: int, sigma_min: float) -> np.ndarray:
    """sigma_i = sigma_min ** ((i-1)/(m-1)), i = 1..m: sigma_1 = 1, sigma_m = sigma_min."""
    if m == 1:
        return np.ones(1)
    return np.power(float(sigma_min), np.arange(m, dtype=np.float64) / (m - 1))


def haar_spectrum_matrix(m: int, n: int, sigma_min: float, seed: int,
                         dtype=np.float64, return_factors: bool = False, device=None):
    """A = U diag(sigma) V^T, m x n row-major, with kappa(A) = 1/sigma_min.

    U is m x m and V is n x m, both Haar; sigma is log-spaced over
    [sigma_min, 1]. With ``return_factors`` the tuple (A, U, sigma, V) is
    returned, V being the right singular vectors of the exact product (the
    stored A differs from it by rounding).

    ``device`` (a torch device) moves the QR of the n x m Gaussian behind V and
    the product onto that device (float64 LAPACK-style QR of the library torch
    links, the same sign fix); the Gaussian is the same seeded draw, so A agrees
    with the host construction to rounding. It exists for sizes whose host QR
    takes minutes (2048 x 262144).
    """
    if not (1 <= m <= n):
        raise ValueError("need 1 <= m <= n")
    rng = np.random.default_rng(seed)
    u = haar_orthonormal(rng, m, m)
    sig = log_spaced_sigma(m, sigma_min)
    if device is not None:
        import torch
        g = torch.from_numpy(rng.standard_normal((n, m))).to(device)
        q, r = torch.linalg.qr(g)
        del g
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        q *= s[None, :]
        del r
        a_t = (torch.from_numpy(u * sig[None, :]).to(device) @ q.T).contiguous()
        a = np.ascontiguousarray(a_t.cpu().numpy().astype(dtype))
        v = q.cpu().numpy() if return_factors else None
        del q, a_t
        if return_factors:
            return a, u, sig, v
        return a
    v = haar_orthonormal(rng, n, m)
    a = (u * sig[None, :]) @ v.T
    a = np.ascontiguousarray(a.astype(dtype))
    if return_factors:
        return a, u, sig, v
    return a


def paper_test_matrix(m: int, n: int, kappa: float, seed: int, return_parts: bool = False):
    """The sparse test matrix of the paper's Section 5, Eqs. (20)-(21), densified.

    B (m x m) is circulant with B[j,k] = 1 for j = k-2 mod m, -4 for
    j = k-1 mod m, 6+d on the diagonal, -4 for j = k+1 mod m, 1 for
    j = k+2 mod m, and d = 16/(kappa-1). A = U [B|...|B] V, where U (m x m)
    and V (n x n) are uniformly random permutation matrices and n is a
    multiple of m. Stored densely, row-major.

    Permutations are represented by index arrays: ``pu[i]`` is the row of
    [B|...|B] that lands in row i of A, and column c of [B|...|B] lands in
    column ``pv[c]`` of A, i.e. A[i, pv[c]] = C[pu[i], c].
    """
    if n % m != 0:
        raise ValueError("n must be a multiple of m")
    if m < 5:
        raise ValueError("the pentadiagonal stencil needs m >= 5")
    rng = np.random.default_rng(seed)
    d = 16.0 / (float(kappa) - 1.0)
    b = np.zeros((m, m))
    for k in range(m):
        b[(k - 2) % m, k] = 1.0
        b[(k - 1) % m, k] = -4.0
        b[k, k] = 6.0 + d
        b[(k + 1) % m, k] = -4.0
        b[(k + 2) % m, k] = 1.0
    q = n // m
    c = np.tile(b, (1, q))
    pu = rng.permutation(m)
    pv = rng.permutation(n)
    a = np.empty((m, n))
    a[:, pv] = c[pu, :]
    a = np.ascontiguousarray(a)
    if return_parts:
        return a, b, pu, pv
    return a


def paper_test_csr(m: int, n: int, kappa: float, seed: int):
    """The same matrix as ``paper_test_matrix(m, n, kappa, seed)`` (same B, same
    permutations), in compressed sparse row form without densifying: row i of A is row
    pu[i] of [B|...|B], whose nonzeros sit in columns t m + (pu[i] + o) mod m, o = -2..2,
    of each block t, moved to column pv[t m + k]. Entries within a row are ordered by
    block, then by offset o (not by column). Returns (row_ptr int64, col_idx int32,
    val float64, b, pu, pv)."""
    if n % m != 0:
        raise ValueError("n must be a multiple of m")
    if m < 5:
        raise ValueError("the pentadiagonal stencil needs m >= 5")
    rng = np.random.default_rng(seed)
    d = 16.0 / (float(kappa) - 1.0)
    b = np.zeros((m, m))
    for k in range(m):
        b[(k - 2) % m, k] = 1.0
        b[(k - 1) % m, k] = -4.0
        b[k, k] = 6.0 + d
        b[(k + 1) % m, k] = -4.0
        b[(k + 2) % m, k] = 1.0
    pu = rng.permutation(m)
    pv = rng.permutation(n)
    q = n // m
    offs = np.arange(-2, 3)
    j = pu[:, None]                                       # row of [B|...|B] behind row i
    k = (j + offs[None, :]) % m                           # m x 5: its nonzero columns in B
    cols = (np.arange(q)[None, :, None] * m + k[:, None, :])      # m x q x 5, in [B|...|B]
    col_idx = pv[cols].reshape(m, 5 * q).astype(np.int32)
    val = np.broadcast_to(b[j, k][:, None, :], (m, q, 5)).reshape(m, 5 * q).copy()
    row_ptr = np.arange(m + 1, dtype=np.int64) * (5 * q)
    return row_ptr, col_idx.reshape(-1), val.reshape(-1), b, pu, pv


def paper_low_rank(m: int, n: int, seed: int, r: int = 10):
    """The low-rank term of the paper's Eq. 22: E F / sqrt(m n) with E (m x r) and F
    (r x n) i.i.d. standard normal, returned as U = E / sqrt(m n) and V = F."""
    rng = np.random.default_rng(seed)
    E = rng.standard_normal((m, r))
    F = rng.standard_normal((r, n))
    return np.ascontiguousarray(E / np.sqrt(float(m) * float(n))), np.ascontiguousarray(F)


def rhs(k: int, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """k right-hand sides with i.i.d. N(0,1) entries, as a k x n row-major array."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((k, n)).astype(dtype))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic configuration: sizes, spectrum, sketch size and seeds."""
    name: str
    m: int
    n: int
    sigma_min: float
    k: int
    l: int
    seed_a: int
    seed_omega: int
    seed_b: int

    def matrix(self, **kw):
        return haar_spectrum_matrix(self.m, self.n, self.sigma_min, self.seed_a, **kw)

    def paper_family(self, **kw):
        """The paper's own test matrix (Eqs. 20-21) at this workload's size and kappa."""
        return paper_test_matrix(self.m, self.n, 1.0 / self.sigma_min, self.seed_a, **kw)

    def rhs(self, k: int | None = None):
        return rhs(self.k if k is None else k, self.n, self.seed_b)


# Small dense configuration (oracle-sized, l = 4m), the headline dense configuration
# (l = m + 4, the sketch size Section 4 suggests) and the precision-at-scale configuration
# (A 4.3 GB, l = 2m + 32, up to 256 right-hand sides per call; also run at k = 1 and 16).
WORKLOADS = {
    "dense_64x2048": Workload("dense_64x2048_kappa1e8_k16", 64, 2048, 1e-8, 16, 256, 1, 11, 21),
    "dense_512x65536": Workload("dense_512x65536_kappa1e10_k64", 512, 65536, 1e-10, 64, 516, 2, 12, 22),
    "dense_2048x262144": Workload("dense_2048x262144_kappa1e12_k256", 2048, 262144, 1e-12, 256, 4128, 3, 13, 23),
}
