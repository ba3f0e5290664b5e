"""Philox4x32-10 and the entries of the random test matrix G (Omega).

Test infrastructure only (see ``oracle/__init__.py``).

Section 4 builds S = AG with G an n x l matrix of i.i.d. random entries that is
never stored (Eq. 12). Both this oracle and the CUDA library draw G from the
counter-based generator Philox4x32-10 of Salmon, Moraes, Dror & Shaw
("Parallel random numbers: as easy as 1, 2, 3", SC'11), each side with its own
implementation of the published definition:

* state: counter (c0, c1, c2, c3) and key (k0, k1), all 32-bit words;
* one round: (hi0, lo0) = mulhilo(0xD2511F53, c0), (hi1, lo1) = mulhilo(0xCD9E8D57, c2),
  new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
* between rounds the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85);
* ten rounds.

Entry (i, j) of G (row i < n, column j < l) for seed s uses the block with
counter (i >> 4, j, 0, 0) and key (s mod 2^32, s >> 32); of the 16 output bytes
(word w = (i & 15) >> 2, byte (i & 3) of that word, least significant first)
it takes byte u, and maps it by the chosen distribution:

* ``uniform``:    G_ij = (2u - 255) / 256, uniform on the 256 odd multiples of
                  1/256 in (-1, 1) -- the uniform-on-[-1,1] variates of Tables
                  1, 2, 5 and 6, quantised so that every entry is exact in bfloat16;
* ``rademacher``: G_ij = +1 if u >= 128 else -1.

Both maps are exact integer arithmetic, so the two sides agree bit for bit.

* ``gaussian`` (the variates of Section 3's theory, Theorem 3.1, and of Tables 3-4):
  entries 4q .. 4q+3 of column j come from the block (x, y, z, w) with counter
  (q, j, 1, 0) by the Box-Muller transform (G. E. P. Box and M. E. Muller, "A note on
  the generation of random normal deviates", Ann. Math. Stat. 29, 1958): with
  u1 = ((x >> 9) + 1/2) 2^-23 in (0, 1) and u2 = (y >> 9) 2^-23 in [0, 1),
  r = sqrt(-2 ln u1), entries 4q and 4q+1 are r cos(2 pi u2) and r sin(2 pi u2);
  (z, w) give 4q+2 and 4q+3 the same way. Each variate is rounded to the nearest
  multiple of 2^-12 (ties to even). The oracle evaluates the transform in float64; the
  GPU in float32, so the two can round to neighbouring multiples when the variate lies
  within float32's error of a midpoint: ``gaussian_ambiguous`` marks those entries
  (a few per thousand), and everywhere else the two sides agree bit for bit.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

DISTRIBUTIONS = ("uniform", "rademacher", "gaussian")
GAUSS_GRID = 4096.0          # Gaussian entries are multiples of 1/4096

__all__ = ["philox4x32_10_scalar", "philox4x32_10", "omega_bytes", "omega", "gaussian_variates",
           "gaussian_ambiguous", "DISTRIBUTIONS", "GAUSS_GRID"]


def philox4x32_10_scalar(ctr, key):
    """Plain Python-integer Philox4x32-10 of one counter block (4 words) and key (2 words)."""
    c0, c1, c2, c3 = (int(x) & MASK32 for x in ctr)
    k0, k1 = (int(x) & MASK32 for x in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return c0, c1, c2, c3


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x32-10 over arrays of counters (numpy uint64 arithmetic)."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    s32 = np.uint64(32)
    msk = np.uint64(MASK32)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = m0 * c0          # exact: both factors < 2^32
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & msk
        hi1, lo1 = p1 >> s32, p1 & msk
        c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
    return c0, c1, c2, c3


def omega_bytes(seed: int, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """The byte u used for entries G[rows, cols] (broadcast shapes), as uint8."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    rows, cols = np.broadcast_arrays(rows, cols)
    seed = int(seed)
    words = philox4x32_10(rows >> 4, cols, 0, 0, seed & MASK32, (seed >> 32) & MASK32)
    w = (rows & 15) >> 2
    sel = np.where(w == 0, words[0], np.where(w == 1, words[1], np.where(w == 2, words[2], words[3])))
    shift = (8 * (rows & 3)).astype(np.uint64)
    return ((sel >> shift) & np.uint64(0xFF)).astype(np.uint8)


def gaussian_variates(seed: int, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """The unrounded Box-Muller variates z for entries G[rows, cols] (float64 transform)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    rows, cols = np.broadcast_arrays(rows, cols)
    seed = int(seed)
    w = philox4x32_10(rows >> 2, cols, 1, 0, seed & MASK32, (seed >> 32) & MASK32)
    second_pair = (rows & 2) != 0
    a = np.where(second_pair, w[2], w[0])
    b = np.where(second_pair, w[3], w[1])
    nine = np.uint64(9)
    u1 = ((a >> nine).astype(np.float64) + 0.5) * 2.0 ** -23
    u2 = (b >> nine).astype(np.float64) * 2.0 ** -23
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    return np.where((rows & 1) == 0, r * np.cos(theta), r * np.sin(theta))


def gaussian_ambiguous(seed: int, n: int, l: int, row0: int = 0, col0: int = 0,
                       nrows: int | None = None, ncols: int | None = None) -> np.ndarray:
    """Entries whose rounding to the 2^-12 grid a float32 evaluation of the transform may
    decide the other way: 4096 z within 4096 |z| 2^-20 of a midpoint between grid points.
    (float32 log, square root, sine/cosine and the product each err by at most about one
    unit in the last place, 2^-23 relative, so the whole transform stays within
    2^-21.5 |z|; the window is three times that.)"""
    nrows = n - row0 if nrows is None else nrows
    ncols = l - col0 if ncols is None else ncols
    r = np.arange(row0, row0 + nrows, dtype=np.int64)[:, None]
    c = np.arange(col0, col0 + ncols, dtype=np.int64)[None, :]
    t = gaussian_variates(seed, r, c) * GAUSS_GRID
    dist_to_mid = np.abs(t - (np.floor(t) + 0.5))
    return dist_to_mid <= np.abs(t) * 2.0 ** -20 + 1e-9


def omega(seed: int, n: int, l: int, dist: str = "gaussian", row0: int = 0, col0: int = 0,
          nrows: int | None = None, ncols: int | None = None) -> np.ndarray:
    """The block G[row0:row0+nrows, col0:col0+ncols] of the n x l test matrix (float64)."""
    if dist not in DISTRIBUTIONS:
        raise ValueError(f"unknown distribution {dist!r}")
    nrows = n - row0 if nrows is None else nrows
    ncols = l - col0 if ncols is None else ncols
    r = np.arange(row0, row0 + nrows, dtype=np.int64)[:, None]
    c = np.arange(col0, col0 + ncols, dtype=np.int64)[None, :]
    if dist == "gaussian":
        return np.rint(gaussian_variates(seed, r, c) * GAUSS_GRID) / GAUSS_GRID
    u = omega_bytes(seed, r, c).astype(np.float64)
    if dist == "uniform":
        return (2.0 * u - 255.0) / 256.0
    return np.where(u >= 128.0, 1.0, -1.0)
