"""Pins for oracle.philox (the generator of the test matrix G)."""
import random

import numpy as np

from oracle import philox


def test_vectorised_matches_plain_integer_definition():
    rnd = random.Random(5)
    ctrs = [[rnd.getrandbits(32) for _ in range(4)] for _ in range(64)]
    key = [rnd.getrandbits(32), rnd.getrandbits(32)]
    vec = philox.philox4x32_10(*[np.array([c[i] for c in ctrs], dtype=np.uint64) for i in range(4)], *key)
    for t, c in enumerate(ctrs):
        assert tuple(int(w[t]) for w in vec) == philox.philox4x32_10_scalar(c, key)


def test_output_bytes_are_uniform():
    u = philox.omega_bytes(12345, np.arange(4096)[:, None], np.arange(64)[None, :]).ravel()
    counts = np.bincount(u, minlength=256)
    expected = u.size / 256
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    assert chi2 < 400          # 255 dof: mean 255, sd ~22.6


def test_omega_moments_and_exact_bfloat16_values():
    G = philox.omega(7, 8192, 32, "uniform")
    assert abs(G.mean()) < 0.01
    assert abs(G.var() - 1.0 / 3.0) < 0.01
    # every value is an odd multiple of 1/256 in (-1, 1): 8 significant bits, exact in bfloat16
    k = G * 256.0
    assert np.all(k == np.round(k)) and np.all(np.abs(k) <= 255) and np.all(np.abs(k) % 2 == 1)
    R = philox.omega(7, 8192, 32, "rademacher")
    assert set(np.unique(R)) == {-1.0, 1.0}
    assert abs(R.mean()) < 0.02


def test_adjacent_columns_and_rows_uncorrelated():
    G = philox.omega(3, 20000, 4)
    c = np.corrcoef(G.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.05
    assert abs(np.corrcoef(G[:-1, 0], G[1:, 0])[0, 1]) < 0.05


def test_block_extraction_consistent_and_seed_dependent():
    G = philox.omega(11, 100, 20)
    blk = philox.omega(11, 100, 20, row0=37, col0=5, nrows=21, ncols=9)
    np.testing.assert_array_equal(G[37:58, 5:14], blk)
    assert not np.array_equal(G, philox.omega(12, 100, 20))
    big = (1 << 40) + 11
    assert not np.array_equal(G, philox.omega(big, 100, 20))
