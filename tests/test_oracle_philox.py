"""Pins for oracle.philox (the generator of the test matrix G)."""
import json
import os
import random

import numpy as np
import pytest

from oracle import philox


def _kat(golden_dir):
    with open(os.path.join(golden_dir, "philox4x32_10_kat.json")) as f:
        cases = json.load(f)["cases"]
    h = lambda ws: [int(w, 16) for w in ws]
    return [(h(c["ctr"]), h(c["key"]), h(c["out"])) for c in cases]


def test_published_known_answer_vectors(golden_dir):
    """Both forms reproduce the three Random123 known-answer vectors bit for bit."""
    for ctr, key, out in _kat(golden_dir):
        assert list(philox.philox4x32_10_scalar(ctr, key)) == out
        vec = philox.philox4x32_10(*[np.array([c], dtype=np.uint64) for c in ctr], *key)
        assert [int(w[0]) for w in vec] == out


@pytest.mark.parametrize("mistake", ["swapped_multipliers", "swapped_outputs", "no_key_bump"])
def test_planted_round_mistakes_fail_the_known_answers(golden_dir, monkeypatch, mistake):
    """A transposed multiplier, a swapped round output or a missing Weyl key bump each
    break every known-answer vector."""
    if mistake == "swapped_multipliers":
        monkeypatch.setattr(philox, "M0", philox.M1)
        monkeypatch.setattr(philox, "M1", 0xD2511F53)
    elif mistake == "no_key_bump":
        monkeypatch.setattr(philox, "W0", 0)
        monkeypatch.setattr(philox, "W1", 0)
    for ctr, key, out in _kat(golden_dir):
        got = list(philox.philox4x32_10_scalar(ctr, key))
        if mistake == "swapped_outputs":
            got = [got[2], got[1], got[0], got[3]]
        assert got != out


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


def test_gaussian_entries_are_standard_normal():
    """Kolmogorov-Smirnov against N(0,1) on 2^18 entries, plus the first four moments:
    a wrong scale (a missing factor 2 in r or in the angle), a shifted uniform or a
    transform of the wrong words fails one of them."""
    from scipy import stats
    G = philox.omega(2024, 4096, 64, "gaussian").ravel()
    ks = stats.kstest(G, "norm")
    assert ks.pvalue > 1e-3, ks
    assert abs(G.mean()) < 0.01
    assert abs(G.var() - 1.0) < 0.01
    assert abs(stats.skew(G)) < 0.03
    assert abs(stats.kurtosis(G, fisher=False) - 3.0) < 0.05


def test_gaussian_pairs_share_radius_and_angle():
    """Entries 4q, 4q+1 (and 4q+2, 4q+3) are the cosine and sine of one Box-Muller pair:
    their squared sum is -2 ln u1 and their angle 2 pi u2, u1 and u2 taken from the words
    of the KAT-pinned scalar Philox at counter (q, j, 1, 0)."""
    seed = (7 << 32) + 99
    n, l = 64, 3
    G = philox.omega(seed, n, l, "gaussian")
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for j in range(l):
        for q in range(n // 4):
            w = philox.philox4x32_10_scalar((q, j, 1, 0), key)
            for pair, (a, b) in enumerate(((w[0], w[1]), (w[2], w[3]))):
                z0, z1 = G[4 * q + 2 * pair, j], G[4 * q + 2 * pair + 1, j]
                u1 = ((a >> 9) + 0.5) * 2.0 ** -23
                u2 = (b >> 9) * 2.0 ** -23
                r = np.hypot(z0, z1)
                assert abs(r * r - (-2.0 * np.log(u1))) <= 4 * r * 2.0 ** -12 + 1e-12
                if r > 0.05:
                    ang = np.arctan2(z1, z0) % (2 * np.pi)
                    d = abs(ang - 2 * np.pi * u2)
                    assert min(d, 2 * np.pi - d) <= 2.0 ** -11 / r


def test_gaussian_grid_range_and_ambiguity():
    G = philox.omega(5, 8192, 16, "gaussian")
    k = G * philox.GAUSS_GRID
    assert np.all(k == np.round(k))                     # multiples of 2^-12
    assert np.max(np.abs(G)) < 5.78                     # r <= sqrt(-2 ln 2^-24)
    amb = philox.gaussian_ambiguous(5, 8192, 16)
    assert amb.shape == G.shape
    assert 0 < amb.mean() < 0.01
    # an ambiguous entry sits next to a midpoint: its unrounded variate is within the window
    z = philox.gaussian_variates(5, np.arange(8192)[:, None], np.arange(16)[None, :])
    t = z[amb] * philox.GAUSS_GRID
    assert np.all(np.abs(np.abs(t - np.floor(t)) - 0.5) <= np.abs(t) * 2.0 ** -20 + 1e-9)


def test_gaussian_columns_and_rows_independent():
    G = philox.omega(8, 40000, 4, "gaussian")
    c = np.corrcoef(G.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.03
    for lag in (1, 2, 3, 4):                            # within and across Box-Muller pairs
        assert abs(np.corrcoef(G[:-lag, 0], G[lag:, 0])[0, 1]) < 0.03
    # cosine and sine of one pair are uncorrelated but not independent: their squares are
    # tied through the shared radius, which the moments of z0^2 + z1^2 (chi-square, 2 dof) show
    r2 = G[0::2, 0] ** 2 + G[1::2, 0] ** 2
    assert abs(r2.mean() - 2.0) < 0.05 and abs(r2.var() - 4.0) < 0.2
