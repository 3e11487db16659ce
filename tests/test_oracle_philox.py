"""Pins for oracle.philox: published Philox4x32-10 known answers, noise moments."""
import os

import numpy as np

from oracle import philox

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = philox.philox4x32_10(np.array(ctr), np.array(key))
        assert [int(v) for v in got] == want


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(17, 4), dtype=np.uint64)
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint64)
    block = philox.philox4x32_10(ctr, key)
    for i in range(17):
        assert np.array_equal(block[i], philox.philox4x32_10(ctr[i], key))


def test_rademacher_values_and_moments():
    n, s = 12 * 4096, 8
    Z = philox.rademacher(n, seed=102, samples=range(s))
    assert set(np.unique(Z)) == {-1.0, 1.0}
    # E[z_i] = 0 and E[z_i z_j] = delta_ij (Sec. 1): sample moments within 6 sigma
    assert abs(Z.mean()) < 6.0 / np.sqrt(Z.size)
    G = Z.T @ Z / n
    assert np.allclose(np.diag(G), 1.0)
    off = G[~np.eye(s, dtype=bool)]
    assert np.max(np.abs(off)) < 6.0 / np.sqrt(n)


def test_rademacher_is_counter_based():
    # a sample does not depend on which other samples are drawn with it,
    # and a prefix of the dof range equals the same prefix of a longer range
    a = philox.rademacher(1000, 7, [3, 4, 5])
    b = philox.rademacher(1300, 7, [5])
    assert np.array_equal(a[:, 2], b[:1000, 0])
    c = philox.rademacher(1000, 8, [3])
    assert not np.array_equal(a[:, 0], c[:, 0])


def test_random_starts_are_unit_complex_signs():
    Y = philox.random_starts(500, 11, 3)
    assert np.all(np.abs(Y.real) == 1.0) and np.all(np.abs(Y.imag) == 1.0)
    assert abs(Y.real.mean()) < 0.2 and abs(Y.imag.mean()) < 0.2
