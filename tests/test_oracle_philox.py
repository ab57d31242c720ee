"""Pins for the oracle's Philox4x32-10 (not gpu)."""
import numpy as np
import pytest
from scipy import stats

from conftest import golden_rows
from oracle import philox


@pytest.mark.parametrize("row", golden_rows("philox_kat.txt"))
def test_known_answer_vectors(row):
    name, rounds = row[0], int(row[1])
    width = 32 if name == "philox4x32" else 64
    vals = [int(v, 16) for v in row[2:]]
    ctr, key, expect = vals[0:4], vals[4:6], vals[6:10]
    assert list(philox.philox_generic(ctr, key, width, rounds)) == expect


def test_generic_64bit_matches_numpy_philox():
    # numpy's Philox is Philox4x64-10 and advances its counter before each
    # block, so block c of a fresh generator is counter c + 1.
    for key in (0, 12345, (1 << 64) - 7):
        bg = np.random.Philox(key=key)
        raw = bg.random_raw(4 * 5)
        kw = bg.state["state"]["key"]
        for c in range(5):
            got = philox.philox_generic((c + 1, 0, 0, 0), (int(kw[0]), int(kw[1])), 64)
            assert list(got) == [int(v) for v in raw[4 * c:4 * c + 4]]


def test_vectorised_matches_generic():
    g = np.random.default_rng(0)
    c = g.integers(0, 2 ** 32, size=(200, 4), dtype=np.uint64)
    k = g.integers(0, 2 ** 32, size=2)
    vec = philox.philox4x32(c[:, 0], c[:, 1], c[:, 2], c[:, 3], int(k[0]), int(k[1]))
    for r in range(200):
        assert tuple(int(v[r]) for v in vec) == philox.philox_generic(c[r], k, 32)


def test_negative_index_uniform_chi2():
    n = 97
    u = philox.negative_words(np.arange(200_000), t=3, neg=5, seed=42).ravel()
    m = philox.negative_index(u, n)
    assert m.min() >= 0 and m.max() < n
    counts = np.bincount(m, minlength=n)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4


def test_negative_words_layout():
    # word j' of entry e at epoch t is word (j' mod 4) of block j' div 4
    e = np.array([0, 7, 123456], dtype=np.uint64)
    w = philox.negative_words(e, t=9, neg=6, seed=(5 << 32) | 3)
    for r, ev in enumerate(e):
        for jj in range(6):
            blk = philox.philox_generic((int(ev), 9, jj // 4, 0), (3, 5), 32)
            assert int(w[r, jj]) == blk[jj % 4]
