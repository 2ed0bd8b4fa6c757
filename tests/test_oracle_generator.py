"""Pins of the oracle's counter-based Gaussian generator (used for G in Algorithm 1 and the
randomized-SVD test matrices of Algorithm 2 / Section 3.2.1)."""
import numpy as np
import pytest
from scipy import stats

from oracle import philox

# Known-answer vectors published with the Random123 library for Philox4x32-10
# (counter, key) -> output, all words hexadecimal.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    out = philox.philox4x32_10(np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32))
    assert tuple(int(v) for v in out) == expect


def test_gaussian_is_standard_normal():
    g = philox.gaussian_matrix(12345, philox.STREAM_G, 400, 500).ravel()
    assert abs(g.mean()) < 5 * 1 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    assert stats.kstest(g, "norm").pvalue > 1e-3
    # the cos and sin halves of Box-Muller are independent N(0,1)
    pairs = g[: (g.size // 4) * 4].reshape(-1, 4)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 0.02


def test_gaussian_streams_and_prefix_consistency():
    a = philox.gaussian_matrix(7, 1, 10, 10)
    b = philox.gaussian_matrix(7, 2, 10, 10)
    c = philox.gaussian_matrix(8, 1, 10, 10)
    assert np.abs(a - b).max() > 0.1 and np.abs(a - c).max() > 0.1
    # entry e depends only on (seed, stream, e): a 5x20 draw is the same numbers reshaped
    assert np.array_equal(philox.gaussian_matrix(7, 1, 5, 20).ravel(), a.ravel())
    # odd sizes (ragged last block of 4)
    assert np.array_equal(philox.gaussian_matrix(7, 1, 3, 3).ravel(), a.ravel()[:9])
