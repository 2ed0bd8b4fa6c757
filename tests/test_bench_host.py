"""Host-side pieces of bench.py that feed its JSON line: the NMI of the quality field (against
the oracle's metric module) and the algorithmic byte count behind the roofline."""
import os
import sys
from types import SimpleNamespace

import numpy as np

from oracle import metrics

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_nmi_matches_the_oracle_metric():
    rng = np.random.default_rng(0)
    for k1, k2 in [(3, 3), (5, 9), (20, 4)]:
        a = rng.integers(0, k1, 2000)
        b = np.where(rng.random(2000) < 0.7, a % k2, rng.integers(0, k2, 2000))
        assert abs(bench.nmi(a, b) - metrics.nmi(a, b)) < 1e-12
    assert bench.nmi(np.zeros(50, int), np.arange(50) % 3) == 0.0   # one cluster: no information


def test_propagation_bytes_formula():
    g = SimpleNamespace(nnz=1000, n_u=100, n_v=300)
    d, gamma = 16, 3
    per_spmm_index = 1000 * 8
    fp32 = 0.0
    for r in range(gamma):
        zin = 2 if r == 0 else 4
        fp32 += per_spmm_index + 1000 * d * zin + 300 * 12 + 300 * d * 4
        fp32 += per_spmm_index + 1000 * d * 4 + 100 * 12 + 100 * d * (2 + 4)
    assert bench.propagation_bytes(g, d, gamma) == fp32
    bf16 = bench.propagation_bytes(g, d, gamma, "bf16")
    # BF16 storage halves the gathered W / Z rows and their writes, except the final Z
    assert fp32 / 2 < bf16 < fp32
