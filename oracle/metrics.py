"""Clustering quality metrics (Appendix A.3) — TEST INFRASTRUCTURE ONLY.

ACC uses the Hungarian matching of predicted to true clusters; NMI and ARI
follow the standard contingency-table forms the appendix writes out (the
printed NMI numerator drops the |U| factor inside the logarithm; the standard
Strehl-Ghosh form with it is used here).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def contingency(truth: np.ndarray, pred: np.ndarray) -> np.ndarray:
    a = np.unique(truth, return_inverse=True)[1]
    b = np.unique(pred, return_inverse=True)[1]
    M = np.zeros((a.max() + 1, b.max() + 1), dtype=np.int64)
    np.add.at(M, (a, b), 1)
    return M


def acc(truth: np.ndarray, pred: np.ndarray) -> float:
    M = contingency(truth, pred)
    rows, cols = linear_sum_assignment(-M)
    return float(M[rows, cols].sum()) / truth.shape[0]


def nmi(truth: np.ndarray, pred: np.ndarray) -> float:
    M = contingency(truth, pred).astype(np.float64)
    n = M.sum()
    a = M.sum(axis=1)
    b = M.sum(axis=0)
    nz = M > 0
    num = float(np.sum(M[nz] * np.log(n * M[nz] / np.outer(a, b)[nz])))
    ha = float(np.sum(a * np.log(a / n)))
    hb = float(np.sum(b * np.log(b / n)))
    if ha == 0.0 or hb == 0.0:
        return 1.0 if ha == hb else 0.0
    return num / np.sqrt(ha * hb)


def ari(truth: np.ndarray, pred: np.ndarray) -> float:
    M = contingency(truth, pred).astype(np.float64)
    n = M.sum()

    def c2(x):
        return x * (x - 1.0) / 2.0

    s_ij = c2(M).sum()
    s_a = c2(M.sum(axis=1)).sum()
    s_b = c2(M.sum(axis=0)).sum()
    expected = s_a * s_b / c2(n)
    maximum = 0.5 * (s_a + s_b)
    if maximum == expected:
        return 1.0
    return float((s_ij - expected) / (maximum - expected))
