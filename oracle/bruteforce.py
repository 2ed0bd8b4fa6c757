"""Brute-force definitions on explicit n x n matrices — TEST INFRASTRUCTURE ONLY.

These build, for tiny graphs, the objects the method is designed never to
materialise, straight from their definitions, so the oracle's implicit steps
can be checked against them.
"""
from __future__ import annotations

import numpy as np


def msa_exact(Zhat: np.ndarray) -> np.ndarray:
    """S[i, j] = s(u_i, u_j) by Eq. 1: exp(Zh_i.Zh_j) / (sqrt(sum_l exp(Zh_i.Zh_l)) sqrt(sum_l exp(Zh_j.Zh_l)))."""
    E = np.exp(Zhat @ Zhat.T)
    rs = np.sqrt(E.sum(axis=1))
    return E / rs[:, None] / rs[None, :]


def propagation_closed_form(L: np.ndarray, X: np.ndarray, alpha: float, gamma: int) -> np.ndarray:
    """Eq. 6 with the explicit |U| x |U| matrix L L^T and its powers."""
    LL = L @ L.T
    P = np.eye(L.shape[0])
    acc = np.zeros_like(X, dtype=np.float64)
    for r in range(gamma + 1):
        acc += alpha ** r * (P @ X)
        P = P @ LL
    return (1.0 - alpha) * acc


def propagation_limit(L: np.ndarray, X: np.ndarray, alpha: float) -> np.ndarray:
    """gamma -> infinity: the stationary point of Eq. 3, ((1-a) I + a (I - L L^T)) Z = (1-a) X
    (proof of the closed-form lemma, Appendix A.5)."""
    n = L.shape[0]
    A = (1.0 - alpha) * np.eye(n) + alpha * (np.eye(n) - L @ L.T)
    return np.linalg.solve(A, (1.0 - alpha) * X)


def og_pairwise(B: np.ndarray, Z: np.ndarray) -> float:
    """O_g of Eq. 5 as the explicit double sum over pairs, with w_hat(u_i, u_j) =
    sum over common neighbours v_l of w(u_i, v_l) w(v_l, u_j) / D_V[l, l]."""
    du = B.sum(axis=1)
    dv = B.sum(axis=0)
    n = B.shape[0]
    total = 0.0
    for i in range(n):
        for j in range(n):
            common = (B[i] > 0) & (B[j] > 0)
            what = float(np.sum(B[i, common] * B[j, common] / dv[common]))
            if what == 0.0:
                continue
            diff = Z[i] / np.sqrt(du[i]) - Z[j] / np.sqrt(du[j])
            total += what * float(diff @ diff)
    return 0.5 * total


def objective_pairwise(S: np.ndarray, labels: np.ndarray, k: int) -> float:
    """Eq. 8 as written: sum_l (1/|C_l|) sum_{u_i in C_l} sum_{u_j not in C_l} S[i, j]."""
    total = 0.0
    for l in range(k):
        inside = labels == l
        if inside.any():
            total += S[np.ix_(inside, ~inside)].sum() / inside.sum()
    return float(total)


def objective_laplacian(S: np.ndarray, labels: np.ndarray, k: int) -> float:
    """sum_l Y[:, l]^T (S_d - S) Y[:, l] with S_d = diag(row sums of S) and Y the NCI of
    Eq. 10 (proof of Lemma obj2)."""
    n = S.shape[0]
    Sd = np.diag(S.sum(axis=1))
    total = 0.0
    for l in range(k):
        inside = labels == l
        if inside.any():
            y = inside / np.sqrt(inside.sum())
            total += float(y @ (Sd - S) @ y)
    return total


def onmf_unreordered(R: np.ndarray, Phi: np.ndarray, H: np.ndarray):
    """Eqs. 16-17 with the products in the order Section 3.3 says it avoids: the 2d x |U| matrix
    H Phi^T and the |U| x |U| matrix Phi Phi^T are built explicitly. Same clamps as the oracle
    (max(numerator, 0); a non-positive denominator gives 0)."""
    HPt = H @ Phi.T                       # 2d x |U|
    num = R.T @ Phi
    den = HPt @ Phi
    H_new = np.where(den > 0, H * np.maximum(num, 0.0) / np.where(den > 0, den, 1.0), 0.0)
    PPt = Phi @ Phi.T                     # |U| x |U|
    RH = R @ H_new
    den = PPt @ RH
    ratio = np.maximum(RH, 0.0) / np.where(den > 0, den, 1.0)
    Phi_new = np.where(den > 0, Phi * np.sqrt(ratio), 0.0)
    return Phi_new, H_new
