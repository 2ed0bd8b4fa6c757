"""Pins of the oracle's MSA (Eq. 1) and random features (Eqs. 13-14, Theorem 1)."""
import numpy as np
import pytest

from conftest import load_golden
from oracle import bruteforce, tpo


def test_worked_example_msa():
    # Appendix A.1 running example: Eq. 1 applied to the printed Z_hat reproduces the printed
    # MSA matrix. Z_hat is printed to 2 decimals (+-0.005 per entry moves each dot product by up
    # to ~0.015, i.e. ~0.002 on MSA values near 0.143), so the bound is 3e-3.
    gold = load_golden("worked_example_msa.txt")
    S = bruteforce.msa_exact(gold["zhat"])
    assert np.abs(S - gold["msa"]).max() < 3e-3
    assert np.allclose(S, S.T)  # MSA is symmetric (Section 2.2)
    # the printed matrix itself names each node's nearest neighbour as the text states
    P = gold["msa"].copy()
    np.fill_diagonal(P, -1)
    assert list(P.argmax(axis=1) + 1) == [int(v) for v in gold["nearest"][0]]


def test_orthogonal_matrix_is_orthogonal_and_seeded():
    Q = tpo.orthogonal_matrix(3, 24)
    assert np.allclose(Q.T @ Q, np.eye(24), atol=1e-13)
    assert np.array_equal(Q, tpo.orthogonal_matrix(3, 24))
    assert np.abs(Q - tpo.orthogonal_matrix(4, 24)).max() > 0.1


def _unit_rows(n, d, seed):
    Z = np.random.default_rng(seed).standard_normal((n, d))
    Z[1] = Z[0] + 0.3 * Z[1]  # one close pair
    return tpo.normalize_rows(Z)


def test_feature_rows_have_norm_e_and_scale_invariance():
    Zh = _unit_rows(10, 12, 0)
    Q = tpo.orthogonal_matrix(1, 12)
    Rp, r, R, clamped = tpo.random_features(Zh, Q)
    # sin^2 + cos^2 = 1 per feature: ||R'[i]||^2 = (e/d) * d = e
    assert np.allclose((Rp ** 2).sum(axis=1), np.e, rtol=1e-14)
    assert R.shape == (10, 24) and clamped == 0
    # Eq. 14 is invariant to a global scale of R' (reading R4 relies on this)
    c = 3.7
    Rs = c * Rp / np.sqrt((c * Rp) @ (c * r))[:, None]
    assert np.allclose(Rs, R, rtol=1e-13)
    # rows of R satisfy R[i].r' = sqrt(R'[i].r) where r' = sum of R' rows
    assert np.allclose(R @ r, np.sqrt(Rp @ r), rtol=1e-12)


def _feature_moments(Zh, d, M, base):
    n = Zh.shape[0]
    acc = np.zeros((n, n))
    acc2 = np.zeros((n, n))
    for s in range(M):
        Rp, _, _, _ = tpo.random_features(Zh, tpo.orthogonal_matrix(base + s, d))
        G = Rp @ Rp.T
        acc += G
        acc2 += G * G
    mean = acc / M
    return mean, np.sqrt(np.maximum(acc2 / M - mean ** 2, 0) / M)


def test_theorem1_random_features_estimate_exp_kernel():
    # Proof of Theorem 1: E[R'[i].R'[j]] = (e/d) sum_l E[cos(Qhat[l].z)], z = Zh_i - Zh_j, and the
    # lemma it cites (Yu et al. 2016, orthogonal random features, Lemma 5) gives
    #   |E[cos]/exp(-|z|^2/2) - (1 - |z|^4/(4d))| <= |z|^4 (|z|^4 + 8|z|^2 + 8) / (16 d^2).
    # The printed bound [1 -+ 17/(16d^2) -+ 1/(4d)] follows from it when |z|^2 <= 1, i.e. for
    # pairs with Zh_i.Zh_j >= 1/2 (the proof assumes |z|^2 in [0,1]; for unit rows it reaches 4).
    d, M = 16, 3000
    rng = np.random.default_rng(1)
    Zh = _unit_rows(6, d, 1)
    mean, se = _feature_moments(Zh, d, M, 1000)
    ratio = mean / np.exp(Zh @ Zh.T)
    slack = 4 * se / np.exp(Zh @ Zh.T)
    z2 = 2.0 * (1.0 - Zh @ Zh.T)
    lemma_mid = 1 - z2 ** 2 / (4 * d)
    lemma_rad = z2 ** 2 * (z2 ** 2 + 8 * z2 + 8) / (16 * d * d)
    assert np.all(np.abs(ratio - lemma_mid) <= lemma_rad + slack + 1e-12)
    close = z2 <= 1.0
    assert close.sum() > 6                       # the diagonal plus the planted close pair
    paper = 17 / (16 * d * d) + 1 / (4 * d)
    assert np.all(np.abs(ratio[close] - 1) <= paper + slack[close] + 1e-12)
    # the bias term is real: a pair at |z|^2 = 2 sits well below 1 (a missing sqrt(d) inside
    # sin/cos would instead push the ratio far above 1)
    assert ratio[~close].mean() < 1 - 0.5 * (z2[~close] ** 2).mean() / (4 * d)


def test_theorem1_normalised_features_approach_msa():
    # R R^T averaged over draws of Q approaches the MSA of Eq. 1; at d = 64 the |z|^4/(4d) bias
    # of random unit rows (|z|^2 ~ 2) is ~1.6%, the ratio-of-expectations step adds a little
    d, n = 64, 8
    Zh = _unit_rows(n, d, 2)
    accR = np.zeros((n, n))
    M = 400
    for s in range(M):
        _, _, R, _ = tpo.random_features(Zh, tpo.orthogonal_matrix(5000 + s, d))
        accR += R @ R.T
    S = bruteforce.msa_exact(Zh)
    assert np.abs(accR / M / S - 1).max() < 0.05


def test_zero_row_features():
    # reading R3: a zero row of Z has Z_hat = 0 -> R' = sqrt(e/d) (0 || 1)
    Zh = np.zeros((3, 4))
    Zh[1] = [1, 0, 0, 0]
    Rp, _, _, _ = tpo.random_features(Zh, np.eye(4))
    assert np.allclose(Rp[0], np.sqrt(np.e / 4) * np.r_[np.zeros(4), np.ones(4)])
