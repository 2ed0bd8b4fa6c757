"""Pins of the oracle's truncated randomized SVD (Algorithm 2 seeding, Eq. 15 reduction) and the
orthogonal NMF updates (Eqs. 16-17)."""
import numpy as np
import pytest

import synth
from oracle import bruteforce, philox, tpo


def _lowrank(n, m, sig, seed):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((n, len(sig))))[0]
    V = np.linalg.qr(rng.standard_normal((m, len(sig))))[0]
    return U @ np.diag(sig) @ V.T


def test_randomized_svd_exact_on_low_rank():
    sig = np.array([9.0, 5.0, 3.0, 2.0, 1.5, 1.0])
    A = _lowrank(300, 40, sig, 0)
    G, S, P = tpo.randomized_svd(A, 4, seed=1, stream=philox.STREAM_OMEGA_R, oversample=3,
                                 power_iters=2)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)   # library SVD as the independent check
    assert np.allclose(S, s[:4], rtol=1e-12)
    for j in range(4):
        sgn = np.sign(U[np.argmax(np.abs(U[:, j])), j])
        assert np.allclose(G[:, j], sgn * U[:, j], atol=1e-10)
        assert np.allclose(P[:, j], sgn * Vt[j], atol=1e-10)
    # sign convention of reading R7: each column's largest-magnitude entry is positive
    assert np.all(G[np.argmax(np.abs(G), axis=0), np.arange(4)] > 0)
    assert np.allclose(G.T @ G, np.eye(4), atol=1e-12)


def test_randomized_svd_eckart_young():
    # full-rank matrix with decaying spectrum: ||A - G S P^T||_2 = sigma_{k+1} (Theorem A.5)
    rng = np.random.default_rng(2)
    A = rng.standard_normal((500, 60)) @ np.diag(0.8 ** np.arange(60)) @ rng.standard_normal((60, 60))
    k = 8
    G, S, P = tpo.randomized_svd(A, k, seed=3, stream=2, oversample=10, power_iters=4)
    s = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - G @ np.diag(S) @ P.T, 2)
    assert err == pytest.approx(s[k], rel=1e-6)
    assert np.allclose(S, s[:k], rtol=1e-8)


def test_attribute_reduction_preserves_gram_and_lemma_bound():
    g = synth.make_small(11, n_u=60, n_v=80, d_u=20, k=3)
    X = g.x_dense_f64()
    # exact rank <= d: X' X'^T = X X^T (Eq. 15 and the identity before it)
    Xr = X[:, :4] @ np.random.default_rng(0).standard_normal((4, 20))
    Xp = tpo.reduce_attributes(Xr, 6, seed=5, oversample=4, power_iters=2)
    assert Xp.shape == (60, 6)
    assert np.allclose(Xp @ Xp.T, Xr @ Xr.T, atol=1e-9 * np.abs(Xr @ Xr.T).max())
    # Lemma FF-ZZ: |Z'[i].Z'[j] - Z[i].Z[j]| <= sigma_{d+1}^2 sqrt(D_U[i,i] D_U[j,j]) / (1-a)
    B = tpo.adjacency(g.n_u, g.n_v, g.u_ptr, g.v_idx, g.w)
    L = tpo.normalized_adjacency(B)
    du, _ = tpo.degrees(B)
    a, d = 0.6, 5
    Z = tpo.propagate(L, X, a, 300)
    Xd = tpo.reduce_attributes(X, d, seed=5, oversample=10, power_iters=6)
    Zd = tpo.propagate(L, Xd, a, 300)
    s = np.linalg.svd(X, compute_uv=False)
    bound = s[d] ** 2 * np.sqrt(np.outer(du, du)) / (1 - a)
    assert np.all(np.abs(Zd @ Zd.T - Z @ Z.T) <= bound * (1 + 1e-9) + 1e-9)


def _nonneg_problem(seed, n=40, m=10, k=3):
    rng = np.random.default_rng(seed)
    return rng.random((n, m)), rng.random((n, k)) + 0.1, rng.random((m, k)) + 0.1


def test_onmf_exact_factorisation_is_a_fixed_point():
    # Phi >= 0 with disjoint supports and unit columns, H >= 0, R = Phi H^T: Eqs. 16-17 leave
    # both factors unchanged
    n, m, k = 30, 8, 3
    rng = np.random.default_rng(4)
    lab = np.arange(n) % k
    Phi = np.zeros((n, k))
    Phi[np.arange(n), lab] = rng.random(n) + 0.5
    Phi /= np.linalg.norm(Phi, axis=0)
    H = rng.random((m, k)) + 0.2
    Phi2, H2 = tpo.onmf_iteration(Phi @ H.T, Phi, H)
    assert np.allclose(Phi2, Phi, rtol=1e-12) and np.allclose(H2, H, rtol=1e-12)


def test_onmf_h_update_is_monotone():
    # Eq. 16 is the Lee-Seung rule for ||R - Phi H^T||_F^2 with Phi fixed: non-increasing
    for seed in range(5):
        R, Phi, H = _nonneg_problem(seed)
        before = np.linalg.norm(R - Phi @ H.T)
        num = R.T @ Phi
        H1 = H * num / (H @ (Phi.T @ Phi))
        _, H2 = tpo.onmf_iteration(R, Phi, H)
        assert np.allclose(H2, H1)
        assert np.linalg.norm(R - Phi @ H2.T) <= before + 1e-12


def test_onmf_matches_unreordered_products():
    # Section 3.3 reorders H Phi^T Phi and Phi Phi^T R H into H (Phi^T Phi) and
    # Phi (Phi^T (R H)); the explicit 2d x |U| and |U| x |U| forms give the same update
    # (a transposed or dropped factor in either rule breaks this on generic inputs)
    for seed in range(4):
        R, Phi, H = _nonneg_problem(seed, n=25, m=7, k=4)
        R = R - 0.3 * (seed % 2)              # also with mixed-sign R (sin features)
        P1, H1 = tpo.onmf_iteration(R, Phi, H)
        P2, H2 = bruteforce.onmf_unreordered(R, Phi, H)
        assert np.allclose(H1, H2, rtol=1e-12, atol=1e-15)
        assert np.allclose(P1, P2, rtol=1e-12, atol=1e-15)


def test_onmf_clamps_and_zero_columns():
    R, Phi, H = _nonneg_problem(8)
    R = R - 0.6                                 # negative entries, as sin features give
    Phi[:, 1] = 0.0                             # a dead column: 0/0 -> stays 0 (reading R9)
    Phi2, H2 = tpo.onmf_iteration(R, Phi, H)
    assert np.all(Phi2 >= 0) and np.all(H2 >= 0)
    assert np.all(np.isfinite(Phi2)) and np.all(np.isfinite(H2))
    assert np.all(Phi2[:, 1] == 0) and np.all(H2[:, 1] == 0)


def test_seed_factors_signs_and_clamps():
    # Eq. 18 with reading R8 on a matrix whose SVD is known exactly: Phi = max(Gamma, 0) and
    # H = max(Psi Sigma, 0), where each left vector carries the sign that makes its entry of
    # largest magnitude positive and its right vector flips with it. Columns are built with mixed
    # signs and one with a negative extreme entry, so an unclamped factor, H without Sigma,
    # Sigma on Phi, a sign flip left on one side only, or H = Psi alone all fail below.
    rng = np.random.default_rng(31)
    n, m, r, k = 400, 24, 8, 5
    U = np.linalg.qr(rng.standard_normal((n, r)))[0]
    V = np.linalg.qr(rng.standard_normal((m, r)))[0]
    U[:, 1] *= -np.sign(U[np.argmax(np.abs(U[:, 1])), 1])   # largest |entry| negative
    s = np.array([7.0, 4.0, 2.5, 1.6, 1.1, 0.5, 0.3, 0.2])
    A = (U * s) @ V.T
    Phi, H, Sig = tpo.seed_factors(A, k, seed=3, oversample=3, power_iters=2)
    sgn = np.where(U[np.argmax(np.abs(U[:, :k]), axis=0), np.arange(k)] < 0, -1.0, 1.0)
    Gam = U[:, :k] * sgn
    Psi = V[:, :k] * sgn
    assert np.allclose(Sig, s[:k], rtol=1e-12)
    assert np.allclose(Phi, np.maximum(Gam, 0.0), atol=1e-10)
    assert np.allclose(H, np.maximum(Psi * s[:k], 0.0), atol=1e-10)
    # both factors really were clamped: the signed vectors have negative entries
    assert (Gam < -1e-3).any() and (Psi < -1e-3).any()
    assert Phi.min() == 0.0 and H.min() == 0.0
    # the flipped column: its largest entry is positive after the flip, H follows the sign
    assert sgn[1] < 0 and Phi[:, 1].max() == np.abs(Gam[:, 1]).max()


def test_sign_rule_is_well_conditioned_on_cluster_vectors():
    # Reading R7 fixes each left singular vector's sign by its largest-magnitude entry. The
    # vectors after the first are orthogonal to the leading, nearly constant one, so their entry
    # sums sit close to zero and a sum-based sign would turn on rounding; the extreme entries of
    # the two signs, in contrast, stay apart. Here (a balanced two-cluster graph, the seeding's
    # randomized SVD of R) the decision margin is far above FP32 rounding while the sum is not.
    g = synth.make_small(112, n_u=60, n_v=78, k=2, d_u=12, deg=5, signal=3.0)
    res = tpo.tpo(g, k=2, alpha=0.6, gamma=4, d=12, t_f=4, t_g=8, seed=17)
    G, _, _ = tpo.randomized_svd(res["R"], 2, 17, philox.STREAM_OMEGA_R)
    g2 = G[:, 1]
    pos, neg = g2.max(), -g2.min()
    assert abs(pos - neg) / max(pos, neg) > 1e-2            # extreme entries well apart
    assert abs(g2.sum()) / np.abs(g2).sum() < 2e-3            # the sum nearly cancels
    assert g2[np.argmax(np.abs(g2))] > 0
