"""Pins of the oracle's NCI generation (Algorithm 3, Eqs. 21-23), the objective (Eq. 8), the
quality metrics (Appendix A.3) and planted-partition recovery end to end."""
import numpy as np
import pytest

import synth
from oracle import bruteforce, metrics, tpo


def _indicator(labels, k):
    Y = np.zeros((labels.shape[0], k))
    Y[np.arange(labels.shape[0]), labels] = 1.0
    n = Y.sum(axis=0)
    return Y / np.sqrt(np.where(n > 0, n, 1.0))


def test_objective_matches_pair_sums_and_trace():
    rng = np.random.default_rng(0)
    n, m, k = 50, 12, 4
    R = rng.standard_normal((n, m))
    labels = rng.integers(0, k, n)
    labels[:k] = np.arange(k)
    S = R @ R.T
    obj1, J = tpo.objective(R, labels, k)
    assert obj1 == pytest.approx(bruteforce.objective_pairwise(S, labels, k), rel=1e-12)
    assert obj1 == pytest.approx(bruteforce.objective_laplacian(S, labels, k), rel=1e-12)
    Y = _indicator(labels, k)
    assert J == pytest.approx(np.trace(Y.T @ S @ Y), rel=1e-12)


def test_objective_with_empty_cluster():
    rng = np.random.default_rng(1)
    R = rng.standard_normal((20, 6))
    labels = np.where(np.arange(20) < 10, 0, 2)
    obj1, J = tpo.objective(R, labels, 4)
    S = R @ R.T
    assert obj1 == pytest.approx(bruteforce.objective_pairwise(S, labels, 4), rel=1e-12)


def test_objective_msa_brute_force_small():
    # with s from Eq. 1 the same pair sum is the paper's objective; the oracle's objective with
    # S := R R^T approaches it as R R^T -> S (Theorem 1): checked loosely with d = 64
    rng = np.random.default_rng(2)
    Zh = tpo.normalize_rows(rng.standard_normal((12, 64)))
    labels = np.arange(12) % 3
    S = bruteforce.msa_exact(Zh)
    exact = bruteforce.objective_pairwise(S, labels, 3)
    est = np.mean([tpo.objective(tpo.random_features(Zh, tpo.orthogonal_matrix(s, 64))[2],
                                 labels, 3)[0] for s in range(200)])
    assert est == pytest.approx(exact, rel=0.05)


def test_nci_fixed_point_and_invariants():
    k, n = 4, 40
    lab = np.arange(n) % k
    Phi = _indicator(lab, k)
    labels, T, margin, changes = tpo.nci(Phi, 5)
    assert np.array_equal(labels, lab)
    assert np.allclose(T, np.eye(k))              # Phi^T Y = Y^T Y = I
    assert changes[1:] == [0] * 4
    Y = tpo.nci_matrix(labels, k).toarray()
    assert np.all((Y > 0).sum(axis=1) == 1)       # one nonzero per row (Eq. 10)
    assert np.allclose(Y.T @ Y, np.eye(k))        # unit columns (Eq. 23) -> Y^T Y = I


def test_nci_noisy_indicator_recovers_partition_and_ties():
    rng = np.random.default_rng(3)
    k, n = 5, 200
    lab = rng.permutation(np.arange(n) % k)
    Phi = np.abs(_indicator(lab, k) + 0.02 * rng.standard_normal((n, k)))
    Phi[0] = 0.0                                  # all-zero row: every score ties at 0
    labels, T, margin, _ = tpo.nci(Phi, 10)
    assert labels[0] == 0                         # lowest index wins (reading R11)
    assert np.array_equal(labels[1:], lab[1:])
    assert margin[0] == 0.0


def test_nci_empty_cluster_has_zero_column():
    rng = np.random.default_rng(4)
    Phi = rng.random((30, 3))
    Phi[:, 2] = 0.0
    Phi[:, 1] += 1.0
    labels, T, _, _ = tpo.nci(Phi, 4)
    assert np.all(labels == 1)
    assert np.all(T[:, 0] == 0) and np.all(T[:, 2] == 0)
    assert np.all(np.isfinite(T))


def test_metrics_basic():
    t = np.array([0, 0, 1, 1, 2, 2, 2])
    p = np.array([5, 5, 3, 3, 9, 9, 9])
    assert metrics.acc(t, p) == 1.0 and metrics.nmi(t, p) == pytest.approx(1.0)
    assert metrics.ari(t, p) == pytest.approx(1.0)
    q = np.array([0, 1, 0, 1, 0, 1, 0])
    assert metrics.acc(t, q) == pytest.approx(3 / 7)
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    a, b = rng.integers(0, 4, 300), rng.integers(0, 5, 300)
    assert metrics.nmi(a, b) == pytest.approx(skm.normalized_mutual_info_score(a, b, average_method="geometric"))
    assert metrics.ari(a, b) == pytest.approx(skm.adjusted_rand_score(a, b))


def test_planted_partition_recovery_config1():
    # workload 1 (2,000 U nodes, k=5, well separated): TPO recovers the planted clusters
    g = synth.make_config1()
    p = g.params
    res = tpo.tpo(g, k=p["k"], alpha=p["alpha"], gamma=p["gamma"], d=p["d"], t_f=p["t_f"],
                  t_g=p["t_g"], seed=0)
    assert metrics.acc(g.truth, res["labels"]) >= 0.9
    assert metrics.nmi(g.truth, res["labels"]) >= 0.75
    # the returned objective is the pair sum of Eq. 8 over R R^T, and the planted partition's
    # own objective is of the same order
    assert res["objective"] > 0 and np.isfinite(res["trace_obj"])


def test_polar_is_the_nearest_orthogonal_matrix():
    # polar decomposition M = T P with T orthogonal and P = T^T M symmetric positive
    # semidefinite; no orthogonal matrix is closer to M (checked against random rotations)
    rng = np.random.default_rng(5)
    M = rng.standard_normal((5, 5))
    T = tpo.polar(M)
    assert np.allclose(T.T @ T, np.eye(5), atol=1e-12)
    P = T.T @ M
    assert np.allclose(P, P.T, atol=1e-12)
    assert np.linalg.eigvalsh((P + P.T) / 2).min() > -1e-12
    best = np.linalg.norm(M - T)
    for _ in range(200):
        Qr = np.linalg.qr(rng.standard_normal((5, 5)))[0]
        assert np.linalg.norm(M - Qr) >= best - 1e-12


def test_polar_rank_deficient_and_k1():
    # an empty cluster zeroes a column of Phi^T Y: T keeps that column zero and is a partial
    # isometry on the rest; for k = 1 the factor is the sign of the one entry
    rng = np.random.default_rng(6)
    M = rng.standard_normal((4, 4))
    M[:, 2] = 0.0
    T = tpo.polar(M)
    assert np.allclose(T[:, 2], 0.0, atol=1e-12)
    assert np.allclose(T @ T.T @ T, T, atol=1e-12)
    assert np.allclose(tpo.polar(np.array([[-3.0]])), [[-1.0]])
    assert np.allclose(tpo.polar(np.zeros((3, 3))), 0.0)


def test_nci_procrustes_scores_and_fixed_point():
    # with an orthogonal T the scores Phi T preserve row norms; a planted indicator converges,
    # and early stopping ends at the first pass that changes nothing with the same labels and T
    rng = np.random.default_rng(8)
    n, k = 600, 5
    truth = rng.integers(0, k, n)
    Phi = np.abs(0.05 * rng.standard_normal((n, k)))
    Phi[np.arange(n), truth] += 1.0
    lab, T, _, ch = tpo.nci(Phi, 12, procrustes=True)
    assert np.allclose(T.T @ T, np.eye(k), atol=1e-10)
    assert np.allclose(np.linalg.norm(Phi @ T, axis=1), np.linalg.norm(Phi, axis=1))
    assert ch[-1] == 0
    lab2, T2, _, ch2 = tpo.nci(Phi, 12, procrustes=True, early_stop=True)
    assert len(ch2) < 12 and ch2[-1] == 0 and all(c > 0 for c in ch2[1:-1])
    assert np.array_equal(lab, lab2) and np.allclose(T, T2, atol=1e-12)
    lab3, T3, _, ch3 = tpo.nci(Phi, 12, early_stop=True)
    lab4, T4, _, _ = tpo.nci(Phi, 12)
    assert np.array_equal(lab3, lab4) and np.allclose(T3, T4, atol=1e-12) and len(ch3) <= 12


def test_printed_t_collapses_many_clusters_procrustes_keeps_them():
    # the large workload's generator at 1% (20,000 U nodes, k = 100): with T = Phi^T Y as
    # printed every score Phi[i].T[:, l] = sum_{j in C_l} Phi[i].Phi[j] / sqrt(|C_l|) is positive
    # and grows with the cluster, so one cluster absorbs the rest; the orthogonal Procrustes T
    # (the constraint T T^T = I of Eq. 20) keeps the clusters apart
    g = synth.make_config3(scale=0.01)
    p = dict(k=100, alpha=0.9, gamma=10, d=128, t_f=5, t_g=20, seed=0)
    printed = tpo.tpo(g, **p)
    assert np.unique(printed["labels"]).size == 1 and printed["objective"] == 0.0
    proc = tpo.tpo(g, procrustes=True, **p)
    assert np.unique(proc["labels"]).size >= 90
    assert metrics.nmi(g.truth, proc["labels"]) >= 0.4
    # Algorithm 3 feeds its labels back into T: a change of Phi of the size of the difference
    # between an FP32 and an FP64 evaluation of the steps before it (1e-5 to 1e-4 of max |Phi|)
    # moves some labels even on nodes whose final margin exceeds 1e-4, by way of a near-tie in
    # an earlier pass, while 1e-9 moves none. The GPU parity tests of this workload rest on this.
    sure = proc["margin"] > 1e-4
    moved = {}
    for eps in (1e-9, 1e-4):
        rng = np.random.default_rng(0)
        Phi = proc["Phi"]
        Phi2 = np.maximum(Phi + eps * np.abs(Phi).max() * rng.standard_normal(Phi.shape), 0.0)
        lab2, _, _, _ = tpo.nci(Phi2, p["t_g"], procrustes=True)
        moved[eps] = int(np.count_nonzero(lab2[sure] != proc["labels"][sure]))
        obj2, _ = tpo.objective(proc["R"], lab2, p["k"])
        assert abs(obj2 / proc["objective"] - 1.0) < 2e-5
    assert moved[1e-9] == 0 and 0 < moved[1e-4] <= 0.005 * sure.sum()
