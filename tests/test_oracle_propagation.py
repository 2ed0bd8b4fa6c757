"""Pins of the oracle's Algorithm 1 propagation (Eqs. 2, 3-7, 12) on tiny graphs."""
import numpy as np
import pytest

import synth
from oracle import bruteforce, tpo


def _graph(seed, **kw):
    g = synth.make_small(seed, **kw)
    B = tpo.adjacency(g.n_u, g.n_v, g.u_ptr, g.v_idx, g.w)
    return g, B


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_walk_matrix_is_row_stochastic(seed):
    # proof of Lemma FF-ZZ: D_U^-1 B D_V^-1 B^T is row-stochastic; with L of Eq. 7 it equals
    # D_U^-1/2 (L L^T) D_U^1/2
    g, B = _graph(seed, isolated_u=2, isolated_v=3)
    L = tpo.normalized_adjacency(B).toarray()
    du, dv = tpo.degrees(B)
    act = du > 0
    M = (np.diag(1 / np.sqrt(du[act])) @ (L @ L.T)[np.ix_(act, act)] @ np.diag(np.sqrt(du[act])))
    assert np.allclose(M.sum(axis=1), 1.0, atol=1e-12)
    # L L^T is symmetric with spectral radius exactly 1 (Neumann series in the lemma's proof)
    LL = L @ L.T
    assert np.allclose(LL, LL.T, atol=1e-14)
    ev = np.linalg.eigvalsh(LL)
    assert ev.max() == pytest.approx(1.0, abs=1e-10) and ev.min() > -1e-12
    # the isolated U nodes have zero rows in L (reading R2)
    assert np.all(L[~act] == 0)


@pytest.mark.parametrize("alpha,gamma", [(0.6, 6), (0.9, 10), (0.5, 1), (0.3, 0)])
def test_propagation_matches_closed_form(alpha, gamma):
    g, B = _graph(3, n_u=30, n_v=45, d_u=5)
    L = tpo.normalized_adjacency(B)
    X = g.x_dense_f64()
    Z = tpo.propagate(L, X, alpha, gamma)
    Zc = bruteforce.propagation_closed_form(L.toarray(), X, alpha, gamma)
    assert np.allclose(Z, Zc, rtol=1e-12, atol=1e-12)


def test_propagation_limit_solves_the_objective():
    # gamma -> infinity: Z minimises (1-a)||Z-X||^2 + a O_g (Eq. 3), O_g from the pair sum of Eq. 5
    g, B = _graph(4, n_u=24, n_v=30, d_u=4, isolated_v=2)
    alpha = 0.7
    L = tpo.normalized_adjacency(B)
    X = g.x_dense_f64()
    Z = tpo.propagate(L, X, alpha, 200)
    Zs = bruteforce.propagation_limit(L.toarray(), X, alpha)
    assert np.allclose(Z, Zs, rtol=1e-10, atol=1e-10)
    Bd = B.toarray()

    def f(Zm):
        return (1 - alpha) * np.sum((Zm - X) ** 2) + alpha * bruteforce.og_pairwise(Bd, Zm)

    f0 = f(Zs)
    rng = np.random.default_rng(0)
    for _ in range(5):
        E = rng.standard_normal(Z.shape) * 1e-3
        assert f(Zs + E) > f0
    # O_g (pair sum with w_hat) equals Tr(Z^T (I - L L^T) Z) (first step of the proof)
    Ld = L.toarray()
    tr = np.trace(Z.T @ (np.eye(Ld.shape[0]) - Ld @ Ld.T) @ Z)
    assert bruteforce.og_pairwise(Bd, Z) == pytest.approx(tr, rel=1e-10)


def test_special_cases_alpha_and_gamma():
    g, B = _graph(5)
    L = tpo.normalized_adjacency(B)
    X = g.x_dense_f64()
    assert np.array_equal(tpo.propagate(L, X, 0.0, 6), X)          # alpha = 0: Z = X
    assert np.allclose(tpo.propagate(L, X, 0.4, 0), 0.6 * X)       # gamma = 0
    # alpha = 1 leaves the restart form without any attribute input (Z = 0): the library
    # therefore accepts alpha in [0, 1)
    assert np.array_equal(tpo.propagate(L, X, 1.0, 3), 0 * X)


def test_printed_iteration_gives_same_normalised_features():
    # reading R1: the iteration printed with Eq. 12 (Z_0 = aX, Z <- a(X + L L^T Z)) is the
    # restart sum times a/(1-a); Eq. 2 removes the scalar
    g, B = _graph(6)
    L = tpo.normalized_adjacency(B)
    X = g.x_dense_f64()
    a, gam = 0.6, 6
    Zp = a * X
    for _ in range(gam):
        Zp = a * (X + L @ (L.T @ Zp))
    Z = tpo.propagate(L, X, a, gam)
    assert np.allclose(Zp, Z * a / (1 - a), rtol=1e-12)
    assert np.allclose(tpo.normalize_rows(Zp), tpo.normalize_rows(Z), atol=1e-14)


def test_normalize_rows_unit_and_zero_rows():
    Z = np.array([[3.0, 4.0], [0.0, 0.0], [-1.0, 0.0]])
    Zh = tpo.normalize_rows(Z)
    assert np.allclose(Zh, [[0.6, 0.8], [0, 0], [-1, 0]])


def test_isolated_u_keeps_restart_term():
    g, B = _graph(7, isolated_u=3)
    L = tpo.normalized_adjacency(B)
    X = g.x_dense_f64()
    Z = tpo.propagate(L, X, 0.6, 5)
    assert np.allclose(Z[-3:], 0.4 * X[-3:])


def test_transposed_graph_has_the_transposed_operator():
    # clustering V runs the same method on B^T: its L is the transpose of U's L (Eq. 7)
    g = synth.make_small(3, n_u=50, n_v=70, k=3, d_u=4, deg=4)
    L = tpo.normalized_adjacency(tpo.adjacency(g.n_u, g.n_v, g.u_ptr, g.v_idx, g.w))
    order = np.argsort(g.v_idx, kind="stable")
    v_ptr = np.zeros(g.n_v + 1, dtype=np.int64)
    np.cumsum(np.bincount(g.v_idx, minlength=g.n_v), out=v_ptr[1:])
    rows = np.repeat(np.arange(g.n_u, dtype=np.int32), np.diff(g.u_ptr))
    Lt = tpo.normalized_adjacency(tpo.adjacency(g.n_v, g.n_u, v_ptr, rows[order], g.w[order]))
    assert abs(Lt - L.T).max() < 1e-15
