"""Plain FP64 CPU oracle of TPO (arXiv 2405.11922) — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and its ``--impl reference`` arm) may import this module. The CUDA
library never calls it and shares no code with it.

Each function follows one step of the method in the paper's order and
notation; numpy / scipy primitives (dense and sparse matrix products, QR,
SVD) serve as single steps, with no blocking, fusion or reordering beyond
what the paper writes. Where the paper is silent or inconsistent the reading
taken is named in the docstring of the function that uses it (R1..R13, each
stated in full below; R14 and R17 with ``nci`` and ``polar``).

Readings used here
  R1  restart form of the propagation: Z_0 = (1-a) X and
      Z <- (1-a) X + a L (L^T Z), gamma times. This is the closed form of
      Eq. 6 exactly; the iteration printed in Algorithm 1 / Eq. 12 is the same
      sum scaled by a/(1-a), which the row normalisation of Eq. 2 cancels.
  R2  a node of zero degree gets the scale 0 in D^{-1/2} (Eq. 7).
  R3  an all-zero row of Z stays zero under Eq. 2.
  R4  with attribute reduction on, d in Eq. 13 is the reduced width.
  R5  R'[i].r <= 0 is clamped to 1e-300 before the square root of Eq. 14.
  R6  Q = the orthogonal factor of a Householder QR of G with diag(R_qr) > 0.
  R7  randomized SVD = randomized subspace iteration of Halko, Martinsson and
      Tropp (2011): l = min(k + p, rows, cols) Gaussian columns, q power
      iterations, every block re-orthonormalised; the small factor's SVD gives
      the top k triplets; each left vector is signed so that its entry of
      largest magnitude is positive (the first such entry on ties).
  R8  Phi = max(Gamma, 0), H = max(Psi Sigma, 0) (Eq. 18 with the
      non-negativity Eq. 11 asks for).
  R9  Eqs. 16 / 17 use max(numerator, 0); an entry whose denominator is <= 0
      becomes 0.
  R10 H is updated from the old Phi, then Phi from the new H (Algorithm 2).
  R11 argmax ties go to the lowest cluster index (Eq. 21).
  R12 an empty cluster keeps a zero column in Y and in T (Eq. 23).
  R13 the objective reported is Eq. 8 with s(u_i, u_j) := R[i].R[j], plus
      J = Tr(Y^T R R^T Y) from the proof of Lemma obj3.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .philox import STREAM_G, STREAM_OMEGA_R, STREAM_OMEGA_X, gaussian_matrix

CLAMP_RR = 1e-300  # R5


# ----------------------------------------------------------------------------
# Section 2.1 / Eq. 7: degrees and the normalised adjacency L_U
# ----------------------------------------------------------------------------

def adjacency(n_u: int, n_v: int, u_ptr, v_idx, w=None) -> sp.csr_matrix:
    """B_U (|U| x |V|) with B[i, j] = w(u_i, v_j) (Section 2.1); unit weights when w is None."""
    nnz = int(u_ptr[-1])
    data = np.ones(nnz) if w is None else np.asarray(w, dtype=np.float64)
    return sp.csr_matrix((data, np.asarray(v_idx), np.asarray(u_ptr)), shape=(n_u, n_v))


def degrees(B: sp.csr_matrix) -> tuple[np.ndarray, np.ndarray]:
    """Diagonals of D_U and D_V: weighted degrees of U and V nodes (Section 2.1)."""
    du = np.asarray(B.sum(axis=1)).ravel()
    dv = np.asarray(B.sum(axis=0)).ravel()
    return du, dv


def inv_sqrt_or_zero(deg: np.ndarray) -> np.ndarray:
    """D^{-1/2} with the scale 0 for a zero degree (R2)."""
    out = np.zeros_like(deg, dtype=np.float64)
    pos = deg > 0
    out[pos] = 1.0 / np.sqrt(deg[pos])
    return out


def normalized_adjacency(B: sp.csr_matrix) -> sp.csr_matrix:
    """L_U = D_U^{-1/2} B_U D_V^{-1/2} (Eq. 7)."""
    du, dv = degrees(B)
    return (sp.diags(inv_sqrt_or_zero(du)) @ B @ sp.diags(inv_sqrt_or_zero(dv))).tocsr()


# ----------------------------------------------------------------------------
# Algorithm 1: MSA approximation
# ----------------------------------------------------------------------------

def propagate(L: sp.csr_matrix, X: np.ndarray, alpha: float, gamma: int) -> np.ndarray:
    """Z_U = (1-a) sum_{r=0..gamma} a^r (L L^T)^r X (Eq. 6), evaluated as in Eq. 12 with the
    product ordered L (L^T Z) and the restart weights of R1."""
    X = np.asarray(X, dtype=np.float64)
    Z = (1.0 - alpha) * X
    for _ in range(gamma):
        Z = (1.0 - alpha) * X + alpha * (L @ (L.T @ Z))
    return Z


def normalize_rows(Z: np.ndarray) -> np.ndarray:
    """Z_hat[i] = Z[i] / ||Z[i]|| (Eq. 2); zero rows stay zero (R3)."""
    nrm = np.linalg.norm(Z, axis=1)
    out = np.zeros_like(Z)
    pos = nrm > 0
    out[pos] = Z[pos] / nrm[pos, None]
    return out


def orthonormal_basis(Y: np.ndarray) -> np.ndarray:
    """Orthogonal factor of Y = QR with a positive diagonal in R (unique for full column rank)."""
    Q, Rq = np.linalg.qr(Y)
    sgn = np.where(np.diag(Rq) < 0, -1.0, 1.0)
    return Q * sgn[None, :]


def orthogonal_matrix(seed: int, d: int) -> np.ndarray:
    """Sample G in R^{d x d} with N(0,1) entries and take Q from its QR decomposition
    (Algorithm 1; reading R6)."""
    G = gaussian_matrix(seed, STREAM_G, d, d)
    return orthonormal_basis(G)


def random_features(Zhat: np.ndarray, Q: np.ndarray):
    """R' = sqrt(e/d) (sin(Z°) || cos(Z°)) with Z° = sqrt(d) Zhat Q^T (Eq. 13), then
    R[i] = R'[i] / sqrt(R'[i].r) with r = sum_l R'[l] (Eq. 14). Returns (R', r, R, #clamped)."""
    d = Zhat.shape[1]
    Zc = np.sqrt(d) * (Zhat @ Q.T)
    Rp = np.sqrt(np.e / d) * np.concatenate([np.sin(Zc), np.cos(Zc)], axis=1)
    r = Rp.sum(axis=0)
    dots = Rp @ r
    clamped = int(np.count_nonzero(dots <= CLAMP_RR))
    R = Rp / np.sqrt(np.maximum(dots, CLAMP_RR))[:, None]
    return Rp, r, R, clamped


# ----------------------------------------------------------------------------
# Truncated randomized SVD (Algorithm 2 seeding, Section 3.2.1 reduction)
# ----------------------------------------------------------------------------

def randomized_svd(A, k: int, seed: int, stream: int, oversample: int = 10, power_iters: int = 4):
    """Top-k (Gamma, Sigma, Psi) of A by randomized subspace iteration (R7)."""
    n, m = A.shape
    l = min(k + oversample, n, m)
    Omega = gaussian_matrix(seed, stream, m, l)
    Qb = orthonormal_basis(A @ Omega)
    for _ in range(power_iters):
        Qt = orthonormal_basis(np.asarray(A.T @ Qb))
        Qb = orthonormal_basis(np.asarray(A @ Qt))
    Bs = np.asarray(A.T @ Qb).T          # B = Q^T A  (l x m)
    Ub, s, Vt = np.linalg.svd(Bs, full_matrices=False)
    Gamma = Qb @ Ub[:, :k]
    Sigma = s[:k].copy()
    Psi = Vt[:k].T.copy()
    big = np.argmax(np.abs(Gamma), axis=0)              # first largest |entry| per column
    flip = Gamma[big, np.arange(Gamma.shape[1])] < 0
    Gamma[:, flip] *= -1.0
    Psi[:, flip] *= -1.0
    return Gamma, Sigma, Psi


def reduce_attributes(X, d: int, seed: int, oversample: int = 10, power_iters: int = 4) -> np.ndarray:
    """X'_U = Gamma Sigma from the top-d SVD of X_U (Eq. 15, Section 3.2.1)."""
    Gamma, Sigma, _ = randomized_svd(X, d, seed, STREAM_OMEGA_X, oversample, power_iters)
    return Gamma * Sigma[None, :]


# ----------------------------------------------------------------------------
# Algorithm 2: greedy orthogonal NMF
# ----------------------------------------------------------------------------

def seed_factors(R: np.ndarray, k: int, seed: int, oversample: int = 10, power_iters: int = 4):
    """Phi = Gamma, H = Psi Sigma from the truncated randomized SVD of R (Eq. 18; R8)."""
    Gamma, Sigma, Psi = randomized_svd(R, k, seed, STREAM_OMEGA_R, oversample, power_iters)
    return np.maximum(Gamma, 0.0), np.maximum(Psi * Sigma[None, :], 0.0), Sigma


def onmf_iteration(R: np.ndarray, Phi: np.ndarray, H: np.ndarray):
    """One pass of Algorithm 2's loop: H by Eq. 16, then Phi by Eq. 17 (R9, R10)."""
    num = R.T @ Phi                       # (R^T Phi)
    den = H @ (Phi.T @ Phi)               # H (Phi^T Phi)
    H_new = np.zeros_like(H)
    pos = den > 0
    H_new[pos] = H[pos] * np.maximum(num[pos], 0.0) / den[pos]
    P = R @ H_new                         # R H
    den = Phi @ (Phi.T @ P)               # Phi (Phi^T (R H))
    Phi_new = np.zeros_like(Phi)
    pos = den > 0
    Phi_new[pos] = Phi[pos] * np.sqrt(np.maximum(P[pos], 0.0) / den[pos])
    return Phi_new, H_new


def onmf(R: np.ndarray, Phi: np.ndarray, H: np.ndarray, t_f: int):
    for _ in range(t_f):
        Phi, H = onmf_iteration(R, Phi, H)
    return Phi, H


# ----------------------------------------------------------------------------
# Algorithm 3: NCI generation
# ----------------------------------------------------------------------------

def nci_matrix(labels: np.ndarray, k: int) -> sp.csr_matrix:
    """Y with Y[i, l*] = 1 (Eq. 22), columns scaled to unit L2 norm (Eq. 23; R12)."""
    n = labels.shape[0]
    counts = np.bincount(labels, minlength=k).astype(np.float64)
    vals = 1.0 / np.sqrt(counts[labels])
    return sp.csr_matrix((vals, (np.arange(n), labels)), shape=(n, k))


def polar(M: np.ndarray, rcond: float = 1e-5) -> np.ndarray:
    """Orthogonal Procrustes factor of M (the T nearest to M with orthonormal columns on M's
    range): T = U_r V_r^T from the SVD M = U S V^T, keeping the singular values above
    rcond * s_1 (empty clusters make M rank deficient; the product is then still unique)."""
    if M.size == 0:
        return M.copy()
    U, s, Vt = np.linalg.svd(M)
    if s[0] <= 0:
        return np.zeros_like(M)
    r = int(np.count_nonzero(s > rcond * s[0]))
    return U[:, :r] @ Vt[:r]


def nci(Phi: np.ndarray, t_g: int, procrustes: bool = False, early_stop: bool = False):
    """T = I; t_g times: l* = argmax_l Phi[i].T[:, l] (Eq. 21; R11), Y by Eqs. 22-23,
    T <- Phi^T Y (Algorithm 3), or with ``procrustes`` the orthogonal factor of Phi^T Y (the
    constraint T T^T = I of Eq. 20 enforced exactly). With ``early_stop`` the passes end after
    the first pass, other than the first, that changes no label: Y, hence T, is then a fixed
    point and every later pass would repeat it. Returns labels, T, the last scores'
    top1-top2 margin and the label changes per pass (its length = the passes run)."""
    n, k = Phi.shape
    T = np.eye(k)
    labels = np.zeros(n, dtype=np.int64)
    margin = np.full(n, np.inf)
    changes = []
    prev = None
    for _ in range(t_g):
        S = Phi @ T
        labels = np.argmax(S, axis=1)
        if k > 1:
            top2 = np.partition(S, k - 2, axis=1)[:, k - 2:]
            margin = top2[:, 1] - top2[:, 0]
        changes.append(n if prev is None else int(np.count_nonzero(labels != prev)))
        prev = labels
        Y = nci_matrix(labels, k)
        M = np.asarray((Y.T @ Phi).T)
        T = polar(M) if procrustes else M
        if early_stop and len(changes) > 1 and changes[-1] == 0:
            break
    return labels.astype(np.int32), T, margin, changes


# ----------------------------------------------------------------------------
# Eq. 8: the k-ABGC objective with S := R R^T
# ----------------------------------------------------------------------------

def objective(R: np.ndarray, labels: np.ndarray, k: int) -> tuple[float, float]:
    """obj1 = sum_l (1/|C_l|) sum_{i in C_l, j not in C_l} R[i].R[j] (Eq. 8 with R13) and
    J = Tr(Y^T R R^T Y); both through the per-cluster sums s_l = sum_{i in C_l} R[i]."""
    n = R.shape[0]
    counts = np.bincount(labels, minlength=k).astype(np.float64)
    onehot = sp.csr_matrix((np.ones(n), (np.arange(n), labels)), shape=(n, k))
    s = np.asarray(onehot.T @ R)          # k x m
    total = R.sum(axis=0)
    obj1 = 0.0
    J = 0.0
    for l in range(k):
        if counts[l] > 0:
            obj1 += float(s[l] @ (total - s[l])) / counts[l]
            J += float(s[l] @ s[l]) / counts[l]
    return obj1, J


# ----------------------------------------------------------------------------
# the whole pipeline
# ----------------------------------------------------------------------------

def attributes_of(g) -> np.ndarray | sp.csr_matrix:
    """X_U as float64: dense for dense inputs, CSR for sparse ones (exact stored values)."""
    if g.x_kind == "csr_f32":
        return sp.csr_matrix((g.x_val.astype(np.float64), g.x_idx, g.x_ptr), shape=(g.n_u, g.d_u))
    return g.x_dense_f64()


def tpo(g, k: int, alpha: float, gamma: int, d: int | None = None, t_f: int = 5, t_g: int = 20,
        seed: int = 0, oversample: int = 10, power_iters: int = 4, procrustes: bool = False,
        early_stop: bool = False) -> dict:
    """Algorithms 1-3 end to end on the graph ``g`` (a synth.ABG-like object)."""
    d = g.d_u if d is None else d
    if not (1 <= d <= g.d_u):
        raise ValueError("need 1 <= d <= d_u")
    if not (1 <= k <= min(g.n_u, 2 * d)):
        raise ValueError("need 1 <= k <= min(|U|, 2d)")
    B = adjacency(g.n_u, g.n_v, g.u_ptr, g.v_idx, g.w)
    L = normalized_adjacency(B)
    X = attributes_of(g)
    if d < g.d_u:
        X = reduce_attributes(X, d, seed, oversample, power_iters)
    elif sp.issparse(X):
        X = X.toarray()
    Z = propagate(L, X, alpha, gamma)
    Zhat = normalize_rows(Z)
    Q = orthogonal_matrix(seed, d)
    Rp, r, R, clamped = random_features(Zhat, Q)
    Phi0, H0, Sigma = seed_factors(R, k, seed, oversample, power_iters)
    Phi, H = onmf(R, Phi0, H0, t_f)
    labels, T, margin, changes = nci(Phi, t_g, procrustes, early_stop)
    obj1, J = objective(R, labels, k)
    return dict(X=X, Z=Z, Zhat=Zhat, Q=Q, R=R, r=r, clamped=clamped, Sigma=Sigma, Phi0=Phi0,
                H0=H0, Phi=Phi, H=H, labels=labels, T=T, margin=margin, changes=changes,
                objective=obj1, trace_obj=J)
