"""Planted-partition attributed bipartite graphs (ABGs) for the five workloads.

Every graph is drawn from a counter-based bit generator (numpy's Philox,
keyed through a SeedSequence of integers), so a (config, graph, stream) key
gives the same arrays on every machine. The shapes follow the paper's
workloads (Table 2: a few thousand to a few million U nodes, power-law
degrees, sparse or dense attributes); the datasets themselves are not used.

Structure shared by all configs
  * cluster of u_i: ``i mod k`` (balanced), returned as ``truth``;
  * V is cut into k contiguous blocks; an edge from u (cluster c) lands in
    block c with probability ``p_in``, otherwise anywhere in V;
  * inside the chosen range the V endpoint is drawn proportionally to a
    Chung-Lu weight ``(rank+1)^(-1/(a-1))`` (rank = a random permutation,
    so hubs are spread over the blocks), or uniformly when no exponent is
    given;
  * repeated (u, v) draws are merged into one edge whose weight is the
    multiplicity (except workload 1, which redraws to keep unit weights).

Nothing here computes any step of the clustering method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Default method parameters per workload (alpha, gamma, reduced d, T_f, T_g).
CONFIG_PARAMS = {
    1: dict(k=5, alpha=0.6, gamma=6, d=500, t_f=5, t_g=20),
    2: dict(k=20, alpha=0.6, gamma=6, d=128, t_f=5, t_g=20),
    3: dict(k=100, alpha=0.9, gamma=10, d=128, t_f=5, t_g=20),
    4: dict(alpha=0.6, gamma=6, d=32, t_f=5, t_g=20),
    5: dict(alpha=0.6, gamma=6, t_f=5, t_g=20),
}


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(x) for x in key])))


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even); returns uint16 bit patterns."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    rounding = ((b >> 16) & 1) + np.uint32(0x7FFF)
    return ((b + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(h: np.ndarray) -> np.ndarray:
    return (h.astype(np.uint32) << 16).view(np.float32)


@dataclass
class ABG:
    """One attributed bipartite graph in CSR form (rows = U) plus attributes."""

    name: str
    n_u: int
    n_v: int
    u_ptr: np.ndarray            # int64 [n_u + 1]
    v_idx: np.ndarray            # int32 [nnz], sorted within each row
    w: np.ndarray | None         # float32 [nnz]; None = unit weights
    d_u: int
    x_kind: str                  # "dense_f32" | "dense_bf16" | "csr_f32"
    x: np.ndarray | None = None  # dense: float32 [n_u, d_u] or uint16 bf16 bits
    x_ptr: np.ndarray | None = None   # csr: int64 [n_u + 1]
    x_idx: np.ndarray | None = None   # csr: int32
    x_val: np.ndarray | None = None   # csr: float32
    k: int = 2
    truth: np.ndarray | None = None   # int32 [n_u]
    params: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.u_ptr[-1])

    def weights_f64(self) -> np.ndarray:
        if self.w is None:
            return np.ones(self.nnz, dtype=np.float64)
        return self.w.astype(np.float64)

    def x_dense_f64(self) -> np.ndarray:
        """Attributes as exact float64 values (the stored numbers, widened)."""
        if self.x_kind == "dense_f32":
            return self.x.astype(np.float64)
        if self.x_kind == "dense_bf16":
            return bf16_bits_to_f32(self.x).astype(np.float64)
        out = np.zeros((self.n_u, self.d_u), dtype=np.float64)
        rows = np.repeat(np.arange(self.n_u), np.diff(self.x_ptr))
        np.add.at(out, (rows, self.x_idx), self.x_val.astype(np.float64))
        return out

    def x_nnz(self) -> int:
        return int(self.x_ptr[-1]) if self.x_kind == "csr_f32" else self.n_u * self.d_u


# ----------------------------------------------------------------------------
# edge builders
# ----------------------------------------------------------------------------

def _powerlaw_weights(n: int, exponent: float | None, rng: np.random.Generator) -> np.ndarray:
    if exponent is None:
        return np.ones(n, dtype=np.float64)
    rank = rng.permutation(n).astype(np.float64)
    return (rank + 1.0) ** (-1.0 / (exponent - 1.0))


def _draw_in_ranges(cum: np.ndarray, lo: np.ndarray, hi: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Index j in [lo, hi) drawn with probability w_j / sum(w[lo:hi]) (cum = prefix sums)."""
    t = cum[lo] + u * (cum[hi] - cum[lo])
    j = np.searchsorted(cum, t, side="right") - 1
    return np.clip(j, lo, hi - 1)


def _block_bounds(c: np.ndarray, n_v: int, k: int) -> tuple[np.ndarray, np.ndarray]:
    lo = (c.astype(np.int64) * n_v) // k
    hi = ((c.astype(np.int64) + 1) * n_v) // k
    return lo, hi


def _sample_edges(rng, n_u, n_v, k, truth, src_u, p_in, v_exponent):
    """V endpoints for the edge sources ``src_u`` (one draw per entry)."""
    wv = _powerlaw_weights(n_v, v_exponent, rng)
    cum = np.concatenate([[0.0], np.cumsum(wv)])
    m = src_u.shape[0]
    inside = rng.random(m) < p_in
    lo, hi = _block_bounds(truth[src_u], n_v, k)
    lo = np.where(inside, lo, 0)
    hi = np.where(inside, hi, n_v)
    return _draw_in_ranges(cum, lo, hi, rng.random(m))


def _coalesce(n_u, n_v, src_u, dst_v):
    key = src_u.astype(np.int64) * np.int64(n_v) + dst_v.astype(np.int64)
    key, counts = np.unique(key, return_counts=True)
    u = key // n_v
    v = (key % n_v).astype(np.int32)
    u_ptr = np.zeros(n_u + 1, dtype=np.int64)
    np.cumsum(np.bincount(u, minlength=n_u), out=u_ptr[1:])
    return u_ptr, v, counts.astype(np.float32)


def _binary_attributes(rng, n_u, d, k, truth, density, subset, boost):
    """Sparse 0/1 attributes: Bernoulli(density), x``boost`` on a per-cluster column window."""
    sub_lo = (truth.astype(np.int64) * d) // k
    rows, cols = [], []
    # draw row by row in blocks to bound memory
    block = max(1, 2_000_000 // d)
    for r0 in range(0, n_u, block):
        r1 = min(n_u, r0 + block)
        p = np.full((r1 - r0, d), density)
        off = (np.arange(d)[None, :] - sub_lo[r0:r1, None]) % d
        p[off < subset] = min(1.0, density * boost)
        hit = rng.random((r1 - r0, d)) < p
        rr, cc = np.nonzero(hit)
        rows.append(rr + r0)
        cols.append(cc)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols).astype(np.int32)
    x_ptr = np.zeros(n_u + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n_u), out=x_ptr[1:])
    return x_ptr, cols, np.ones(cols.shape[0], dtype=np.float32)


def _tfidf_attributes(rng, n_u, d, k, truth, per_row, subset, boost):
    """Sparse lognormal(0,1) attributes with exactly ``per_row`` distinct columns, rows L2-normalised."""
    n_cand = per_row + 8
    sub_lo = (truth.astype(np.int64) * d) // k
    # column draw: with prob (subset*boost)/(subset*boost + d - subset) inside the cluster window
    p_sub = subset * boost / (subset * boost + (d - subset))
    in_sub = rng.random((n_u, n_cand)) < p_sub
    c_sub = (sub_lo[:, None] + rng.integers(0, subset, (n_u, n_cand))) % d
    c_out = (sub_lo[:, None] + subset + rng.integers(0, d - subset, (n_u, n_cand))) % d
    cand = np.where(in_sub, c_sub, c_out)
    dup = np.zeros_like(cand, dtype=bool)
    for j in range(1, n_cand):
        dup[:, j] = (cand[:, :j] == cand[:, j:j + 1]).any(axis=1)
    order = np.argsort(dup, axis=1, kind="stable")[:, :per_row]
    cols = np.take_along_axis(cand, order, axis=1)
    ok = ~np.take_along_axis(dup, order, axis=1)
    for i in np.nonzero(~ok.all(axis=1))[0]:  # rare: fewer than per_row distinct candidates
        cols[i] = rng.choice(d, per_row, replace=False)
    cols = np.sort(cols, axis=1).astype(np.int32)
    vals = rng.lognormal(0.0, 1.0, (n_u, per_row))
    vals /= np.linalg.norm(vals, axis=1, keepdims=True)
    x_ptr = np.arange(0, n_u * per_row + 1, per_row, dtype=np.int64)
    return x_ptr, cols.reshape(-1), vals.reshape(-1).astype(np.float32)


def _gaussian_mixture_bf16(rng, n_u, d, k, truth, sigma):
    mu = rng.standard_normal((k, d), dtype=np.float32)
    out = np.empty((n_u, d), dtype=np.uint16)
    block = 1 << 18
    for r0 in range(0, n_u, block):
        r1 = min(n_u, r0 + block)
        noise = rng.standard_normal((r1 - r0, d), dtype=np.float32)
        out[r0:r1] = f32_to_bf16_bits(mu[truth[r0:r1]] + np.float32(sigma) * noise)
    return out


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def make_config1(seed: int = 0) -> ABG:
    """|U|=2,000, |V|=3,000, k=5, 20,000 unit edges (10 distinct neighbours per u,
    80% in own block), binary attributes d=500 at 2% with a 50-column cluster window at 5x."""
    n_u, n_v, k, deg = 2000, 3000, 5, 10
    rng = _rng(seed, 1, 0)
    truth = (np.arange(n_u) % k).astype(np.int32)
    v_idx = np.empty(n_u * deg, dtype=np.int32)
    for i in range(n_u):
        lo, hi = (truth[i] * n_v) // k, ((truth[i] + 1) * n_v) // k
        picked: list[int] = []
        while len(picked) < deg:
            v = int(rng.integers(lo, hi)) if rng.random() < 0.8 else int(rng.integers(0, n_v))
            if v not in picked:
                picked.append(v)
        v_idx[i * deg:(i + 1) * deg] = np.sort(picked)
    u_ptr = np.arange(0, n_u * deg + 1, deg, dtype=np.int64)
    x_ptr, x_idx, x_val = _binary_attributes(_rng(seed, 1, 1), n_u, 500, k, truth, 0.02, 50, 5.0)
    return ABG("config1", n_u, n_v, u_ptr, v_idx, None, 500, "csr_f32", None, x_ptr, x_idx, x_val,
               k, truth, dict(CONFIG_PARAMS[1]))


def make_config2(seed: int = 0, scale: float = 1.0) -> ABG:
    """|U|=200k, |V|=500k, k=20, 5M edge draws (u-degree 25), Zipf(2.1) V weights, 70/30 mixing;
    TF-IDF-like attributes d=1,000 with 10 lognormal entries per row, rows unit-norm."""
    n_u, n_v, k = int(200_000 * scale), int(500_000 * scale), 20
    rng = _rng(seed, 2, 0)
    truth = (np.arange(n_u) % k).astype(np.int32)
    src = np.repeat(np.arange(n_u, dtype=np.int64), 25)
    dst = _sample_edges(rng, n_u, n_v, k, truth, src, 0.7, 2.1)
    u_ptr, v_idx, w = _coalesce(n_u, n_v, src, dst)
    x_ptr, x_idx, x_val = _tfidf_attributes(_rng(seed, 2, 1), n_u, 1000, k, truth, 10, 100, 5.0)
    return ABG(f"config2(x{scale:g})", n_u, n_v, u_ptr, v_idx, w, 1000, "csr_f32", None,
               x_ptr, x_idx, x_val, k, truth, dict(CONFIG_PARAMS[2]))


def make_config3(seed: int = 0, scale: float = 1.0, k: int | None = None) -> ABG:
    """|U|=2M, |V|=5M, k=100, 50M edge draws, Chung-Lu exponent 2.2 on both sides, 60/40 mixing;
    dense Gaussian-mixture attributes d=128 (means N(0,1), noise sigma 1.5) stored as BF16.
    ``scale`` shrinks |U|, |V| and the edge count together (same structure)."""
    n_u, n_v = int(2_000_000 * scale), int(5_000_000 * scale)
    m = int(50_000_000 * scale)
    k = 100 if k is None else k
    rng = _rng(seed, 3, 0)
    truth = (np.arange(n_u) % k).astype(np.int32)
    wu = _powerlaw_weights(n_u, 2.2, rng)
    cu = np.concatenate([[0.0], np.cumsum(wu)])
    src = np.searchsorted(cu, rng.random(m) * cu[-1], side="right") - 1
    src = np.clip(src, 0, n_u - 1)
    dst = _sample_edges(rng, n_u, n_v, k, truth, src, 0.6, 2.2)
    u_ptr, v_idx, w = _coalesce(n_u, n_v, src, dst)
    del src, dst
    x = _gaussian_mixture_bf16(_rng(seed, 3, 1), n_u, 128, k, truth, 1.5)
    params = dict(CONFIG_PARAMS[3])
    params["k"] = k
    return ABG(f"config3(x{scale:g})", n_u, n_v, u_ptr, v_idx, w, 128, "dense_bf16", x,
               None, None, None, k, truth, params)


def make_config4_graph(g: int, seed: int = 0) -> ABG:
    """One of the 512 batched graphs: |U| log-uniform in [500, 50,000], |V|=1.5|U|, 10 edge draws
    per u (80% in own block, uniform weights), k uniform in [3, 30], binary attributes d=300 at 3%."""
    rng = _rng(seed, 4, g)
    n_u = int(np.floor(np.exp(rng.uniform(np.log(500), np.log(50_000)))))
    n_v = int(1.5 * n_u)
    k = int(rng.integers(3, 31))
    truth = (np.arange(n_u) % k).astype(np.int32)
    src = np.repeat(np.arange(n_u, dtype=np.int64), 10)
    dst = _sample_edges(rng, n_u, n_v, k, truth, src, 0.8, None)
    u_ptr, v_idx, w = _coalesce(n_u, n_v, src, dst)
    x_ptr, x_idx, x_val = _binary_attributes(rng, n_u, 300, k, truth, 0.03, min(50, 300 // k), 5.0)
    params = dict(CONFIG_PARAMS[4])
    params["k"] = k
    return ABG(f"config4[{g}]", n_u, n_v, u_ptr, v_idx, w, 300, "csr_f32", None, x_ptr, x_idx,
               x_val, k, truth, params)


def make_config5_request(r: int, seed: int = 0, max_u: int = 1_000_000) -> ABG:
    """One served request: workload-2-style edges with |U| log-uniform in [1,000, max_u],
    |V| = 2.5|U|, k uniform in [5, 100]; half dense d=128 (BF16), half sparse d=500 at 1%
    (reduced to d=64)."""
    rng = _rng(seed, 5, r)
    n_u = int(np.floor(np.exp(rng.uniform(np.log(1000), np.log(max_u)))))
    n_v = int(2.5 * n_u)
    k = int(rng.integers(5, 101))
    dense = bool(rng.random() < 0.5)
    truth = (np.arange(n_u) % k).astype(np.int32)
    src = np.repeat(np.arange(n_u, dtype=np.int64), 25)
    dst = _sample_edges(rng, n_u, n_v, k, truth, src, 0.7, 2.1)
    u_ptr, v_idx, w = _coalesce(n_u, n_v, src, dst)
    params = dict(CONFIG_PARAMS[5])
    params["k"] = min(k, n_u)
    if dense:
        x = _gaussian_mixture_bf16(rng, n_u, 128, k, truth, 1.5)
        params["d"] = 128
        return ABG(f"config5[{r}]", n_u, n_v, u_ptr, v_idx, w, 128, "dense_bf16", x, None, None,
                   None, k, truth, params)
    x_ptr, x_idx, x_val = _tfidf_attributes(rng, n_u, 500, k, truth, 5, max(1, 500 // k), 5.0)
    params["d"] = 64
    return ABG(f"config5[{r}]", n_u, n_v, u_ptr, v_idx, w, 500, "csr_f32", None, x_ptr, x_idx,
               x_val, k, truth, params)


def config5_arrivals(n: int, rate: float = 200.0, seed: int = 1) -> np.ndarray:
    """Poisson arrival times (seconds) of ``n`` requests: exponential gaps of mean 1/rate."""
    return np.cumsum(_rng(seed, 5, 1 << 30).exponential(1.0 / rate, n))


def make_small(seed: int, n_u: int = 40, n_v: int = 60, k: int = 3, d_u: int = 8,
               deg: int = 4, p_in: float = 0.8, weighted: bool = True, x_kind: str = "dense_f32",
               isolated_u: int = 0, isolated_v: int = 0, v_exponent: float | None = None,
               signal: float = 2.0) -> ABG:
    """Tiny planted graph for tests: optional non-unit weights, isolated nodes on either side,
    dense float32 / bf16 or CSR attributes."""
    rng = _rng(seed, 99, n_u * 1000 + n_v)
    truth = (np.arange(n_u) % k).astype(np.int32)
    active = n_u - isolated_u
    src = np.repeat(np.arange(active, dtype=np.int64), deg)
    n_v_active = n_v - isolated_v
    dst = _sample_edges(rng, active, n_v_active, k, truth[:active], src, p_in, v_exponent)
    u_ptr_a, v_idx, w = _coalesce(active, n_v_active, src, dst)
    u_ptr = np.concatenate([u_ptr_a, np.full(isolated_u, u_ptr_a[-1], dtype=np.int64)])
    if weighted:
        w = (w * rng.uniform(0.5, 2.0, w.shape[0])).astype(np.float32)
    else:
        w = None
    mu = rng.standard_normal((k, d_u)) * signal
    xd = (mu[truth] + rng.standard_normal((n_u, d_u))).astype(np.float32)
    params = dict(k=k, alpha=0.6, gamma=4, d=d_u, t_f=5, t_g=10)
    if x_kind == "dense_f32":
        return ABG("small", n_u, n_v, u_ptr, v_idx, w, d_u, x_kind, xd, k=k, truth=truth,
                   params=params)
    if x_kind == "dense_bf16":
        return ABG("small", n_u, n_v, u_ptr, v_idx, w, d_u, x_kind, f32_to_bf16_bits(xd), k=k,
                   truth=truth, params=params)
    keep = rng.random((n_u, d_u)) < 0.5
    xs = np.where(keep, np.abs(xd), 0.0).astype(np.float32)
    rr, cc = np.nonzero(xs)
    x_ptr = np.zeros(n_u + 1, dtype=np.int64)
    np.cumsum(np.bincount(rr, minlength=n_u), out=x_ptr[1:])
    return ABG("small", n_u, n_v, u_ptr, v_idx, w, d_u, "csr_f32", None, x_ptr,
               cc.astype(np.int32), xs[rr, cc].astype(np.float32), k, truth, params)
