"""BF16 storage of the propagation's intermediate blocks (ABG_BF16_PROPAGATION): W = L^T Z and the
Z of rounds 1..gamma-1 are rounded to BF16 (nearest even) when stored; every sparse product still
accumulates in FP32 and Z_hat is FP32.

Two references:
  * the FP64 oracle followed by BF16 rounding at exactly the stored points (the emulation below,
    test-side, built from the oracle's L): the GPU result differs from it only by FP32 summation
    order, except where that order moves a stored value across a BF16 rounding boundary (one
    BF16 ulp, 2^-8 relative, in that entry). Bound: at most 1% of the entries differ by more than
    1e-5 and none by more than 2^-8 (measured on the graphs below: <= 0.09% and 3.1e-4).
  * the plain FP64 oracle: each stored entry carries a relative error <= 2^-9, and each round
    contracts earlier errors by alpha (||L|| <= 1), so the row-normalised Z_hat moves by
    O(2^-9 alpha / (1 - alpha)) per row. Bound: every row within 2^-7 in 2-norm (measured
    <= 2.3e-3 at alpha = 0.9, gamma = 10).
Solves: labels identical to the oracle's wherever its top1 - top2 margin exceeds 1e-2, the
objective within 1e-4 relative (measured: labels identical above 1e-4, objective <= 1.0e-5).
"""
import numpy as np
import pytest

import synth
from oracle import tpo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402

DEV = torch.device("cuda:0")

GRAPHS = {
    "weighted": lambda: synth.make_small(1, n_u=120, n_v=150, k=3, d_u=10, deg=5),
    "isolated": lambda: synth.make_small(2, n_u=90, n_v=130, k=3, d_u=7, isolated_u=4,
                                         isolated_v=6, weighted=False),
    "bf16_x": lambda: synth.make_small(3, n_u=200, n_v=260, k=4, d_u=32, x_kind="dense_bf16"),
    "csr_x": lambda: synth.make_small(4, n_u=150, n_v=170, k=3, d_u=24, x_kind="csr_f32"),
    "heavy": lambda: synth.make_config3(scale=0.005, k=10),
    "gather_f32": lambda: synth.make_small(10, n_u=3000, n_v=4100, k=4, d_u=100, deg=9,
                                           isolated_u=70, isolated_v=90),
    "gather_bf16": lambda: synth.make_small(11, n_u=2500, n_v=3000, k=4, d_u=72, deg=6,
                                            x_kind="dense_bf16", isolated_u=40),
    "gather_wide": lambda: synth.make_small(12, n_u=1200, n_v=1500, k=3, d_u=200, deg=7,
                                            isolated_v=50),
}


def _bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even)."""
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()


def emulate(L, X, alpha, gamma):
    """The oracle's propagation with BF16 rounding where the GPU path stores BF16: W after each
    L^T product, Z after every round but the last."""
    Z = (1 - alpha) * X
    Zs = None
    for t in range(gamma):
        W = _bf16((1 - alpha) * (L.T @ X) if t == 0 else L.T @ Zs)
        Z = (1 - alpha) * X + alpha * (L @ W)
        if t < gamma - 1:
            Zs = _bf16(Z)
    return Z


@pytest.fixture(scope="module", params=list(GRAPHS))
def graph(request):
    g = GRAPHS[request.param]()
    h = abg.abg_create(g)
    L = tpo.normalized_adjacency(tpo.adjacency(g.n_u, g.n_v, g.u_ptr, g.v_idx, g.w))
    X = tpo.attributes_of(g)
    X = X.toarray() if hasattr(X, "toarray") else X
    yield g, h, L, X
    h.close()


def _run(h, g, alpha, gamma, bf16):
    ld = ((g.d_u + 3) // 4) * 4
    zh = torch.zeros((g.n_u, ld), dtype=torch.float32, device=DEV)
    abg.abg_propagate(h, None, g.d_u, alpha, gamma, zh, bf16_propagation=bf16)
    torch.cuda.synchronize()
    return zh[:, :g.d_u].double().cpu().numpy()


@pytest.mark.parametrize("alpha,gamma", [(0.6, 6), (0.9, 10), (0.5, 1), (0.3, 2)])
def test_bf16_propagation(graph, alpha, gamma):
    g, h, L, X = graph
    got = _run(h, g, alpha, gamma, True)
    em = tpo.normalize_rows(emulate(L, X, alpha, gamma))
    diff = np.abs(got - em)
    assert (diff > 1e-5).mean() <= 1e-2
    assert diff.max() <= 2.0 ** -8
    ref = tpo.normalize_rows(tpo.propagate(L, X, alpha, gamma))
    assert np.linalg.norm(got - ref, axis=1).max() <= 2.0 ** -7


@pytest.mark.parametrize("alpha,gamma", [(0.0, 5), (0.7, 0)])
def test_bf16_propagation_exact_cases(graph, alpha, gamma):
    # alpha = 0 (Z = X) and gamma = 0 store nothing in BF16 that reaches Z_hat: same bits
    g, h, _, _ = graph
    assert np.array_equal(_run(h, g, alpha, gamma, True), _run(h, g, alpha, gamma, False))


@pytest.mark.parametrize("name,p", [
    ("weighted", dict(k=3, alpha=0.6, gamma=4, d=10, t_f=5, t_g=10, seed=1)),
    ("bf16_x", dict(k=4, alpha=0.6, gamma=4, d=32, t_f=5, t_g=10, seed=1)),
    ("gather_f32", dict(k=4, alpha=0.6, gamma=6, d=100, t_f=5, t_g=20, seed=0)),
    ("heavy", dict(k=10, alpha=0.9, gamma=10, d=128, t_f=5, t_g=20, seed=0)),
])
def test_solve_bf16_propagation(name, p):
    g = GRAPHS[name]()
    h = abg.abg_create(g)
    lab, res = abg.abg_cluster(h, abg.params(**p, bf16_propagation=True))
    h.close()
    ref = tpo.tpo(g, **p)
    sure = ref["margin"] > 1e-2
    assert np.array_equal(lab[sure], ref["labels"][sure])
    assert res.objective == pytest.approx(ref["objective"], rel=1e-4)


def test_bf16_propagation_batched_equals_alone():
    graphs = [synth.make_small(300 + i, n_u=n, n_v=int(1.3 * n), k=3, d_u=24, deg=6, signal=3.0)
              for i, n in enumerate([80, 700, 2500])]
    ps = [abg.params(k=3, alpha=0.6, gamma=5, t_f=4, t_g=8, seed=i, bf16_propagation=True)
          for i in range(3)]
    b = abg.abg_batch_create(graphs)
    labels, results = abg.abg_batch_cluster(b, ps)
    b.close()
    off = np.cumsum([0] + [g.n_u for g in graphs])
    for i, (g, p, r) in enumerate(zip(graphs, ps, results)):
        h = abg.abg_create(g)
        l1, r1 = abg.abg_cluster(h, p)
        h.close()
        assert np.array_equal(labels[off[i]:off[i + 1]], l1) and r.objective == r1.objective
    # one batch cannot mix storage precisions
    mixed = [abg.params(k=3, alpha=0.6, gamma=5, t_f=4, t_g=8, seed=i,
                        bf16_propagation=(i == 0)) for i in range(3)]
    b = abg.abg_batch_create(graphs)
    with pytest.raises(abg.AbgError) as e:
        abg.abg_batch_cluster(b, mixed)
    assert e.value.status == abg.ABG_EINVAL
    b.close()


# ---------------------------------------------------------------------------
# ABG_BF16_CONTRACT: the products with R (randomized SVD of Algorithm 2, Eqs. 16-17) on the
# BF16 tensor-core kernels, R read as a BF16 copy, the small operand rounded to BF16, FP32
# accumulation.
# ---------------------------------------------------------------------------
def _dev(a):
    a = np.asarray(a)
    r, c = a.shape
    t = torch.zeros((r, ((c + 3) // 4) * 4), dtype=torch.float32, device=DEV)
    t[:, :c] = torch.as_tensor(a, dtype=torch.float32)
    return t


def _host(t, c):
    torch.cuda.synchronize()
    return t[:, :c].double().cpu().numpy()


def test_onmf_step_bf16_contract_emulated():
    # one pass of Eqs. 16-17 against the same pass in FP64 on BF16-rounded operands where the
    # kernels round: A = bf16(R)^T bf16(Phi) (nothing rounded after it, so H follows A to the
    # tensor cores' FP32 accumulation error: 3e-5, measured 1.4e-5, where the FP32 path is
    # 8.5e-5 away), P = bf16(R) bf16(H') (a summation-order change can move an H' entry
    # across a BF16 rounding boundary: Phi within 2^-7, 99% of it within 1e-4)
    g = synth.make_small(31, n_u=2500, n_v=3000, k=7, d_u=24, deg=6, signal=3.0)
    p = dict(k=7, alpha=0.6, gamma=4, d=24, t_f=5, t_g=10, seed=3)
    ref = tpo.tpo(g, **p)
    R = ref["R"].astype(np.float32).astype(np.float64)
    P0 = ref["Phi0"].astype(np.float32).astype(np.float64)
    H0 = ref["H0"].astype(np.float32).astype(np.float64)
    n, m, k = R.shape[0], R.shape[1], p["k"]
    phi, H = _dev(P0), _dev(H0)
    abg.abg_onmf(_dev(R), n, m, k, 1, phi, H, bf16_contract=True)
    A = _bf16(R).T @ _bf16(P0)
    den = H0 @ (P0.T @ P0)
    He = np.where(den > 0, H0 * np.maximum(A, 0) / np.where(den > 0, den, 1), 0.0)
    P = _bf16(R) @ _bf16(He)
    C = A.T @ He
    den = P0 @ C
    Pe = np.where(den > 0, P0 * np.sqrt(np.maximum(P, 0) / np.where(den > 0, den, 1)), 0.0)
    Hg, Pg = _host(H, k), _host(phi, k)
    assert np.abs(Hg - He).max() <= 3e-5 * np.abs(He).max()
    rel = np.abs(Pg - Pe) / np.abs(Pe).max()
    assert (rel > 1e-4).mean() <= 1e-2 and rel.max() <= 2.0 ** -7
    # and the BF16 path did run: the unrounded pass is further away
    Pr, Hr = tpo.onmf(R, P0, H0, 1)
    assert np.abs(Hg - Hr).max() > 3e-5 * np.abs(Hr).max()


@pytest.mark.parametrize("n,m,k,ratio", [(2000, 40, 6, 0.6), (20000, 256, 100, 0.97),
                                         (5000, 200, 30, 0.9)])
def test_seed_factors_bf16_contract(n, m, k, ratio):
    # rounding A (and the small operands) to BF16 perturbs each product by <= 2^-9 of its
    # operands: by Weyl the singular values move by <= 2 * 2^-9 ||A||_F (measured <= 2.3e-4
    # sigma_1); singular vectors separated by a gap move by <= that / gap (Davis-Kahan)
    rng = np.random.default_rng(n + m)
    U = np.linalg.qr(rng.standard_normal((n, m)))[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    s = ratio ** np.arange(m) * 10
    A = ((U * s) @ V.T).astype(np.float32).astype(np.float64)
    phi, H = torch.zeros((n, ((k + 3) // 4) * 4), device=DEV), torch.zeros((m, ((k + 3) // 4) * 4), device=DEV)
    sig = torch.zeros(k, dtype=torch.float64, device=DEV)
    abg.abg_seed_factors(_dev(A), n, m, k, phi, H, sig, seed=4, bf16_contract=True)
    P0, H0, S0 = tpo.seed_factors(A, k, 4)
    eps = 2.0 ** -8 * np.linalg.norm(A)
    assert np.abs(sig.cpu().numpy() - S0).max() <= eps
    gaps = np.abs(np.diff(s[:k + 1]))
    gap = np.minimum(np.r_[np.inf, gaps[:-1]], gaps)       # distance to both neighbours
    P, Hh = _host(phi, k), _host(H, k)
    for j in range(k):
        if eps / gap[j] < 0.05:                            # well separated
            assert np.abs(P[:, j] - P0[:, j]).max() <= 4 * eps / gap[j]
            assert np.abs(Hh[:, j] - H0[:, j]).max() <= 4 * eps / gap[j] * s[0] + eps


SOLVES_BF16 = [
    ("weighted", dict(k=3, alpha=0.6, gamma=4, d=10, t_f=5, t_g=10, seed=1)),
    ("bf16_x", dict(k=4, alpha=0.6, gamma=4, d=32, t_f=5, t_g=10, seed=1)),
    ("gather_f32", dict(k=4, alpha=0.6, gamma=6, d=100, t_f=5, t_g=20, seed=0)),
    ("heavy", dict(k=10, alpha=0.9, gamma=10, d=128, t_f=5, t_g=20, seed=0)),
    ("reduce_bf16", dict(k=5, alpha=0.6, gamma=5, d=16, t_f=5, t_g=10, seed=2)),
    ("k100", dict(k=100, alpha=0.9, gamma=10, d=128, t_f=5, t_g=20, seed=0, procrustes=True)),
]
GRAPHS["reduce_bf16"] = lambda: synth.make_small(8, n_u=3000, n_v=4000, k=5, d_u=80,
                                                 x_kind="dense_bf16", signal=4.0)
GRAPHS["k100"] = lambda: synth.make_config3(scale=0.01)


@pytest.mark.parametrize("name,p", SOLVES_BF16)
def test_solve_bf16_contract(name, p):
    # labels identical where the oracle's margin exceeds 1e-2, objective within 2e-3
    # (measured: identical above 1e-2 everywhere, objective <= 2.3e-4)
    g = GRAPHS[name]()
    h = abg.abg_create(g)
    lab, res = abg.abg_cluster(h, abg.params(**p, bf16_contract=True))
    h.close()
    ref = tpo.tpo(g, **p)
    sure = ref["margin"] > 1e-2
    assert np.array_equal(lab[sure], ref["labels"][sure])
    assert res.objective == pytest.approx(ref["objective"], rel=2e-3)


def test_bf16_contract_batched_equals_alone():
    # a batch streams B with every stage (several segments); alone, B stays in shared memory:
    # the same BF16 operands and MMAs, so the same bits
    graphs = [synth.make_small(400 + i, n_u=n, n_v=int(1.3 * n), k=4, d_u=40, deg=6, signal=3.0)
              for i, n in enumerate([300, 2600, 900])]
    ps = [abg.params(k=4, alpha=0.6, gamma=5, t_f=4, t_g=8, seed=i, bf16_contract=True)
          for i in range(3)]
    b = abg.abg_batch_create(graphs)
    labels, results = abg.abg_batch_cluster(b, ps)
    b.close()
    off = np.cumsum([0] + [g.n_u for g in graphs])
    for i, (g, p, r) in enumerate(zip(graphs, ps, results)):
        h = abg.abg_create(g)
        l1, r1 = abg.abg_cluster(h, p)
        h.close()
        assert np.array_equal(labels[off[i]:off[i + 1]], l1) and r.objective == r1.objective
