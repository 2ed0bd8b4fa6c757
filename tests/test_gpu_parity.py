"""GPU parity: each step of the CUDA path against the FP64 oracle on the same seeded inputs,
called through the C ABI. Inputs handed to a GPU step come from the generator or from the
oracle (never the reverse).

Tolerances (FP32 kernels vs FP64 oracle; u = 2^-24 ~ 6e-8):
  * Z_hat: gamma rounds of sums of <= a few thousand products of numbers <= 1, each round a
    contraction (spectral radius of L L^T is 1): |dZ_hat| <= 2e-5.
  * R: sin/cos of arguments |sqrt(d) Zhat.q| <= sqrt(d) carry ~sqrt(d) * d * u error, then
    Eq. 14 rescales: max|dR| <= 2e-4 * max|R|.
  * NMF factors after t_f multiplicative steps: max|d| <= 1e-3 * max (growth of FP32 error
    through 5 nonlinear steps, measured < 1e-4).
  * labels: identical wherever the oracle's top1 - top2 margin exceeds 1e-4.
  * objective (FP64 sums of FP32 rows): relative 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import philox, tpo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a: np.ndarray, width: int | None = None, dtype=torch.float32):
    """Host matrix -> device tensor whose row stride is rounded up to 4 elements."""
    a = np.asarray(a)
    rows, cols = a.shape
    ld = ((cols + 3) // 4) * 4
    t = torch.zeros((rows, ld), dtype=dtype, device=DEV)
    t[:, :cols] = torch.as_tensor(a, dtype=dtype)
    return t


def empty(rows, cols, dtype=torch.float32):
    ld = ((cols + 3) // 4) * 4
    return torch.zeros((rows, ld), dtype=dtype, device=DEV)


def host(t, cols):
    torch.cuda.synchronize()
    return t[:, :cols].double().cpu().numpy()


GRAPHS = {
    "weighted": lambda: synth.make_small(1, n_u=120, n_v=150, k=3, d_u=10, deg=5),
    "isolated": lambda: synth.make_small(2, n_u=90, n_v=130, k=3, d_u=7, isolated_u=4,
                                         isolated_v=6, weighted=False),
    "bf16": lambda: synth.make_small(3, n_u=200, n_v=260, k=4, d_u=32, x_kind="dense_bf16"),
    "csr_x": lambda: synth.make_small(4, n_u=150, n_v=170, k=3, d_u=24, x_kind="csr_f32"),
    "heavy": lambda: synth.make_config3(scale=0.005, k=10),
    "wide": lambda: synth.make_small(5, n_u=160, n_v=200, k=3, d_u=300, deg=8),
    # rows of 17..64 float4 chunks take the TMA-gather kernel: f32 and bf16 rows, one and two
    # chunks per lane, runs of isolated rows (tasks without edges), several tasks per warp
    "gather_f32": lambda: synth.make_small(10, n_u=3000, n_v=4100, k=4, d_u=100, deg=9,
                                           isolated_u=70, isolated_v=90),
    "gather_bf16": lambda: synth.make_small(11, n_u=2500, n_v=3000, k=4, d_u=72, deg=6,
                                            x_kind="dense_bf16", isolated_u=40),
    "gather_wide": lambda: synth.make_small(12, n_u=1200, n_v=1500, k=3, d_u=200, deg=7,
                                            isolated_v=50),
}


@pytest.fixture(scope="module", params=list(GRAPHS))
def graph(request):
    g = GRAPHS[request.param]()
    h = abg.abg_create(g)
    yield g, h
    h.close()


def oracle_L(g):
    return tpo.normalized_adjacency(tpo.adjacency(g.n_u, g.n_v, g.u_ptr, g.v_idx, g.w))


@pytest.mark.parametrize("d", [1, 3, 5, 16, 64, 128, 130, 500])
def test_orthogonal_matrix(d):
    q = torch.empty((d, d), dtype=torch.float64, device=DEV)
    abg.abg_orthogonal_matrix(11, d, q)
    ref = tpo.orthogonal_matrix(11, d)
    assert np.abs(q.cpu().numpy() - ref).max() < 1e-11


@pytest.mark.parametrize("alpha,gamma", [(0.6, 6), (0.9, 10), (0.3, 0), (0.0, 2), (0.5, 1)])
def test_propagation(graph, alpha, gamma):
    g, h = graph
    d = g.d_u
    zh = empty(g.n_u, d)
    abg.abg_propagate(h, None, d, alpha, gamma, zh)
    X = tpo.attributes_of(g)
    X = X.toarray() if hasattr(X, "toarray") else X
    ref = tpo.normalize_rows(tpo.propagate(oracle_L(g), X, alpha, gamma))
    assert np.abs(host(zh, d) - ref).max() < 2e-5


def test_propagation_explicit_attributes(graph):
    # a caller-supplied X (here: the oracle's own values, narrower than the graph's d_u)
    g, h = graph
    rng = np.random.default_rng(0)
    X = rng.standard_normal((g.n_u, 6))
    zh = empty(g.n_u, 6)
    abg.abg_propagate(h, dev(X), 6, 0.7, 5, zh)
    ref = tpo.normalize_rows(tpo.propagate(oracle_L(g), X.astype(np.float32).astype(np.float64),
                                           0.7, 5))
    assert np.abs(host(zh, 6) - ref).max() < 2e-5


@pytest.mark.parametrize("n,d", [(50, 3), (300, 16), (1000, 128), (257, 500)])
def test_random_features(n, d):
    rng = np.random.default_rng(d)
    Zh = tpo.normalize_rows(rng.standard_normal((n, d))).astype(np.float32).astype(np.float64)
    Zh[7] = 0.0                                       # zero row (reading R3)
    R = empty(n, 2 * d)
    clamped = abg.abg_random_features(dev(Zh), n, d, 5, R)
    _, _, ref, cl_ref = tpo.random_features(Zh, tpo.orthogonal_matrix(5, d))
    assert clamped == cl_ref
    assert np.abs(host(R, 2 * d) - ref).max() <= 2e-4 * np.abs(ref).max()


def _pipeline_inputs(g, p):
    """The oracle's R for graph g (FP64), used as the input of the later GPU steps."""
    res = tpo.tpo(g, **p)
    return res


@pytest.fixture(scope="module")
def planted():
    g = synth.make_config1()
    p = dict(k=5, alpha=0.6, gamma=6, d=500, t_f=5, t_g=20, seed=0)
    return g, p, tpo.tpo(g, **p)


def test_seed_factors_well_separated():
    # spectrum with clear gaps: Gamma, Sigma, Psi are well defined, so Phi_0 and H_0 match
    rng = np.random.default_rng(3)
    n, m, k = 2000, 40, 6
    U = np.linalg.qr(rng.standard_normal((n, m)))[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    s = 0.6 ** np.arange(m) * 10
    A = (U * s) @ V.T
    A32 = A.astype(np.float32).astype(np.float64)
    phi, H = empty(n, k), empty(m, k)
    sig = torch.zeros(k, dtype=torch.float64, device=DEV)
    abg.abg_seed_factors(dev(A32), n, m, k, phi, H, sig, seed=9)
    P0, H0, S0 = tpo.seed_factors(A32, k, 9)
    assert np.allclose(sig.cpu().numpy(), S0, rtol=1e-5)
    assert np.abs(host(phi, k) - P0).max() <= 1e-4 * np.abs(P0).max()
    assert np.abs(host(H, k) - H0).max() <= 1e-4 * np.abs(H0).max()


def test_seed_factors_pipeline(planted):
    g, p, ref = planted
    R = ref["R"].astype(np.float32).astype(np.float64)
    n, m, k = R.shape[0], R.shape[1], p["k"]
    phi, H = empty(n, k), empty(m, k)
    sig = torch.zeros(k, dtype=torch.float64, device=DEV)
    abg.abg_seed_factors(dev(R), n, m, k, phi, H, sig, seed=p["seed"])
    P0, H0, S0 = tpo.seed_factors(R, k, p["seed"])
    assert np.allclose(sig.cpu().numpy(), S0, rtol=1e-5)
    # sigma_1(R) = 1 exactly: R R^T = D^-1/2 R' R'^T D^-1/2 with D = diag(R' r) has the
    # eigenvector D^1/2 1 with eigenvalue 1 (Eq. 14)
    assert abs(sig[0].item() - 1.0) < 1e-5
    # left/right factors: compare where the singular gaps are wide enough for FP32
    gaps = np.diff(-S0)
    ok = np.r_[gaps[0], np.minimum(gaps[:-1], gaps[1:]), gaps[-1]] / S0[0] > 5e-3
    P, Hh = host(phi, k), host(H, k)
    for j in np.nonzero(ok)[0]:
        assert np.abs(P[:, j] - P0[:, j]).max() <= 1e-3 * np.abs(P0).max()
        assert np.abs(Hh[:, j] - H0[:, j]).max() <= 1e-3 * np.abs(H0).max()


def test_onmf(planted):
    g, p, ref = planted
    R = ref["R"].astype(np.float32).astype(np.float64)
    P0 = ref["Phi0"].astype(np.float32).astype(np.float64)
    H0 = ref["H0"].astype(np.float32).astype(np.float64)
    n, m, k = R.shape[0], R.shape[1], p["k"]
    phi, H = dev(P0), dev(H0)
    abg.abg_onmf(dev(R), n, m, k, p["t_f"], phi, H)
    Pr, Hr = tpo.onmf(R, P0, H0, p["t_f"])
    assert np.abs(host(phi, k) - Pr).max() <= 1e-3 * np.abs(Pr).max()
    assert np.abs(host(H, k) - Hr).max() <= 1e-3 * np.abs(Hr).max()


@pytest.mark.parametrize("k", [1, 2, 5, 17, 64, 100, 128])
def test_nci(k):
    rng = np.random.default_rng(k)
    n = 3001
    lab = rng.integers(0, k, n)
    Phi = np.abs(0.3 * rng.standard_normal((n, k)) / np.sqrt(n))
    Phi[np.arange(n), lab] += 1.0 / np.sqrt(n / k)
    Phi[5] = 0.0                                      # tie everywhere -> cluster 0
    Phi = Phi.astype(np.float32).astype(np.float64)
    labels = torch.zeros(n, dtype=torch.int32, device=DEV)
    margin = torch.zeros(n, dtype=torch.float32, device=DEV)
    T = torch.zeros((k, k), dtype=torch.float64, device=DEV)
    abg.abg_nci(dev(Phi), n, k, 20, labels, margin, T)
    rl, rT, rm, _ = tpo.nci(Phi, 20)
    got = labels.cpu().numpy()
    sure = rm > 1e-4
    assert np.array_equal(got[sure], rl[sure])
    assert got[5] == 0
    if k > 1:
        assert np.abs(margin.cpu().numpy()[sure] - rm[sure]).max() < 1e-5
    assert np.abs(T.cpu().numpy() - rT).max() < 1e-5 * max(1.0, np.abs(rT).max())


def test_nci_pipeline(planted):
    g, p, ref = planted
    Phi = ref["Phi"].astype(np.float32).astype(np.float64)
    n, k = Phi.shape
    labels = torch.zeros(n, dtype=torch.int32, device=DEV)
    abg.abg_nci(dev(Phi), n, k, p["t_g"], labels)
    rl, _, rm, _ = tpo.nci(Phi, p["t_g"])
    sure = rm > 1e-4
    assert np.array_equal(labels.cpu().numpy()[sure], rl[sure])


@pytest.mark.parametrize("k,m", [(1, 8), (5, 1000), (100, 256), (128, 64)])
def test_objective(k, m):
    rng = np.random.default_rng(m + k)
    n = 5003
    R = rng.standard_normal((n, m)).astype(np.float32).astype(np.float64)
    lab = rng.integers(0, max(1, k - 1), n).astype(np.int32)   # leaves the last cluster empty
    obj = abg.abg_objective(dev(R), n, m, torch.as_tensor(lab, device=DEV), k)
    ref = tpo.objective(R, lab, k)
    assert obj[0] == pytest.approx(ref[0], rel=1e-5)
    assert obj[1] == pytest.approx(ref[1], rel=1e-5)


def test_attribute_reduction():
    g = synth.make_small(6, n_u=400, n_v=500, k=3, d_u=60, x_kind="csr_f32")
    h = abg.abg_create(g)
    d = 8
    X = tpo.attributes_of(g)
    ref = tpo.reduce_attributes(X, d, 3)
    out = empty(g.n_u, d)
    abg.abg_reduce_attributes(h, d, out, seed=3)
    s = np.linalg.svd(X.toarray(), compute_uv=False)
    got = host(out, d)
    # compare the columns whose singular value is separated from its neighbours
    gap = np.minimum(np.r_[np.inf, -np.diff(s[:d + 1])][:d], -np.diff(s[:d + 1])) / s[0]
    for j in np.nonzero(gap > 1e-2)[0]:
        assert np.abs(got[:, j] - ref[:, j]).max() <= 1e-3 * np.abs(ref).max()
    # X' X'^T approximates X X^T as well as the oracle's does
    e_got = np.linalg.norm(got @ got.T - X @ X.T.toarray())
    e_ref = np.linalg.norm(ref @ ref.T - X @ X.T.toarray())
    assert e_got <= e_ref * (1 + 1e-3) + 1e-6
    h.close()


def _end_to_end(g, p):
    h = abg.abg_create(g)
    labels, res = abg.abg_cluster(h, abg.params(**p))
    h.close()
    ref = tpo.tpo(g, **p)
    sure = ref["margin"] > 1e-4
    return labels, res, ref, sure


@pytest.mark.parametrize("name", ["weighted", "isolated", "bf16", "csr_x"])
def test_end_to_end_small(name):
    g = GRAPHS[name]()
    p = dict(k=g.k, alpha=0.6, gamma=4, d=g.d_u, t_f=5, t_g=10, seed=1)
    labels, res, ref, sure = _end_to_end(g, p)
    assert np.array_equal(labels[sure], ref["labels"][sure])
    assert res.objective == pytest.approx(ref["objective"], rel=1e-5)
    assert res.trace_obj == pytest.approx(ref["trace_obj"], rel=1e-5)


def test_end_to_end_config1(planted):
    g, p, ref = planted
    h = abg.abg_create(g)
    labels, res = abg.abg_cluster(h, abg.params(**p))
    h.close()
    sure = ref["margin"] > 1e-4
    assert np.array_equal(labels[sure], ref["labels"][sure])
    assert res.objective == pytest.approx(ref["objective"], rel=1e-5)


def test_end_to_end_reduced_attributes():
    g = synth.make_small(8, n_u=500, n_v=700, k=4, d_u=80, x_kind="csr_f32", signal=4.0)
    p = dict(k=4, alpha=0.6, gamma=5, d=12, t_f=5, t_g=10, seed=2)
    labels, res, ref, sure = _end_to_end(g, p)
    assert np.mean(labels[sure] == ref["labels"][sure]) == 1.0
    assert res.objective == pytest.approx(ref["objective"], rel=1e-5)


def test_edge_cases_end_to_end():
    g = synth.make_small(9, n_u=30, n_v=40, k=3, d_u=2, isolated_u=3)
    for p in [dict(k=1, alpha=0.5, gamma=3, d=2, t_f=2, t_g=3, seed=0),
              dict(k=4, alpha=0.0, gamma=0, d=2, t_f=0, t_g=1, seed=1),
              dict(k=3, alpha=0.6, gamma=2, d=2, t_f=3, t_g=0, seed=2)]:
        labels, res, ref, sure = _end_to_end(g, p)
        assert labels.min() >= 0 and labels.max() < p["k"]
        assert np.array_equal(labels[sure], ref["labels"][sure])
        assert res.objective == pytest.approx(ref["objective"], rel=1e-5, abs=1e-9)



def test_graph_without_edges_end_to_end():
    # every U node isolated: Z = (1 - alpha) X (Eq. 6 with L = 0, scales 0 by reading R2), so
    # the solve clusters the normalised attributes alone
    g = synth.make_small(11, n_u=30, n_v=40, k=3, d_u=4, isolated_u=30)
    assert g.u_ptr[-1] == 0
    p = dict(k=3, alpha=0.6, gamma=3, d=4, t_f=3, t_g=4, seed=1)
    labels, res, ref, sure = _end_to_end(g, p)
    assert np.array_equal(labels[sure], ref["labels"][sure])
    assert res.objective == pytest.approx(ref["objective"], rel=1e-5)


def test_single_node_end_to_end():
    # one U node and k = 1: every step runs on one row (a single tile with a 127-row ragged
    # tail, l = 1 in the randomized SVD), the label is 0 and Eq. 8 is 0
    g = synth.make_small(11, n_u=1, n_v=5, k=1, d_u=3)
    p = dict(k=1, alpha=0.6, gamma=3, d=3, t_f=3, t_g=4, seed=1)
    labels, res, ref, _ = _end_to_end(g, p)
    assert labels.tolist() == [0] and ref["labels"].tolist() == [0]
    assert res.objective == pytest.approx(ref["objective"], abs=1e-9)

def test_invalid_parameters_rejected():
    g = synth.make_small(10)
    h = abg.abg_create(g)
    for bad in [dict(k=0), dict(k=2 * g.d_u + 1), dict(k=2, alpha=1.0), dict(k=2, gamma=-1),
                dict(k=2, d=g.d_u + 1), dict(k=129, d=g.d_u)]:
        with pytest.raises(abg.AbgError) as e:
            abg.abg_cluster(h, abg.params(**bad))
        assert e.value.status == abg.ABG_EINVAL
    h.close()


def _csc(g):
    order = np.argsort(g.v_idx, kind="stable")
    v_ptr = np.zeros(g.n_v + 1, dtype=np.int64)
    np.cumsum(np.bincount(g.v_idx, minlength=g.n_v), out=v_ptr[1:])
    rows = np.repeat(np.arange(g.n_u, dtype=np.int32), np.diff(g.u_ptr))
    return v_ptr, rows[order].copy(), g.w[order].copy()


def test_invalid_edges_rejected_with_a_given_csc():
    # with the CSC given, the edge indices and weights of both orders are checked on the
    # device after the upload, before any kernel indexes with them; a good graph creates
    g = synth.make_small(11, n_u=500, n_v=700, k=3, d_u=4, deg=6)
    abg.abg_create(g, csc=_csc(g)).close()
    cases = []
    v_ptr, u_idx, w_t = _csc(g)
    bad = u_idx.copy(); bad[17] = g.n_u + 3
    cases.append(("CSC: index", g, (v_ptr, bad, w_t)))
    bad = w_t.copy(); bad[5] = -1.0
    cases.append(("CSC: weight", g, (v_ptr, u_idx, bad)))
    g2 = synth.make_small(11, n_u=500, n_v=700, k=3, d_u=4, deg=6)
    g2.v_idx = g2.v_idx.copy(); g2.v_idx[40] = -2
    cases.append(("CSR: index", g2, _csc(g)))
    g3 = synth.make_small(11, n_u=500, n_v=700, k=3, d_u=4, deg=6)
    g3.w = g3.w.copy(); g3.w[9] = float("nan")
    cases.append(("CSR: weight", g3, _csc(g)))
    for what, gg, csc in cases:
        with pytest.raises(abg.AbgError) as e:
            abg.abg_create(gg, csc=csc)
        assert e.value.status == abg.ABG_EINVAL, what
        assert what in str(e.value), (what, str(e.value))
    abg.abg_create(g, csc=_csc(g)).close()   # the device is fine afterwards


def _nan_padded(a: np.ndarray):
    """Device copy of `a` whose row padding (columns width..ld-1) holds NaN."""
    t = dev(a)
    if t.shape[1] > a.shape[1]:
        t[:, a.shape[1]:] = float("nan")
    return t


def test_row_padding_is_ignored_by_every_step():
    # widths that are not multiples of 4 leave padding columns in every row; whatever the
    # caller keeps there (here NaN) must not reach any result
    g = synth.make_small(21, n_u=300, n_v=400, k=3, d_u=6, deg=5)
    h = abg.abg_create(g)
    X = g.x_dense_f64()
    zh = empty(g.n_u, 6)
    abg.abg_propagate(h, _nan_padded(X), 6, 0.6, 4, zh)
    ref_z = tpo.normalize_rows(tpo.propagate(oracle_L(g), X.astype(np.float32).astype(np.float64),
                                             0.6, 4))
    got = host(zh, 6)
    assert np.all(np.isfinite(got)) and np.abs(got - ref_z).max() < 2e-5
    assert torch.all(zh[:, 6:] == 0)                       # padding written back as 0
    Zh = ref_z.astype(np.float32).astype(np.float64)
    R = empty(g.n_u, 12)
    abg.abg_random_features(_nan_padded(Zh), g.n_u, 6, 4, R)
    _, _, ref_r, _ = tpo.random_features(Zh, tpo.orthogonal_matrix(4, 6))
    assert np.abs(host(R, 12) - ref_r).max() <= 2e-4 * np.abs(ref_r).max()
    Rm = ref_r.astype(np.float32).astype(np.float64)[:, :11]     # width 11: one padding column
    phi, H = empty(g.n_u, 3), empty(11, 3)
    abg.abg_seed_factors(_nan_padded(Rm), g.n_u, 11, 3, phi, H, seed=2)
    assert torch.isfinite(phi[:, :3]).all() and torch.isfinite(H[:, :3]).all()
    P0, H0, _ = tpo.seed_factors(Rm, 3, 2)
    assert np.abs(host(phi, 3) - P0).max() <= 1e-3 * np.abs(P0).max()
    labels = torch.zeros(g.n_u, dtype=torch.int32, device=DEV)
    abg.abg_nci(_nan_padded(P0), g.n_u, 3, 5, labels)
    rl, _, rm, _ = tpo.nci(P0.astype(np.float32).astype(np.float64), 5)
    sure = rm > 1e-4
    assert np.array_equal(labels.cpu().numpy()[sure], rl[sure])
    obj = abg.abg_objective(_nan_padded(Rm), g.n_u, 11, labels, 3)
    ref_o = tpo.objective(Rm, labels.cpu().numpy(), 3)
    assert obj[0] == pytest.approx(ref_o[0], rel=1e-5)
    h.close()


@pytest.mark.parametrize("k", [1, 3, 17, 100])
@pytest.mark.parametrize("flags", [abg.ABG_NCI_PROCRUSTES, abg.ABG_NCI_EARLY_STOP,
                                   abg.ABG_NCI_PROCRUSTES | abg.ABG_NCI_EARLY_STOP])
def test_nci_variants(k, flags):
    # the Procrustes factor (T T^T = I enforced) and early stopping at the fixed point
    rng = np.random.default_rng(300 + k)
    n = 2999
    lab = rng.integers(0, k, n)
    Phi = np.abs(0.3 * rng.standard_normal((n, k)) / np.sqrt(n))
    Phi[np.arange(n), lab] += 1.0 / np.sqrt(n / k)
    if k > 3:
        Phi[:, 2] = 0.0                                  # a column nobody picks: empty cluster
    Phi = Phi.astype(np.float32).astype(np.float64)
    labels = torch.zeros(n, dtype=torch.int32, device=DEV)
    margin = torch.zeros(n, dtype=torch.float32, device=DEV)
    T = torch.zeros((k, k), dtype=torch.float64, device=DEV)
    _, passes = abg.abg_nci(dev(Phi), n, k, 20, labels, margin, T, nci_flags=flags,
                            with_passes=True)
    proc = bool(flags & abg.ABG_NCI_PROCRUSTES)
    early = bool(flags & abg.ABG_NCI_EARLY_STOP)
    rl, rT, rm, ch = tpo.nci(Phi, 20, procrustes=proc, early_stop=early)
    assert passes == len(ch)
    sure = rm > 1e-4
    assert np.array_equal(labels.cpu().numpy()[sure], rl[sure])
    assert np.abs(T.cpu().numpy() - rT).max() < 2e-5 * max(1.0, np.abs(rT).max())
    if proc:
        Tg = T.cpu().numpy()
        keep = np.abs(rT).sum(axis=0) > 1e-8        # columns of clusters that are not empty
        assert np.allclose((Tg.T @ Tg)[np.ix_(keep, keep)], np.eye(keep.sum()), atol=1e-4)


def test_solve_with_nci_variants(planted):
    g, p, ref = planted
    for proc, early in [(True, False), (False, True), (True, True)]:
        q = abg.params(k=p["k"], alpha=p["alpha"], gamma=p["gamma"], d=p["d"], t_f=p["t_f"],
                       t_g=p["t_g"], seed=p["seed"], procrustes=proc, early_stop=early)
        h = abg.abg_create(g)
        lab, res = abg.abg_cluster(h, q)
        h.close()
        r = tpo.tpo(g, procrustes=proc, early_stop=early, **p)
        sure = r["margin"] > 1e-4
        assert np.array_equal(lab[sure], r["labels"][sure])
        assert res.objective == pytest.approx(r["objective"], rel=1e-5)
        assert res.nci_passes == len(r["changes"])


@pytest.mark.parametrize("k", [1, 3, 17, 100, 128])
def test_procrustes_factor_newton_schulz_and_jacobi(k, monkeypatch):
    # the two ways to the Procrustes factor (Newton-Schulz on a thread-block cluster, Jacobi
    # SVD) against the oracle's SVD-based factor, with an empty cluster (a zero column of
    # Phi^T Y) for k > 3
    rng = np.random.default_rng(700 + k)
    n = 4001
    lab = rng.integers(0, k, n)
    Phi = np.abs(0.3 * rng.standard_normal((n, k)) / np.sqrt(n))
    Phi[np.arange(n), lab] += 1.0 / np.sqrt(n / k)
    if k > 3:
        Phi[:, 2] = 0.0
    Phi = Phi.astype(np.float32).astype(np.float64)
    rl, rT, rm, _ = tpo.nci(Phi, 12, procrustes=True)
    out = {}
    for mode in ("newton-schulz", "jacobi"):
        if mode == "jacobi":
            monkeypatch.setenv("ABG_POLAR", "jacobi")
        labels = torch.zeros(n, dtype=torch.int32, device=DEV)
        T = torch.zeros((k, k), dtype=torch.float64, device=DEV)
        abg.abg_nci(dev(Phi), n, k, 12, labels, None, T, nci_flags=abg.ABG_NCI_PROCRUSTES)
        out[mode] = (labels.cpu().numpy(), T.cpu().numpy())
    monkeypatch.delenv("ABG_POLAR", raising=False)
    sure = rm > 1e-4
    for mode, (lb, Tg) in out.items():
        assert np.array_equal(lb[sure], rl[sure]), mode
        assert np.abs(Tg - rT).max() < 2e-5 * max(1.0, np.abs(rT).max()), mode
        keep = np.abs(rT).sum(axis=0) > 1e-8
        assert np.allclose((Tg.T @ Tg)[np.ix_(keep, keep)], np.eye(keep.sum()), atol=1e-5), mode
        if k > 3:
            assert np.all(Tg[:, 2] == 0.0), mode     # the empty cluster's column stays zero


def test_procrustes_solve_same_alone_and_in_batch():
    # segments of different k in one batch: the Procrustes factor (either path) and hence the
    # labels of each graph are those of its solve alone
    graphs = [synth.make_small(900 + i, n_u=n, n_v=int(1.4 * n), k=kk, d_u=24, deg=6, signal=2.0)
              for i, (n, kk) in enumerate([(3000, 40), (1200, 7), (5000, 48), (800, 3)])]
    params = [abg.params(k=g.k, alpha=0.6, gamma=4, d=24, t_f=4, t_g=12, seed=40 + i,
                         procrustes=True) for i, g in enumerate(graphs)]
    batch = abg.abg_batch_create(graphs)
    labels, results = abg.abg_batch_cluster(batch, params)
    batch.close()
    row = 0
    for g, p, r in zip(graphs, params, results):
        h = abg.abg_create(g)
        lab1, r1 = abg.abg_cluster(h, p)
        h.close()
        assert np.array_equal(labels[row:row + g.n_u], lab1)
        assert r.objective == r1.objective
        row += g.n_u
