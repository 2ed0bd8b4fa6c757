"""The tensor-core (tcgen05, three-term tf32 split) products against the FP32 SIMT kernels and
the FP64 oracle: randomized-SVD seeding, ONMF and NCI steps with the tensor-core path on and
off (ABG_TENSOR_CORES=0), on tall inputs with ragged last tiles, several widths and batches."""
import os

import numpy as np
import pytest

import synth
from oracle import tpo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402

DEV = "cuda:0"


def dev(a):
    a = np.asarray(a, dtype=np.float32)
    ld = ((a.shape[1] + 3) // 4) * 4
    t = torch.zeros((a.shape[0], ld), dtype=torch.float32, device=DEV)
    t[:, :a.shape[1]] = torch.from_numpy(a)
    return t


def empty(rows, cols):
    return torch.zeros((rows, ((cols + 3) // 4) * 4), dtype=torch.float32, device=DEV)


def host(t, cols):
    torch.cuda.synchronize()
    return t[:, :cols].double().cpu().numpy()


class simt:
    """Run the enclosed steps on the SIMT kernels."""

    def __enter__(self):
        os.environ["ABG_TENSOR_CORES"] = "0"

    def __exit__(self, *exc):
        os.environ.pop("ABG_TENSOR_CORES", None)


@pytest.mark.parametrize("n,m,k", [(3001, 40, 6), (1000, 256, 100), (257, 130, 20)])
def test_seed_factors_tc_vs_simt_vs_oracle(n, m, k):
    rng = np.random.default_rng(n + m)
    U = np.linalg.qr(rng.standard_normal((n, m)))[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    s = 0.97 ** np.arange(m) * 10   # sigma_k / sigma_1 stays well above the FP32 floor
    A = ((U * s) @ V.T).astype(np.float32).astype(np.float64)
    out = {}
    for mode in ("tc", "simt"):
        phi, H = empty(n, k), empty(m, k)
        sig = torch.zeros(k, dtype=torch.float64, device=DEV)
        c0 = abg.abg_tensor_core_launches()
        if mode == "simt":
            with simt():
                abg.abg_seed_factors(dev(A), n, m, k, phi, H, sig, seed=4)
            assert abg.abg_tensor_core_launches() == c0
        else:
            abg.abg_seed_factors(dev(A), n, m, k, phi, H, sig, seed=4)
            assert abg.abg_tensor_core_launches() > c0      # the tensor cores did the products
        out[mode] = (host(phi, k), host(H, k), sig.cpu().numpy())
    _, _, S0 = tpo.seed_factors(A, k, 4)
    for mode in ("tc", "simt"):   # eigenvalues of B B^T: error ~ eps * sigma_1 in sigma
        assert np.abs(out[mode][2] - S0).max() <= 2e-5 * S0[0]
    P_t, H_t, _ = out["tc"]
    P_s, H_s, _ = out["simt"]
    assert np.abs(P_t - P_s).max() <= 2e-4 * np.abs(P_s).max()
    assert np.abs(H_t - H_s).max() <= 2e-4 * np.abs(H_s).max()


def test_onmf_tc_vs_simt_vs_oracle():
    g = synth.make_small(31, n_u=2500, n_v=3000, k=7, d_u=24, deg=6, signal=3.0)
    p = dict(k=7, alpha=0.6, gamma=4, d=24, t_f=5, t_g=10, seed=3)
    ref = tpo.tpo(g, **p)
    R = ref["R"].astype(np.float32).astype(np.float64)
    P0 = ref["Phi0"].astype(np.float32).astype(np.float64)
    H0 = ref["H0"].astype(np.float32).astype(np.float64)
    n, m, k = R.shape[0], R.shape[1], p["k"]
    res = {}
    for mode in ("tc", "simt"):
        phi, H = dev(P0), dev(H0)
        if mode == "simt":
            with simt():
                abg.abg_onmf(dev(R), n, m, k, p["t_f"], phi, H)
        else:
            abg.abg_onmf(dev(R), n, m, k, p["t_f"], phi, H)
        res[mode] = (host(phi, k), host(H, k))
    Pr, Hr = tpo.onmf(R, P0, H0, p["t_f"])
    for mode in ("tc", "simt"):
        assert np.abs(res[mode][0] - Pr).max() <= 1e-4 * np.abs(Pr).max()
        assert np.abs(res[mode][1] - Hr).max() <= 1e-4 * np.abs(Hr).max()


@pytest.mark.parametrize("k", [1, 3, 16, 50, 100, 128])
def test_nci_tc_vs_oracle(k):
    rng = np.random.default_rng(100 + k)
    n = 4099
    lab = rng.integers(0, k, n)
    Phi = np.abs(0.3 * rng.standard_normal((n, k)) / np.sqrt(n))
    Phi[np.arange(n), lab] += 1.0 / np.sqrt(n / k)
    Phi[9] = 0.0                                      # all scores tie -> cluster 0
    Phi = Phi.astype(np.float32).astype(np.float64)
    labels = torch.zeros(n, dtype=torch.int32, device=DEV)
    margin = torch.zeros(n, dtype=torch.float32, device=DEV)
    T = torch.zeros((k, k), dtype=torch.float64, device=DEV)
    c0 = abg.abg_tensor_core_launches()
    abg.abg_nci(dev(Phi), n, k, 20, labels, margin, T)
    assert abg.abg_tensor_core_launches() > c0
    rl, rT, rm, _ = tpo.nci(Phi, 20)
    got = labels.cpu().numpy()
    sure = rm > 1e-4
    assert np.array_equal(got[sure], rl[sure])
    assert got[9] == 0
    if k > 1:
        assert np.abs(margin.cpu().numpy()[sure] - rm[sure]).max() < 1e-5
    assert np.abs(T.cpu().numpy() - rT).max() < 1e-5 * max(1.0, np.abs(rT).max())


def test_batched_solve_tc_vs_simt():
    graphs = [synth.make_small(40 + i, n_u=[300, 1500, 77][i], n_v=[400, 2000, 120][i],
                               k=[3, 9, 2][i], d_u=20, deg=6, signal=3.0) for i in range(3)]
    params = [abg.params(k=g.k, alpha=0.6, gamma=4, d=20, t_f=4, t_g=8, seed=5 + i)
              for i, g in enumerate(graphs)]
    out = {}
    for mode in ("tc", "simt"):
        b = abg.abg_batch_create(graphs)
        if mode == "simt":
            with simt():
                out[mode] = abg.abg_batch_cluster(b, params)
        else:
            out[mode] = abg.abg_batch_cluster(b, params)
        b.close()
    row = 0
    for g, p, rt, rs_ in zip(graphs, params, out["tc"][1], out["simt"][1]):
        ref = tpo.tpo(g, k=p.k, alpha=p.alpha, gamma=p.gamma, d=p.d, t_f=p.t_f, t_g=p.t_g,
                      seed=p.seed)
        sure = ref["margin"] > 1e-3
        assert np.array_equal(out["tc"][0][row:row + g.n_u][sure], ref["labels"][sure])
        assert rt.objective == pytest.approx(ref["objective"], rel=1e-5)
        assert rt.objective == pytest.approx(rs_.objective, rel=1e-5)
        row += g.n_u


@pytest.mark.parametrize("n,d", [(5003, 128), (777, 16), (4099, 48), (300, 256), (2000, 12), (1500, 6), (999, 3)])
def test_random_features_tc_vs_simt_vs_oracle(n, d):
    # Z_hat Q^T with the sin/cos and column-sum epilogue on the tensor cores (3xTF32) against
    # the SIMT kernel and the FP64 oracle; ragged last tiles, one zero row (reading R3)
    rng = np.random.default_rng(40 + d)
    Zh = tpo.normalize_rows(rng.standard_normal((n, d))).astype(np.float32).astype(np.float64)
    Zh[3] = 0.0
    _, _, ref, cl_ref = tpo.random_features(Zh, tpo.orthogonal_matrix(9, d))
    out = {}
    for mode in ("tc", "simt"):
        R = empty(n, 2 * d)
        t0 = abg.abg_tensor_core_launches()
        if mode == "simt":
            with simt():
                cl = abg.abg_random_features(dev(Zh), n, d, 9, R)
        else:
            cl = abg.abg_random_features(dev(Zh), n, d, 9, R)
        ran_tc = abg.abg_tensor_core_launches() > t0
        assert ran_tc == (mode == "tc")
        assert cl == cl_ref
        out[mode] = host(R, 2 * d)
    for mode, got in out.items():
        assert np.abs(got - ref).max() <= 2e-4 * np.abs(ref).max(), mode
    # the two kernels differ only by the tf32 operand split and the summation order
    assert np.abs(out["tc"] - out["simt"]).max() <= 5e-5 * np.abs(ref).max()
