"""Clustering the V side (the method with the roles of U and V exchanged): a graph described
from the U side with side = ABG_SIDE_V and V attributes must give exactly what the explicitly
transposed graph gives from its own U side, and match the oracle on that transposed graph,
alone, in a batch and through the server."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import tpo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402


def _v_attributes(g, d, k, seed):
    rng = np.random.default_rng(seed)
    truth = rng.integers(0, k, g.n_v)
    mu = 3.0 * rng.standard_normal((k, d))
    return (mu[truth] + rng.standard_normal((g.n_v, d))).astype(np.float32)


def _transposed(g, xv):
    """The same edges seen from V (CSR rows = V nodes, stable by U index), attributes xv."""
    order = np.argsort(g.v_idx, kind="stable")
    v_ptr = np.zeros(g.n_v + 1, dtype=np.int64)
    np.cumsum(np.bincount(g.v_idx, minlength=g.n_v), out=v_ptr[1:])
    rows = np.repeat(np.arange(g.n_u, dtype=np.int32), np.diff(g.u_ptr))
    return synth.ABG("transposed", g.n_v, g.n_u, v_ptr, rows[order],
                     g.w[order] if g.w is not None else None, xv.shape[1], "dense_f32", xv)


def _solve(g, p, side=abg.ABG_SIDE_U):
    h = abg.abg_create(g, side=side)
    lab, res = abg.abg_cluster(h, p)
    h.close()
    return lab, res


@pytest.mark.parametrize("weighted", [True, False])
def test_v_side_equals_transposed_and_oracle(weighted):
    g = synth.make_small(51, n_u=1200, n_v=800, k=4, d_u=8, deg=6, weighted=weighted)
    xv = _v_attributes(g, 10, 3, seed=7)
    gv = dataclasses.replace(g, d_u=10, x=xv, x_kind="dense_f32")
    gt = _transposed(g, xv)
    p = abg.params(k=3, alpha=0.6, gamma=4, d=10, t_f=4, t_g=10, seed=2)
    lab_v, res_v = _solve(gv, p, abg.ABG_SIDE_V)
    lab_t, res_t = _solve(gt, p)
    assert lab_v.shape == (g.n_v,)
    assert np.array_equal(lab_v, lab_t) and res_v.objective == res_t.objective
    ref = tpo.tpo(gt, k=3, alpha=0.6, gamma=4, d=10, t_f=4, t_g=10, seed=2)
    sure = ref["margin"] > 1e-4
    assert np.array_equal(lab_v[sure], ref["labels"][sure])
    assert res_v.objective == pytest.approx(ref["objective"], rel=1e-5)


def test_v_side_batch_and_server():
    graphs, trans, params = [], [], []
    for i in range(4):
        g = synth.make_small(60 + i, n_u=300 + 200 * i, n_v=250 + 100 * i, k=3, d_u=8, deg=5)
        xv = _v_attributes(g, 6, 3, seed=20 + i)
        graphs.append(dataclasses.replace(g, d_u=6, x=xv, x_kind="dense_f32"))
        trans.append(_transposed(g, xv))
        params.append(abg.params(k=3, alpha=0.6, gamma=3, d=6, t_f=3, t_g=6, seed=i))
    b = abg.abg_batch_create(graphs, side=abg.ABG_SIDE_V)
    labels, results = abg.abg_batch_cluster(b, params)
    b.close()
    sv = abg.Server(workers=2, max_batch_graphs=4)
    rids = [sv.submit(g, p, side=abg.ABG_SIDE_V) for g, p in zip(graphs, params)]
    row = 0
    for g, gt, p, r, rid in zip(graphs, trans, params, results, rids):
        lab_t, res_t = _solve(gt, p)
        assert np.array_equal(labels[row:row + g.n_v], lab_t) and r.objective == res_t.objective
        st, lab_s, res_s = sv.poll(rid, 60_000_000)
        assert st == abg.ABG_OK and np.array_equal(lab_s, lab_t)
        assert res_s.objective == res_t.objective
        row += g.n_v
    sv.close()
