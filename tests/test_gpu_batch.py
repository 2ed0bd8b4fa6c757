"""Batched solves: many graphs stacked into one block-diagonal batch, each solved with its own
k and seed in the same kernel launches. A graph's result must be the same in a batch as alone
(fixed per-graph tiles and chunks, fixed reduction order), and must match the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import tpo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402


def _graphs(kind, n, d_u, seed0):
    out = []
    for i in range(n):
        n_u = [60, 300, 1200, 131, 4000][i % 5]
        out.append(synth.make_small(seed0 + i, n_u=n_u, n_v=int(n_u * 1.3), k=2 + i % 4,
                                    d_u=d_u, deg=5, x_kind=kind, signal=3.0))
    return out


def _alone(g, p):
    h = abg.abg_create(g)
    lab, res = abg.abg_cluster(h, p)
    h.close()
    return lab, res


@pytest.mark.parametrize("kind,d_u,d", [("dense_f32", 12, 12), ("dense_bf16", 16, 16),
                                        ("csr_f32", 40, 40), ("csr_f32", 40, 6)])
def test_batch_equals_alone_and_oracle(kind, d_u, d):
    graphs = _graphs(kind, 5, d_u, 100 + d)
    params = [abg.params(k=g.k, alpha=0.6, gamma=4, d=d, t_f=4, t_g=8, seed=17 + i)
              for i, g in enumerate(graphs)]
    batch = abg.abg_batch_create(graphs)
    assert abg.lib().abg_graph_segments(batch.handle) == len(graphs)
    labels, results = abg.abg_batch_cluster(batch, params)
    batch.close()
    row = 0
    for g, p, r in zip(graphs, params, results):
        seg = labels[row:row + g.n_u]
        row += g.n_u
        lab1, r1 = _alone(g, p)
        assert np.array_equal(seg, lab1)                          # same alone and in the mix
        assert r.objective == r1.objective and r.trace_obj == r1.trace_obj
        ref = tpo.tpo(g, k=p.k, alpha=p.alpha, gamma=p.gamma, d=p.d, t_f=p.t_f, t_g=p.t_g,
                      seed=p.seed)
        sure = ref["margin"] > 1e-4
        assert np.array_equal(seg[sure], ref["labels"][sure])
        assert r.objective == pytest.approx(ref["objective"], rel=1e-5)


def test_batch_rejects_mixed_parameters():
    graphs = _graphs("dense_f32", 2, 8, 300)
    batch = abg.abg_batch_create(graphs)
    ps = [abg.params(k=2, gamma=3), abg.params(k=2, gamma=4)]
    with pytest.raises(abg.AbgError) as e:
        abg.abg_batch_cluster(batch, ps)
    assert e.value.status == abg.ABG_EINVAL
    with pytest.raises(abg.AbgError):
        abg.abg_cluster(batch, abg.params(k=2))          # a batch needs per-graph parameters
    batch.close()


def test_batch_rejects_mixed_attribute_kinds():
    g1 = synth.make_small(1, x_kind="dense_f32", d_u=8)
    g2 = synth.make_small(2, x_kind="csr_f32", d_u=8)
    with pytest.raises(abg.AbgError) as e:
        abg.abg_batch_create([g1, g2])
    assert e.value.status == abg.ABG_EINVAL


def test_many_segments_repeatable():
    # hundreds of segments keep hundreds of one-CTA-per-segment kernels in flight at once:
    # the batch must give the same bits twice, and the same bits as solving alone
    rng = np.random.default_rng(7)
    graphs, params = [], []
    for i in range(300):
        n_u = int(rng.integers(40, 400))
        k = int(rng.integers(2, 12))
        graphs.append(synth.make_small(2000 + i, n_u=n_u, n_v=int(1.4 * n_u), k=k, d_u=24,
                                       deg=5, x_kind="csr_f32" if i % 2 else "dense_f32",
                                       signal=3.0))
        params.append(abg.params(k=k, alpha=0.6, gamma=4, d=10, t_f=4, t_g=8, seed=i))
    for kind in ("dense_f32", "csr_f32"):
        idx = [i for i, g in enumerate(graphs) if g.x_kind == kind]
        gs, ps = [graphs[i] for i in idx], [params[i] for i in idx]
        runs = []
        for _ in range(2):
            b = abg.abg_batch_create(gs)
            lab, res = abg.abg_batch_cluster(b, ps)
            b.close()
            runs.append((lab, [r.objective for r in res]))
        assert np.array_equal(runs[0][0], runs[1][0])
        assert runs[0][1] == runs[1][1]
        row = 0
        for j, (g, p) in enumerate(zip(gs, ps)):
            if j % 15 == 0:
                lab1, r1 = _alone(g, p)
                assert np.array_equal(runs[0][0][row:row + g.n_u], lab1)
                assert runs[0][1][j] == r1.objective
            row += g.n_u


def test_batch_with_nci_flags_equals_alone():
    # early stopping is decided per segment; a segment that has converged repeats the same pass
    # while the others continue, so its result and its reported passes equal the solve alone
    graphs = _graphs("dense_f32", 6, 16, 700)
    params = [abg.params(k=g.k, alpha=0.6, gamma=4, d=16, t_f=4, t_g=15, seed=3 + i,
                         procrustes=True, early_stop=True) for i, g in enumerate(graphs)]
    b = abg.abg_batch_create(graphs)
    labels, results = abg.abg_batch_cluster(b, params)
    b.close()
    row = 0
    for g, p, r in zip(graphs, params, results):
        lab1, r1 = _alone(g, p)
        assert np.array_equal(labels[row:row + g.n_u], lab1)
        assert r.objective == r1.objective and r.nci_passes == r1.nci_passes
        row += g.n_u
    mixed = [abg.params(k=2), abg.params(k=2, procrustes=True)]
    b = abg.abg_batch_create(graphs[:2])
    with pytest.raises(abg.AbgError):
        abg.abg_batch_cluster(b, mixed)
    b.close()
