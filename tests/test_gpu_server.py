"""The continuous-batching request loop on the GPU: every served result equals the same request
solved alone (bitwise), requests of two attribute layouts mix in one stream, polls time out
while work is pending, and admission keeps the footprint within the budget."""
import threading
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402


def _requests():
    reqs = []
    for i in range(14):
        n_u = [80, 500, 2000, 9000, 150, 30000, 700][i % 7]
        kind = "csr_f32" if i % 2 else "dense_bf16"
        d_u = 40 if kind == "csr_f32" else 16
        g = synth.make_small(500 + i, n_u=n_u, n_v=int(1.5 * n_u), k=3 + i % 5, d_u=d_u, deg=6,
                             x_kind=kind, signal=3.0)
        d = 8 if kind == "csr_f32" else 16
        p = abg.params(k=3 + i % 5, alpha=0.6, gamma=4, d=d, t_f=4, t_g=8, seed=1000 + i)
        reqs.append((g, p))
    return reqs


def _alone(g, p):
    h = abg.abg_create(g)
    lab, res = abg.abg_cluster(h, p)
    h.close()
    return lab, res


def test_served_results_equal_alone():
    reqs = _requests()
    # a free worker waits up to 30 ms for compatible requests, so batches form however fast
    # the solves run
    sv = abg.Server(workers=3, max_batch_graphs=6, batch_window_us=30_000)
    rids = []
    for g, p in reqs:                 # arrivals spread over time so batches form as work runs
        rids.append(sv.submit(g, p))
        time.sleep(0.002)
    for (g, p), rid in zip(reqs, rids):
        st, lab, res = sv.poll(rid, 60_000_000)
        assert st == abg.ABG_OK, abg.lib().abg_last_error().decode()
        lab1, res1 = _alone(g, p)
        assert np.array_equal(lab, lab1)
        assert res.objective == res1.objective
    s = sv.stats()
    assert s["completed"] == len(reqs) and s["inflight_bytes"] == 0
    assert s["batches"] < len(reqs)   # requests were batched together
    sv.close()


def test_poll_timeout_and_pending():
    g = synth.make_config3(scale=0.05, k=10)    # a request that takes a while
    sv = abg.Server(workers=1)
    rid = sv.submit(g, abg.params(k=10, alpha=0.9, gamma=10, d=128))
    st, _, _ = sv.poll(rid, 0)
    assert st in (abg.ABG_PENDING, abg.ABG_OK)
    if st == abg.ABG_PENDING:
        st2, _, _ = sv.poll(rid, 1)               # 1 microsecond
        assert st2 in (abg.ABG_ETIMEDOUT, abg.ABG_OK)
        if st2 == abg.ABG_ETIMEDOUT:
            st3, lab, _ = sv.poll(rid, -1)
            assert st3 == abg.ABG_OK and lab.shape == (g.n_u,)
    sv.close()


def test_budget_serialises_requests():
    # a budget for about two requests: everything completes, the accounting returns to zero
    reqs = _requests()[:6]
    est = []
    for g, p in reqs:
        h = abg.abg_create(g)
        est.append(h.footprint() + abg.abg_solve_footprint(h, p))
        h.close()
    sv = abg.Server(workers=3, hbm_budget_bytes=2 * max(est) + (256 << 20), max_batch_graphs=1)
    rids = [sv.submit(g, p) for g, p in reqs]
    assert all(r > 0 for r in rids)
    for rid in rids:
        st, _, _ = sv.poll(rid, 60_000_000)
        assert st == abg.ABG_OK
    s = sv.stats()
    assert s["completed"] == 6 and s["inflight_bytes"] == 0 and s["max_batch"] == 1
    sv.close()


def test_concurrent_solves_of_different_widths():
    # host threads solving graphs whose block widths (and so the shared-memory sizes of the
    # one-CTA Cholesky / Jacobi kernels) differ, at the same time: every result equals the
    # same solve run alone
    cases = []
    for i, (d_u, d, k) in enumerate([(16, 16, 3), (40, 8, 5), (64, 64, 20), (24, 24, 40)]):
        g = synth.make_small(900 + i, n_u=1500, n_v=2000, k=k, d_u=d_u, deg=6,
                             x_kind="dense_bf16", signal=3.0)
        p = abg.params(k=k, alpha=0.6, gamma=3, d=d, t_f=3, t_g=5, seed=77 + i)
        cases.append((g, p))
    want = [_alone(g, p) for g, p in cases]
    handles = [abg.abg_create(g) for g, _ in cases]
    errors = []

    def run(i):
        try:
            for _ in range(6):
                lab, res = abg.abg_cluster(handles[i], cases[i][1])
                if not (np.array_equal(lab, want[i][0]) and res.objective == want[i][1].objective):
                    errors.append(f"case {i}: result differs from the solve run alone")
        except Exception as e:          # noqa: BLE001
            errors.append(f"case {i}: {e}")

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for h in handles:
        h.close()
    assert not errors, errors


def test_resident_graph_resolves():
    # re-solving a graph already on the device with other k / alpha / seed / NCI options: no
    # upload, several requests on one graph at once, each equal to the plain solve
    g = synth.make_small(80, n_u=5000, n_v=6000, k=6, d_u=16, deg=6, signal=3.0)
    h = abg.abg_create(g)
    ps = [abg.params(k=k, alpha=a, gamma=4, d=16, t_f=4, t_g=8, seed=s, procrustes=pr)
          for k, a, s, pr in [(3, 0.6, 0, False), (6, 0.5, 1, False), (6, 0.6, 2, True),
                              (4, 0.7, 3, False), (6, 0.6, 2, True)]]
    sv = abg.Server(workers=3)
    rids = [sv.submit_resident(h, p) for p in ps]
    g2 = synth.make_small(81, n_u=700, n_v=900, k=3, d_u=16, deg=5)   # an uploaded request too
    rid2 = sv.submit(g2, abg.params(k=3, alpha=0.6, gamma=4, d=16, t_f=4, t_g=8, seed=9))
    for p, rid in zip(ps, rids):
        st, lab, res = sv.poll(rid, 60_000_000)
        assert st == abg.ABG_OK, abg.lib().abg_last_error().decode()
        lab1, r1 = abg.abg_cluster(h, p)
        assert np.array_equal(lab, lab1) and res.objective == r1.objective
    st, lab2, _ = sv.poll(rid2, 60_000_000)
    assert st == abg.ABG_OK and lab2.shape == (g2.n_u,)
    s = sv.stats()
    assert s["completed"] == 6 and s["inflight_bytes"] == 0
    sv.close()
    tiny = abg.Server(workers=1, hbm_budget_bytes=1 << 20)
    assert tiny.submit_resident(h, ps[0]) < 0                  # footprint above the budget
    b = abg.abg_batch_create([g2, g2])
    with pytest.raises(abg.AbgError):
        tiny.submit_resident(b, ps[0])                          # a batch is not a resident graph
    b.close()
    tiny.close()
    h.close()


def test_served_mixed_precisions_equal_alone():
    # requests asking for the BF16 options are batched only with requests asking for the same
    # precision, and each result equals the request solved alone
    reqs = []
    for i in range(9):
        n_u = [300, 2500, 900][i % 3]
        g = synth.make_small(700 + i, n_u=n_u, n_v=int(1.5 * n_u), k=4, d_u=24, deg=6,
                             signal=3.0)
        p = abg.params(k=4, alpha=0.6, gamma=4, t_f=4, t_g=8, seed=2000 + i,
                       bf16_contract=i % 3 == 1, bf16_propagation=i % 3 == 2)
        reqs.append((g, p))
    sv = abg.Server(workers=2, max_batch_graphs=8)
    rids = [sv.submit(g, p) for g, p in reqs]
    for (g, p), rid in zip(reqs, rids):
        st, lab, res = sv.poll(rid, 60_000_000)
        assert st == abg.ABG_OK, abg.lib().abg_last_error().decode()
        lab1, res1 = _alone(g, p)
        assert np.array_equal(lab, lab1) and res.objective == res1.objective
    sv.close()


@pytest.mark.parametrize("kind,d_u,d", [("dense_bf16", 24, 24), ("csr_f32", 60, 10)])
def test_resident_resolves_reuse_the_propagation(kind, d_u, d):
    # Z_hat depends on alpha, gamma, d (and, with d < d_u, on the reduction's seed): a re-solve
    # with another k or NCI option takes it from the earlier solve and equals a cold solve
    g = synth.make_small(640, n_u=5000, n_v=7000, k=5, d_u=d_u, deg=6, x_kind=kind, signal=3.0)
    h = abg.abg_create(g)
    base = dict(alpha=0.6, gamma=5, d=d, t_f=4, t_g=10, seed=3)
    fp0 = h.footprint()
    lab1, r1 = abg.abg_cluster(h, abg.params(k=5, reuse_propagation=True, **base))
    assert r1.reused_propagation == 0 and h.footprint() > fp0     # computed, then kept
    cold1, c1 = abg.abg_cluster(h, abg.params(k=5, **base))
    assert np.array_equal(lab1, cold1) and r1.objective == c1.objective
    for k, proc in [(7, False), (4, True)]:
        p = abg.params(k=k, procrustes=proc, reuse_propagation=True, **base)
        lab, r = abg.abg_cluster(h, p)
        assert r.reused_propagation == 1 and r.ms_phase[1] < 0.05
        cold, c = abg.abg_cluster(h, abg.params(k=k, procrustes=proc, **base))
        assert c.reused_propagation == 0
        assert np.array_equal(lab, cold)
        assert r.objective == c.objective and r.trace_obj == c.trace_obj
    # another alpha (or, when reduced, another seed) does not match the kept Z_hat
    other = dict(base, alpha=0.5) if d == d_u else dict(base, seed=4)
    _, r = abg.abg_cluster(h, abg.params(k=5, reuse_propagation=True, **other))
    assert r.reused_propagation == 0
    # through the server: a resident re-solve reuses the Z_hat the last solve left
    sv = abg.Server(workers=2)
    p = abg.params(k=6, reuse_propagation=True, **other)
    rid = sv.submit_resident(h, p)
    st, lab, res = sv.poll(rid, 60_000_000)
    assert st == abg.ABG_OK and res.reused_propagation == 1
    assert sv.stats()["propagations_reused"] == 1
    cold, c = abg.abg_cluster(h, abg.params(k=6, **other))
    assert np.array_equal(lab, cold) and res.objective == c.objective
    sv.close()
    h.close()
