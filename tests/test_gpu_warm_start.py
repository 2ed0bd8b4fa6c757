"""Resident re-solves that start Algorithm 2's ONMF steps from an earlier solve's final Phi and
H (ABG_WARM_START) instead of the randomized-SVD seeding of Eq. 18: the warm-started solve
against the oracle run the same way (its own first solve's Phi and H as the start of the
ONMF steps of the second, then Algorithm 3 and Eq. 8), and the cases that must stay cold."""
import numpy as np
import pytest

import synth
from oracle import tpo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402

MARGIN = 1e-3   # as the other end-to-end tests: labels must agree where the oracle is sure
OBJ_RTOL = 1e-5


@pytest.mark.parametrize("procrustes", [False, True])
def test_warm_start_against_oracle_chain(procrustes):
    g = synth.make_small(901, n_u=3000, n_v=4500, k=6, d_u=24, deg=6, signal=3.0)
    base = dict(k=6, gamma=4, d=24, t_f=4, t_g=10, seed=2, procrustes=procrustes)
    h = abg.abg_create(g)
    fp0 = h.footprint()
    lab_a, ra = abg.abg_cluster(h, abg.params(alpha=0.6, warm_start=True, **base))
    assert ra.warm_started == 0 and h.footprint() > fp0          # seeded, then kept
    lab_b, rb = abg.abg_cluster(h, abg.params(alpha=0.8, warm_start=True, **base))
    assert rb.warm_started == 1
    h.close()
    kw = dict(k=6, gamma=4, d=24, t_f=4, t_g=10, seed=2, procrustes=procrustes)
    ref_a = tpo.tpo(g, alpha=0.6, **kw)
    sure_a = ref_a["margin"] > MARGIN
    assert np.array_equal(lab_a[sure_a], ref_a["labels"][sure_a])
    assert ra.objective == pytest.approx(ref_a["objective"], rel=OBJ_RTOL)
    # the second solve in the oracle: R at alpha = 0.8, the ONMF steps from the first solve's
    # final factors, then Algorithm 3 and the objective
    ref_b = tpo.tpo(g, alpha=0.8, **kw)
    phi, _ = tpo.onmf(ref_b["R"], ref_a["Phi"], ref_a["H"], kw["t_f"])
    labels, _, margin, _ = tpo.nci(phi, kw["t_g"], procrustes)
    obj, _ = tpo.objective(ref_b["R"], labels, kw["k"])
    sure = margin > MARGIN
    assert sure.mean() > 0.8
    assert np.array_equal(lab_b[sure], labels[sure])
    assert rb.objective == pytest.approx(obj, rel=OBJ_RTOL)
    # and the start mattered: the cold solve at alpha = 0.8 is another run of the method
    assert not np.allclose(phi, ref_b["Phi"])


def test_warm_start_needs_same_k_and_the_option():
    g = synth.make_small(902, n_u=2500, n_v=3500, k=5, d_u=20, deg=6, signal=3.0)
    base = dict(gamma=4, d=20, t_f=4, t_g=8, seed=1)
    h = abg.abg_create(g)
    abg.abg_cluster(h, abg.params(k=5, alpha=0.6, warm_start=True, **base))
    # another k: nothing to start from, the solve seeds as usual (bitwise a cold solve)
    lab, r = abg.abg_cluster(h, abg.params(k=6, alpha=0.7, warm_start=True, **base))
    cold, c = abg.abg_cluster(h, abg.params(k=6, alpha=0.7, **base))
    assert r.warm_started == 0 and c.warm_started == 0
    assert np.array_equal(lab, cold) and r.objective == c.objective
    # without the option the kept factors are not used
    lab2, r2 = abg.abg_cluster(h, abg.params(k=6, alpha=0.5, **base))
    assert r2.warm_started == 0
    # the k = 6 factors kept just now start the next warm solve with k = 6, twice the same
    w1, s1 = abg.abg_cluster(h, abg.params(k=6, alpha=0.5, warm_start=True, **base))
    assert s1.warm_started == 1
    h.close()
    h2 = abg.abg_create(g)
    for k, a in [(5, 0.6), (6, 0.7)]:
        abg.abg_cluster(h2, abg.params(k=k, alpha=a, warm_start=True, **base))
    w2, s2 = abg.abg_cluster(h2, abg.params(k=6, alpha=0.5, warm_start=True, **base))
    assert s2.warm_started == 1
    assert np.array_equal(w1, w2) and s1.objective == s2.objective
    h2.close()


def test_warm_start_through_the_server():
    g = synth.make_small(903, n_u=2000, n_v=3000, k=4, d_u=16, deg=6, signal=3.0)
    base = dict(k=4, gamma=4, d=16, t_f=4, t_g=8, seed=5)
    h = abg.abg_create(g)
    abg.abg_cluster(h, abg.params(alpha=0.6, warm_start=True, **base))
    direct, rd = abg.abg_cluster(h, abg.params(alpha=0.7, warm_start=True, **base))
    h.close()
    h = abg.abg_create(g)
    abg.abg_cluster(h, abg.params(alpha=0.6, warm_start=True, **base))
    sv = abg.Server(workers=2)
    rid = sv.submit_resident(h, abg.params(alpha=0.7, warm_start=True, **base))
    st, lab, res = sv.poll(rid, 60_000_000)
    assert st == abg.ABG_OK and res.warm_started == 1
    assert np.array_equal(lab, direct) and res.objective == rd.objective
    sv.close()
    h.close()
