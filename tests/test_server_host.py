"""Host-side logic of the request loop, run without a GPU: admission by footprint, input
validation, unknown ids, and a request whose batch fails reporting that failure to its poll."""
import os

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def abg():
    from paper_2405_11922_gb300 import build as b
    b.build()
    import paper_2405_11922_gb300 as m
    return m


def test_admission_rejects_oversized_request(abg):
    sv = abg.Server(workers=1, hbm_budget_bytes=1 << 20)      # 1 MiB budget
    g = synth.make_small(0, n_u=5000, n_v=6000, d_u=64)
    rid = sv.submit(g, abg.params(k=3))
    assert rid < 0                                             # not admitted
    st, lab, res = sv.poll(rid, 0)
    assert st == abg.ABG_ENOTADMITTED and lab is None
    st, _, _ = sv.poll(rid, 0)
    assert st == abg.ABG_ENOTFOUND                             # the id was released
    assert sv.stats()["rejected"] == 1
    sv.close()


def test_invalid_request_and_unknown_id(abg):
    sv = abg.Server(workers=1)
    g = synth.make_small(1)
    g.v_idx = g.v_idx.copy()
    g.v_idx[0] = g.n_v + 5                                     # out of range
    with pytest.raises(abg.AbgError) as e:
        sv.submit(g, abg.params(k=2))
    assert e.value.status == abg.ABG_EINVAL
    st, _, _ = sv.poll(12345, 0)
    assert st == abg.ABG_ENOTFOUND
    sv.close()


def test_failed_batch_reports_to_its_requests(abg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("this test needs a machine without a GPU (the batch upload must fail)")
    sv = abg.Server(workers=2)
    rids = [sv.submit(synth.make_small(i), abg.params(k=2, seed=i)) for i in range(3)]
    for rid in rids:
        st, lab, _ = sv.poll(rid, 10_000_000)
        assert st == abg.ABG_EDEVICE and lab is None
    s = sv.stats()
    assert s["failed"] == 3 and s["completed"] == 0 and s["inflight_bytes"] == 0
    sv.close()
