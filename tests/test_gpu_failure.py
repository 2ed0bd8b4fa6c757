"""Failure detection on the GPU without a fault: every wait inside a kernel is bounded, and a
wait that runs out makes the solve return ABG_EDEVICE with a message while the context stays
usable. The test hook ABG_TEST_WAIT_EXPIRY=spmm (read at the start of each solve) gives the
first wait of every warp of the TMA-gather SpMM no time at all, so it runs out on a copy that
is still in flight; the warp then drains its own copies under the normal limit and stops."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402


def test_wait_expiry_is_reported_and_the_next_solve_is_clean(monkeypatch):
    # rows of 100 floats (25 float4 chunks) take the TMA-gather kernel
    g = synth.make_small(10, n_u=3000, n_v=4100, k=4, d_u=100, deg=9)
    h = abg.abg_create(g)
    p = abg.params(k=4, alpha=0.6, gamma=3, d=100, t_f=3, t_g=5, seed=1)
    lab0, r0 = abg.abg_cluster(h, p)
    l0 = abg.abg_launch_count()
    monkeypatch.setenv("ABG_TEST_WAIT_EXPIRY", "spmm")
    with pytest.raises(abg.AbgError) as e:
        abg.abg_cluster(h, p)
    assert e.value.status == abg.ABG_EDEVICE
    assert "bounded wait" in str(e.value) and "SpMM" in str(e.value)
    assert abg.abg_launch_count() > l0              # the kernels did launch and return
    monkeypatch.delenv("ABG_TEST_WAIT_EXPIRY")
    lab1, r1 = abg.abg_cluster(h, p)                # same process, same context: clean again
    assert np.array_equal(lab0, lab1)
    assert r1.objective == r0.objective and r1.trace_obj == r0.trace_obj
    h.close()
