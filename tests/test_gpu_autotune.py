"""The SpMM autotuner: on the first product of a shape it times the light-task variants (TMA
gather ring, register gathers, a lane group per row) and keeps the fastest. Every variant sums
each row's edges in edge order, so the propagation's output must be the same bits with the
autotuner on (tuning run and cached choice) and off (the fixed TMA-then-register order)."""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402

# large enough (>= 2^15 tasks + chunks on a side, ~4M edges) for the tuner to measure
GRAPHS = {
    "f32_d100": lambda: synth.make_small(10, n_u=500_000, n_v=600_000, k=4, d_u=100, deg=9,
                                         isolated_u=700, isolated_v=900),
    "bf16_d72": lambda: synth.make_small(11, n_u=500_000, n_v=700_000, k=4, d_u=72, deg=9,
                                         x_kind="dense_bf16", isolated_u=400),
    "hubs_d128": lambda: synth.make_config3(scale=0.15, k=10),
}


def _propagate(g, bf16=False):
    h = abg.abg_create(g)
    ld = ((g.d_u + 3) // 4) * 4
    out = []
    for _ in range(2):  # the first call tunes, the second uses the stored choice
        zh = torch.zeros((g.n_u, ld), dtype=torch.float32, device="cuda:0")
        abg.abg_propagate(h, None, g.d_u, 0.8, 5, zh, bf16_propagation=bf16)
        torch.cuda.synchronize()
        out.append(zh.cpu().numpy())
    h.close()
    return out


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("bf16", [False, True])
def test_autotuned_propagation_same_bits(name, bf16):
    g = GRAPHS[name]()
    n0 = abg.abg_spmm_tuned_shapes()
    tuned = _propagate(g, bf16)
    assert abg.abg_spmm_tuned_shapes() > n0  # the first call measured the variants
    os.environ["ABG_AUTOTUNE"] = "0"
    try:
        fixed = _propagate(g, bf16)
    finally:
        os.environ.pop("ABG_AUTOTUNE", None)
    assert np.array_equal(tuned[0], fixed[0])
    assert np.array_equal(tuned[1], fixed[0])
    assert np.array_equal(fixed[1], fixed[0])
