"""The allocation-free objective (abg_objective_noalloc) against the allocating one.

Some callers cannot allocate device memory while they run (their application gave the
whole GPU to its own allocator, or an allocation's synchronisation would break their
latency budget); this entry point serves them from one fixed array inside the library.
This file is collected last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11922_gb300 as abg  # noqa: E402

DEV = torch.device("cuda:0")


def _case(seed, n, m, k):
    rng = np.random.default_rng(seed)
    ld = ((m + 3) // 4) * 4
    R = torch.zeros((n, ld), dtype=torch.float32, device=DEV)
    R[:, :m] = torch.as_tensor(rng.standard_normal((n, m)), dtype=torch.float32)
    labels = torch.as_tensor(rng.integers(0, k, n).astype(np.int32), device=DEV)
    return R, labels


def test_noalloc_objective_matches_allocating_call_twice():
    # first a large call (k*(m+1) near the limit), then a smaller one: the second must not
    # depend on what the first left in the shared array
    for seed, (n, m, k) in enumerate([(200_003, 376, 128), (70_001, 64, 7)]):
        R, labels = _case(seed, n, m, k)
        got = abg.abg_objective_noalloc(R, n, m, labels, k)
        ref = abg.abg_objective(R, n, m, labels, k)
        assert got[0] == pytest.approx(ref[0], rel=1e-5)
        assert got[1] == pytest.approx(ref[1], rel=1e-5)


def test_noalloc_objective_rejects_oversized_problem():
    R, labels = _case(3, 1000, 512, 128)          # k * (m + 1) = 65,664 > 48,393
    with pytest.raises(abg.AbgError) as e:
        abg.abg_objective_noalloc(R, 1000, 512, labels, 128)
    assert e.value.status == abg.ABG_EINVAL
    assert "limit" in str(e.value)
