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


def test_noalloc_objective_takes_no_device_memory():
    # the first call on a device may reserve the fixed array (lazy module loading); every
    # later call must leave the device's free memory exactly where it was
    R, labels = _case(5, 100_003, 256, 100)
    ref = abg.abg_objective_noalloc(R, 100_003, 256, labels, 100)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        got = abg.abg_objective_noalloc(R, 100_003, 256, labels, 100)
        assert got == ref
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0


def test_noalloc_objective_from_two_threads_on_one_stream():
    # two host threads, one stream, alternating a wide call (k = 128) and a narrow one (k = 7):
    # the calls must neither undercut each other's shared-memory limit nor mix partial sums
    import threading
    cases = {128: _case(6, 150_001, 256, 128), 7: _case(7, 90_001, 40, 7)}
    dims = {128: (150_001, 256), 7: (90_001, 40)}
    refs = {k: abg.abg_objective(R, *dims[k], lab, k) for k, (R, lab) in cases.items()}
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()                # inputs written on the default stream are ready
    errors = []

    def worker(order):
        try:
            for k in order:
                R, lab = cases[k]
                got = abg.abg_objective_noalloc(R, *dims[k], lab, k, stream=stream)
                if got[0] != pytest.approx(refs[k][0], rel=1e-5) or \
                        got[1] != pytest.approx(refs[k][1], rel=1e-5):
                    errors.append((k, got, refs[k]))
        except Exception as e:              # noqa: BLE001 - reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=([128, 7, 128] * 4,)),
               threading.Thread(target=worker, args=([7, 128, 7] * 4,))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
