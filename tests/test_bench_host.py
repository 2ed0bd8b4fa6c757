"""Host-side pieces of bench.py that feed its JSON line: the NMI of the quality field (against
the oracle's metric module) and the algorithmic byte count behind the roofline."""
import os
import sys
from types import SimpleNamespace

import numpy as np

from oracle import metrics

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_nmi_matches_the_oracle_metric():
    rng = np.random.default_rng(0)
    for k1, k2 in [(3, 3), (5, 9), (20, 4)]:
        a = rng.integers(0, k1, 2000)
        b = np.where(rng.random(2000) < 0.7, a % k2, rng.integers(0, k2, 2000))
        assert abs(bench.nmi(a, b) - metrics.nmi(a, b)) < 1e-12
    assert bench.nmi(np.zeros(50, int), np.arange(50) % 3) == 0.0   # one cluster: no information


def test_propagation_bytes_formula():
    g = SimpleNamespace(nnz=1000, n_u=100, n_v=300)
    d, gamma = 16, 3
    per_spmm_index = 1000 * 8
    fp32 = 0.0
    for r in range(gamma):
        zin = 2 if r == 0 else 4
        fp32 += per_spmm_index + 1000 * d * zin + 300 * 12 + 300 * d * 4
        fp32 += per_spmm_index + 1000 * d * 4 + 100 * 12 + 100 * d * (2 + 4)
    assert bench.propagation_bytes(g, d, gamma) == fp32
    bf16 = bench.propagation_bytes(g, d, gamma, "bf16")
    # BF16 storage halves the gathered W / Z rows and their writes, except the final Z
    assert fp32 / 2 < bf16 < fp32


class _FakeEvent:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        _FakeCuda.clock += 10.0
        self.t = _FakeCuda.clock

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeCuda:
    clock = 0.0
    Event = _FakeEvent

    @staticmethod
    def synchronize():
        pass


class _FakeRes:
    def __init__(self, objective):
        self.objective = objective
        self.ms_phase = [0.0, 50.0, 8.0, 50.0, 36.0, 0.7]


class _FakeAbg:
    def params(self, **kw):
        return kw

    def abg_cluster(self, graph, p, labels, stream):
        # the BF16 options move one label and the objective a little
        labels[:] = np.arange(labels.size) % 4
        if p.get("bf16_contract"):
            labels[0] = 1
        return labels, _FakeRes(2.0 + (1e-6 if p.get("bf16_propagation") else 0.0))


def test_time_variants_reports_both_bf16_forms_and_restores_labels():
    g = SimpleNamespace(truth=np.arange(40) % 4)
    labels = np.arange(40) % 4
    before = labels.copy()
    args = SimpleNamespace(steps=5, nci="procrustes")
    out = bench.time_variants(_FakeAbg(), SimpleNamespace(cuda=_FakeCuda), None, g, labels,
                              [_FakeRes(2.0)], None, args)
    assert set(out) == {"bf16_contract_variant", "bf16_variant", "printed_t_variant"}
    for key, v in out.items():
        assert v["ms_per_step"] == 10.0 / 5 and v["value"] == 1e3 / 2.0
        if key != "printed_t_variant":
            assert v["labels_equal_to_fp32"] == 39 / 40
        assert v["quality"]["clusters_nonempty"] == 4
        assert v["phase_ms"]["propagation"] == 50.0
    assert out["bf16_contract_variant"]["objective_rel_diff_vs_fp32"] == 0.0
    assert abs(out["bf16_variant"]["objective_rel_diff_vs_fp32"] - 5e-7) < 1e-15
    assert out["printed_t_variant"]["labels_equal_to_fp32"] == 1.0
    assert np.array_equal(labels, before)       # the FP32 labels are back
    # with the printed T already timed, its variant is not repeated
    args = SimpleNamespace(steps=5, nci="printed")
    out = bench.time_variants(_FakeAbg(), SimpleNamespace(cuda=_FakeCuda), None, g, labels,
                              [_FakeRes(2.0)], None, args)
    assert set(out) == {"bf16_contract_variant", "bf16_variant"}
