#!/usr/bin/env python
"""Benchmark of the TPO hot path on one GB300 (and N independent replicas under torchrun).

A step is one full solve (Algorithms 1-3, T of Algorithm 3 as the Procrustes factor of Phi^T Y,
and the objective) of the large planted-partition
workload: |U| = 2,000,000, |V| = 5,000,000, 50M edge draws (Chung-Lu exponent 2.2 on both
sides, 60/40 mixing), dense Gaussian-mixture attributes d = 128 stored as BF16, k = 100,
alpha = 0.9, gamma = 10, T_f = 5, T_g = 20. Inputs are synthetic (seeded generator) and far
larger than L2 (the graph alone is ~1.3 GB, a solve touches ~60 GB).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0. `value` = solves/s of the whole job with the graph resident in
HBM; `e2e` = the same through the C ABI from pinned host buffers (graph upload, solve, labels
back, graph freed, every step). `roofline` covers the propagation SpMMs (the dominant kernels),
timed by CUDA events inside the library on the launch stream. The reference arm times the FP64
CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("TPO iterations/s and SpMM HBM GB/s at |U|=2M; solves/s + p99 latency "
          "(served vs plain)")
WORKLOAD = dict(workload="planted ABG |U|=2M |V|=5M 50M edge draws, Chung-Lu 2.2, 60/40 mixing, "
                         "dense BF16 attributes d=128, k=100, alpha=0.9, gamma=10, T_f=5, T_g=20",
                n_u=2_000_000, n_v=5_000_000, d=128, k=100)
def workload_of(g, scale: float) -> dict:
    """The config label; a scaled-down run names its own sizes."""
    if scale == 1.0:
        return dict(WORKLOAD)
    return dict(workload=f"planted ABG |U|={g.n_u} |V|={g.n_v} (config scaled by {scale}), "
                         "Chung-Lu 2.2, 60/40 mixing, dense BF16 attributes d=128, k=100, "
                         "alpha=0.9, gamma=10, T_f=5, T_g=20",
                n_u=int(g.n_u), n_v=int(g.n_v), d=128, k=100, scale=scale)


PARAMS = dict(k=100, alpha=0.9, gamma=10, d=128, t_f=5, t_g=20, seed=0)
L2_NOTE = "inputs larger than L2 (graph 1.3 GB, solve working set ~11 GB)"


def config_of(nci: str, precision: str, parallelism: str, g=None, scale: float = 1.0) -> dict:
    """The line's config: the workload (named by its sizes), the T update of Algorithm 3, the
    arithmetic and where it runs."""
    return dict(workload_of(g, scale), nci=NCI_NAMES[nci], precision=precision,
                parallelism=parallelism, l2=L2_NOTE)
NCI_NAMES = {"procrustes": "Algorithm 3 with T = orthogonal Procrustes factor of Phi^T Y "
                           "(T T^T = I of Eq. 20)",
             "printed": "Algorithm 3 with T = Phi^T Y"}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms during a timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join("/tmp", f"abg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for nm, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def gpu_id_for_smi(local_rank: int) -> str:
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        return ids[local_rank] if local_rank < len(ids) else str(local_rank)


def propagation_bytes(g, d: int, gamma: int, precision: str = "fp32") -> float:
    """Algorithmic bytes of gamma propagation rounds (both SpMMs): per round, each SpMM reads
    nnz (index + value) and one gathered d-wide row per edge, plus its row pointers and row
    list; the first product gathers BF16 X rows, the rest Z rows; the second product also
    reads the X restart rows (BF16) and writes Z; the first writes W. W and Z are 4-byte FP32
    elements, or 2-byte BF16 ones (all but the final Z) with precision "bf16"."""
    nnz, n_u, n_v = g.nnz, g.n_u, g.n_v
    e = 2 if precision == "bf16" else 4
    per_spmm_index = nnz * 8
    total = 0.0
    for r in range(gamma):
        zin = 2 if r == 0 else e
        zout = 4 if r == gamma - 1 else e
        total += per_spmm_index + nnz * d * zin + n_v * (8 + 4) + n_v * d * e       # W = L^T Z
        total += per_spmm_index + nnz * d * e + n_u * (8 + 4) + n_u * d * (2 + zout)  # Z = ...
    return total


# DRAM bytes of one propagation round (L^T Z then L W, all SpMM launches) of the full-size
# workload, from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum (1-pass
# metrics) of the current SpMM kernels. Only meaningful for the full-size workload.
ROUND_DRAM_BYTES_FULL = 29.84e9


def roofline_of(pbytes: float, prop_ms: float, peak: float, peak_kind: str, scale: float,
                precision: str = "fp32") -> dict:
    """Roofline of the propagation SpMMs, per round: achieved = algorithmic bytes (gathered
    rows counted once per edge) / round time; traffic = measured DRAM bytes of a round (full
    size only); traffic_gbs = the bandwidth the DRAM actually delivered."""
    gamma = PARAMS["gamma"]
    round_s = prop_ms / 1e3 / gamma
    achieved = pbytes / gamma / round_s / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": None,
           "kernel": "propagation SpMMs per round (k_spmm_tma light tasks + heavy-row chunks, "
                     "k_spmm_reduce)",
           "per": "propagation round", "algorithmic_bytes": pbytes / gamma, "peak_kind": peak_kind,
           "note": "frac counts every gathered row once per edge, so L2 hits on hub rows can take "
                   "it above 1; traffic_frac (measured DRAM bytes of a round over the same time) "
                   "is the share of HBM bandwidth the round uses"}
    if scale == 1.0 and precision == "fp32":
        out["traffic"] = ROUND_DRAM_BYTES_FULL
        out["traffic_gbs"] = ROUND_DRAM_BYTES_FULL / round_s / 1e9
        out["traffic_frac"] = out["traffic_gbs"] / peak
    return out


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's); x itself when not
    distributed. device: where the collective's tensor lives ("cuda" for NCCL, "cpu" for gloo)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, elapsed_max_s: float) -> float:
    """Whole-job solves/s: every rank solves `steps` graphs; the job takes the slowest rank's
    time."""
    return world * steps / elapsed_max_s


VARIANTS = (("bf16_contract_variant", "bf16-contract (SpMM FP32, products with R in BF16)",
             dict(bf16_contract=True)),
            ("bf16_variant", "bf16 (bf16-contract + bf16-propagation)",
             dict(bf16_contract=True, bf16_propagation=True)),
            ("printed_t_variant", "fp32, Algorithm 3 as printed (T = Phi^T Y)",
             dict(procrustes=False)))


def time_variants(abg, torch, graph, g, labels, results, stream, args) -> dict:
    """Time the variants of the FP32 solve on its resident graph (the two BF16 options, and
    Algorithm 3 with the printed T when the steps use the Procrustes T): one untimed solve, then
    args.steps timed with CUDA events, each compared with the FP32 result held in `labels` /
    `results`; `labels` holds the FP32 labels again on return."""
    ref_labels = labels.copy()
    out = {}
    for key, desc, flags in VARIANTS:
        flags = dict(dict(procrustes=args.nci == "procrustes"), **flags)
        if key == "printed_t_variant" and not flags["procrustes"] and args.nci == "printed":
            continue                      # the timed steps already are this variant
        pv = abg.params(**PARAMS, **flags)
        abg.abg_cluster(graph, pv, labels, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vres = [abg.abg_cluster(graph, pv, labels, stream)[1] for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        vms = e0.elapsed_time(e1) / args.steps
        out[key] = {"precision": desc, "value": 1e3 / vms, "unit": "solves/s",
                    "ms_per_step": vms,
                    "phase_ms": dict(zip(["attributes", "propagation", "features", "svd_nmf",
                                          "nci", "objective"],
                                         [statistics.median(r.ms_phase[i] for r in vres)
                                          for i in range(6)])),
                    "quality": quality_of(g, labels, vres[-1]),
                    "labels_equal_to_fp32": float(np.mean(labels == ref_labels)),
                    "objective_rel_diff_vs_fp32":
                        vres[-1].objective / results[-1].objective - 1.0}
    labels[:] = ref_labels
    return out


def csc_of(g):
    order = np.argsort(g.v_idx, kind="stable")
    v_ptr = np.zeros(g.n_v + 1, dtype=np.int64)
    np.cumsum(np.bincount(g.v_idx, minlength=g.n_v), out=v_ptr[1:])
    rows = np.repeat(np.arange(g.n_u, dtype=np.int32), np.diff(g.u_ptr))
    return v_ptr, rows[order], (g.w[order] if g.w is not None else None)


class PinnedGraph:
    """The generator's arrays copied into page-locked host memory (for the e2e arm)."""

    def __init__(self, g, csc):
        import torch

        def pin(a):
            return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

        self._keep = [pin(a) for a in (g.u_ptr, g.v_idx, g.w, g.x, csc[0], csc[1], csc[2])]
        arr = [None if t is None else t.numpy() for t in self._keep]
        self.n_u, self.n_v, self.d_u, self.x_kind = g.n_u, g.n_v, g.d_u, g.x_kind
        self.u_ptr, self.v_idx, self.w, self.x = arr[0], arr[1], arr[2], arr[3]
        self.x_ptr = self.x_idx = self.x_val = None
        self.csc = (arr[4], arr[5], arr[6])
        self.h2d_bytes = sum(int(a.nbytes) for a in arr if a is not None)


def nmi(a, b) -> float:
    """Normalised mutual information (geometric mean normalisation) of two labelings."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    ka, kb = int(a.max()) + 1, int(b.max()) + 1
    p = np.bincount(a * kb + b, minlength=ka * kb).reshape(ka, kb) / a.size
    pa, pb = p.sum(1), p.sum(0)
    nz = p > 0
    mi = float((p[nz] * np.log(p[nz] / np.outer(pa, pb)[nz])).sum())
    ha = -float((pa[pa > 0] * np.log(pa[pa > 0])).sum())
    hb = -float((pb[pb > 0] * np.log(pb[pb > 0])).sum())
    return mi / np.sqrt(ha * hb) if ha > 0 and hb > 0 else 0.0


def quality_of(g, labels, res) -> dict:
    return {"clusters_nonempty": int(np.unique(labels).size),
            "nmi_vs_planted": round(nmi(g.truth, labels), 4) if g.truth is not None else None,
            "objective_eq8": res.objective}


ORACLE_SCALE = 0.01   # the oracle's sample: the same generator at 1% of the workload


def oracle_graph(seed: int = 0, scale: float = ORACLE_SCALE):
    import synth
    return synth.make_config3(seed=seed, scale=scale)


def oracle_solve_seconds(g, procrustes: bool = True) -> float:
    """Wall time of one FP64 oracle solve of ``g`` with the workload's parameters."""
    from oracle import tpo
    t0 = time.perf_counter()
    tpo.tpo(g, **PARAMS, procrustes=procrustes)
    return time.perf_counter() - t0


def oracle_threads() -> int:
    """Threads the oracle's BLAS may use: the thread variables when set, else every core."""
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count() or 1


def oracle_single_thread_seconds(procrustes: bool = True, scale: float = ORACLE_SCALE) -> float:
    """One oracle solve of the sample in a child process limited to one thread (BLAS thread
    counts are fixed when numpy loads, so a fresh interpreter is needed)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "g = bench.oracle_graph(scale=%r); print(bench.oracle_solve_seconds(g, %r))"
            % (ROOT, scale, procrustes))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True)
    return float(out.stdout.strip().splitlines()[-1])


def sample_note(g, scale: float, what: str) -> str:
    return (f"{what}: full FP64 oracle solves of the same generator at {scale:g} of the workload "
            f"(|U|={g.n_u}, |V|={g.n_v}, {g.nnz} edges, k=100, d=128), each timed on the host "
            f"cores; value = {scale:g} / seconds per sample solve, i.e. the full workload's "
            "solves/s if the oracle's time grows linearly in |U| and |E| (every step is linear "
            "in both at fixed d and k)")


def cpu_baseline(procrustes: bool) -> dict:
    """The oracle as it stands on the host cores: one solve of the 1% sample on every thread
    (after one untimed solve), and one in a single-threaded child process."""
    g = oracle_graph()
    oracle_solve_seconds(g, procrustes)
    t_all = oracle_solve_seconds(g, procrustes)
    t_one = oracle_single_thread_seconds(procrustes)
    return {"value": ORACLE_SCALE / t_all, "unit": "solves/s", "cores": oracle_threads(),
            "kind": "oracle", "sample": sample_note(g, ORACLE_SCALE, "measured"),
            "measured_sample_s": t_all,
            "single_thread": {"value": ORACLE_SCALE / t_one, "cores": 1,
                              "measured_sample_s": t_one}}


def run_reference(args, rank: int):
    if rank != 0:
        return
    g = oracle_graph()
    proc = args.nci == "procrustes"
    secs = []
    t_start = time.perf_counter()
    for i in range(args.warmup + args.steps):
        t = oracle_solve_seconds(g, proc)
        if i >= args.warmup:
            secs.append(t)
    timed_s = sum(secs)
    step_s = statistics.median(secs)
    v = ORACLE_SCALE / step_s
    cores = oracle_threads()
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * timed_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.nci, "fp64 (oracle)",
                                f"CPU oracle on {cores} host threads"),
            "step": f"one oracle solve of the workload's generator at {ORACLE_SCALE:g} of its "
                    f"size (|U|={g.n_u}); ms_per_step is that solve's measured time",
            "sample_scale": ORACLE_SCALE,
            "extrapolated_full_s": step_s / ORACLE_SCALE,
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample_note(g, ORACLE_SCALE, "measured"),
                             "measured_sample_s": step_s},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch

    import paper_2405_11922_gb300 as abg
    import synth

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    g = synth.make_config3(seed=rank, scale=args.scale)
    csc = csc_of(g)
    p = abg.params(**PARAMS, procrustes=args.nci == "procrustes",
                   bf16_propagation=args.precision in ("bf16-propagation", "bf16"),
                   bf16_contract=args.precision in ("bf16-contract", "bf16"))
    stream = torch.cuda.current_stream()
    graph = abg.abg_create(g, device=local_rank, stream=stream, csc=csc)
    labels = torch.empty(g.n_u, dtype=torch.int32).pin_memory().numpy()

    for _ in range(args.warmup):
        abg.abg_cluster(graph, p, labels, stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id_for_smi(local_rank))
    barrier()
    l0 = abg.abg_launch_count()
    results = []
    with sampler:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            _, res = abg.abg_cluster(graph, p, labels, stream)
            results.append(res)
        ev1.record(stream)
        barrier()
    launches = abg.abg_launch_count() - l0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    clocks = sampler.summary()
    prop_ms = statistics.median(r.ms_phase[1] for r in results)
    phase_ms = [statistics.median(r.ms_phase[i] for r in results) for i in range(6)]
    quality = quality_of(g, labels, results[-1])
    variants = {}
    if args.precision == "fp32" and rank == 0 and not args.no_variant:
        # the same solve with the BF16 options on the same resident graph: the products with R
        # in BF16 on the tensor cores (SpMM in FP32), then also W / Z stored in BF16
        variants = time_variants(abg, torch, graph, g, labels, results, stream, args)
    graph.close()

    # ---- end to end through the C ABI from pinned host memory ----
    pin = PinnedGraph(g, csc)
    for _ in range(1):
        gh = abg.abg_create(pin, device=local_rank, stream=stream, csc=pin.csc)
        abg.abg_cluster(gh, p, labels, stream)
        gh.close()
    barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        gh = abg.abg_create(pin, device=local_rank, stream=stream, csc=pin.csc)
        abg.abg_cluster(gh, p, labels, stream)
        gh.close()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")

    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    prop_prec = "bf16" if args.precision in ("bf16-propagation", "bf16") else "fp32"
    pbytes = propagation_bytes(g, PARAMS["d"], PARAMS["gamma"], prop_prec)
    achieved = pbytes / (prop_ms / 1e3) / 1e9
    value = job_value(world, args.steps, elapsed)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32+bf16",
        "data": "synthetic",
        "config": config_of(args.nci, args.precision,
                            f"{world} independent solves (one graph per rank)" if world > 1
                            else "single GPU", g, args.scale),
        "graph": {"n_u": int(g.n_u), "n_v": int(g.n_v), "nnz": int(g.nnz)},
        "tpo_prop_iters_per_s": PARAMS["gamma"] / (prop_ms / 1e3),
        "spmm_hbm_gbs": achieved,
        "phase_ms": dict(zip(["attributes", "propagation", "features", "svd_nmf", "nci",
                              "objective"], phase_ms)),
        "roofline": roofline_of(pbytes, prop_ms, peak, peak_kind, args.scale, prop_prec),
        "e2e": {"value": world * e2e_steps / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": pin.h2d_bytes, "d2h_bytes_per_step": int(labels.nbytes)},
        "gpu_launches": int(launches),
        "quality": quality,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    line.update(variants)
    if world == 1 and not args.no_systems:
        # the two systems patterns on their own workloads, against the plain one-graph-at-a-time
        # FP32 path on the same inputs (same T update of Algorithm 3 as the steps above)
        proc = args.nci == "procrustes"
        line["batched"] = batched_measure(abg, torch, args.sys_graphs, 2, 1, proc)
        line["served"] = served_measure(abg, torch, args.sys_requests, 200.0, 0, args.workers,
                                        args.max_batch, args.budget_gb, proc)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.nci == "procrustes")
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched workload: 512 independent graphs, one at a time vs one batch
# ---------------------------------------------------------------------------

def _gen_config4(g):
    import synth
    return synth.make_config4_graph(g)


def _gen_config5(r):
    import synth
    return synth.make_config5_request(r)


def _pool_map(fn, items, workers=None):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or min(16, os.cpu_count() or 4)) as pool:
        return pool.map(fn, items, chunksize=max(1, len(items) // 64))


def _params4(abg, g, i, procrustes=False):
    return abg.params(k=g.k, alpha=0.6, gamma=6, d=32, t_f=5, t_g=20, seed=i,
                      procrustes=procrustes)


BATCH_WORKLOAD = ("planted ABGs, |U| log-uniform [500, 50000], |V| = 1.5|U|, 10 edge draws per "
                  "u, k ~ U{3..30}, binary attributes d_u=300 at 3% reduced to d=32, alpha=0.6, "
                  "gamma=6, T_f=5, T_g=20")


def batched_measure(abg, torch, n: int, steps: int, warmup: int, procrustes: bool) -> dict:
    """n workload-4 graphs solved one at a time (graphs resident) and as one batch; both with
    the same parameters, labels compared graph by graph."""
    graphs = _pool_map(_gen_config4, list(range(n)))
    params = [_params4(abg, g, i, procrustes) for i, g in enumerate(graphs)]
    rows = sum(g.n_u for g in graphs)
    stream = torch.cuda.current_stream()
    # ---- plain: one graph at a time, graphs resident ----
    handles = [abg.abg_create(g, stream=stream) for g in graphs]
    for h, p in list(zip(handles, params))[:max(warmup, 1)]:
        abg.abg_cluster(h, p, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_labels = [abg.abg_cluster(h, p, stream=stream)[0] for h, p in zip(handles, params)]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    for h in handles:
        h.close()
    # ---- batched: all graphs in one batch, resident ----
    batch = abg.abg_batch_create(graphs, stream=stream)
    for _ in range(max(1, warmup)):
        abg.abg_batch_cluster(batch, params, stream=stream)
    torch.cuda.synchronize()
    l0 = abg.abg_launch_count()
    t0 = time.perf_counter()
    for _ in range(steps):
        blab, bres = abg.abg_batch_cluster(batch, params, stream=stream)
    torch.cuda.synchronize()
    batch_s = (time.perf_counter() - t0) / steps
    launches = (abg.abg_launch_count() - l0) // steps
    batch.close()
    # ---- end to end: uploads included ----
    t0 = time.perf_counter()
    for g, p in zip(graphs, params):
        h = abg.abg_create(g, stream=stream)
        abg.abg_cluster(h, p, stream=stream)
        h.close()
    plain_e2e = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = abg.abg_batch_create(graphs, stream=stream)
    abg.abg_batch_cluster(b, params, stream=stream)
    b.close()
    batch_e2e = time.perf_counter() - t0
    same = 0
    off = 0
    for g, lab in zip(graphs, plain_labels):
        same += int(np.array_equal(blab[off:off + g.n_u], lab))
        off += g.n_u
    return {"graphs": n, "total_u": int(rows), "batched_solves_per_s": n / batch_s,
            "plain_solves_per_s": n / plain_s, "speedup_vs_plain": plain_s / batch_s,
            "ms_per_batch": 1e3 * batch_s,
            "e2e": {"batched_solves_per_s": n / batch_e2e, "plain_solves_per_s": n / plain_e2e},
            "identical_to_plain": f"{same}/{n}", "gpu_launches_per_batch": int(launches),
            "nci": NCI_NAMES["procrustes" if procrustes else "printed"]}


def run_batched(args):
    import torch

    import paper_2405_11922_gb300 as abg
    r = batched_measure(abg, torch, args.graphs, args.steps, args.warmup,
                        args.nci == "procrustes")
    line = {"metric": "batched TPO solves/s (many small ABGs per launch) vs one graph at a time",
            "value": r["batched_solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.graphs} {BATCH_WORKLOAD}", "total_u": r["total_u"],
                       "nci": r["nci"]}}
    line.update({k: r[k] for k in ("plain_solves_per_s", "speedup_vs_plain", "e2e",
                                   "identical_to_plain", "gpu_launches_per_batch")})
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# served workload: Poisson arrivals, continuous batching vs plain sequential
# ---------------------------------------------------------------------------

SERVE_WORKLOAD = ("Poisson arrivals; graphs as in the mid-size workload with |U| log-uniform "
                  "[1000, 1e6], |V| = 2.5|U|, 25 draws per u, k ~ U{5..100}, half dense d=128 "
                  "BF16, half sparse d_u=500 reduced to 64; alpha=0.6, gamma=6, T_f=5, T_g=20")


def served_measure(abg, torch, requests: int, rate: float, pool: int, workers: int,
                   max_batch: int, budget_gb: float, procrustes: bool) -> dict:
    """`requests` requests arriving as a Poisson process: served by the continuous-batching
    loop, then the same list one at a time (plain), each timed from its arrival; the served
    labels are compared with the plain ones. pool = 0 draws a fresh graph per request, else
    requests cycle through `pool` graphs."""
    import threading

    import synth
    n_graphs = requests if pool <= 0 else min(pool, requests)
    graphs = _pool_map(_gen_config5, list(range(n_graphs)))
    arrivals = synth.config5_arrivals(requests, rate=rate)
    reqs = []
    for r in range(requests):
        g = graphs[r % len(graphs)]
        p = abg.params(k=g.params["k"], alpha=0.6, gamma=6, d=g.params["d"], t_f=5, t_g=20,
                       seed=r, procrustes=procrustes)
        reqs.append((g, p))
    stream = torch.cuda.current_stream()
    # warm-up of both paths on a few requests
    for g, p in reqs[:3]:
        h = abg.abg_create(g, stream=stream)
        abg.abg_cluster(h, p, stream=stream)
        h.close()
    # ---- served ----
    sv = abg.Server(workers=workers, max_batch_graphs=max_batch,
                    hbm_budget_bytes=int(budget_gb * (1 << 30)))
    rids = [None] * len(reqs)
    t_start = time.perf_counter()

    def submitter():
        for i, (g, p) in enumerate(reqs):
            wait = t_start + arrivals[i] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            rids[i] = sv.submit(g, p)

    th = threading.Thread(target=submitter)
    th.start()
    served_lat, served_labels = [], []
    for i in range(len(reqs)):
        while rids[i] is None:
            time.sleep(0.0005)
        st, lab, _ = sv.poll(rids[i], -1)
        assert st == abg.ABG_OK, st
        served_lat.append(sv.stats()["latency_us_last"] / 1e6)
        served_labels.append(lab)
    th.join()
    served_total = time.perf_counter() - t_start
    stats = sv.stats()
    sv.close()
    # ---- plain sequential (same arrival process, one request at a time) ----
    plain_lat, same = [], 0
    t_start = time.perf_counter()
    for i, (g, p) in enumerate(reqs):
        wait = t_start + arrivals[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        h = abg.abg_create(g, stream=stream)
        lab, _ = abg.abg_cluster(h, p, stream=stream)
        h.close()
        plain_lat.append(time.perf_counter() - (t_start + arrivals[i]))
        same += int(np.array_equal(lab, served_labels[i]))
    plain_total = time.perf_counter() - t_start
    q = lambda v, x: float(np.percentile(v, x)) * 1e3
    return {"requests": requests, "rate_per_s": rate,
            "graphs": "a fresh graph per request" if n_graphs == requests
                      else f"{n_graphs} graphs cycled",
            "served": {"solves_per_s": len(reqs) / served_total, "p50_ms": q(served_lat, 50),
                       "p99_ms": q(served_lat, 99), "batches": stats["batches"],
                       "max_batch": stats["max_batch"]},
            "plain": {"solves_per_s": len(reqs) / plain_total, "p50_ms": q(plain_lat, 50),
                      "p99_ms": q(plain_lat, 99)},
            "identical_to_plain": f"{same}/{len(reqs)}", "workers": workers,
            "max_batch": max_batch, "nci": NCI_NAMES["procrustes" if procrustes else "printed"]}


def run_serve(args):
    import torch

    import paper_2405_11922_gb300 as abg
    r = served_measure(abg, torch, args.requests, args.rate, args.pool, args.workers,
                       args.max_batch, args.budget_gb, args.nci == "procrustes")
    line = {"metric": "served TPO solves/s and p50/p99 latency vs plain sequential FP32",
            "value": r["served"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 3,
            "ms_per_step": 1e3 / r["served"]["solves_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.requests} requests at {args.rate}/s, {r['graphs']}; "
                                   + SERVE_WORKLOAD, "workers": args.workers,
                       "max_batch": args.max_batch, "nci": r["nci"]},
            "served": r["served"], "plain": r["plain"],
            "identical_to_plain": r["identical_to_plain"]}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the smaller planted workloads (1: 2,000 x 3,000, d = 500 sparse; 2: 200k x 500k, d = 128
# reduced from 1,000 sparse attributes): solves/s and propagation rounds/s of one graph
# ---------------------------------------------------------------------------

def run_small_config(args):
    import torch

    import paper_2405_11922_gb300 as abg
    import synth
    if args.workload == "config1":
        g = synth.make_config1()
        pdict = dict(k=5, alpha=0.6, gamma=6, d=500, t_f=5, t_g=20, seed=0)
        label = ("planted ABG |U|=2000 |V|=3000, 20,000 unit edges, binary attributes d=500 "
                 "(no reduction), k=5, alpha=0.6, gamma=6, T_f=5, T_g=20")
    else:
        g = synth.make_config2()
        pdict = dict(k=20, alpha=0.6, gamma=6, d=128, t_f=5, t_g=20, seed=0)
        label = ("planted ABG |U|=200k |V|=500k, 5M edge draws (Zipf 2.1), TF-IDF-like sparse "
                 "attributes d_u=1000 reduced to d=128, k=20, alpha=0.6, gamma=6, T_f=5, T_g=20")
    p = abg.params(**pdict, bf16_propagation=args.precision in ("bf16-propagation", "bf16"),
                   bf16_contract=args.precision in ("bf16-contract", "bf16"))
    stream = torch.cuda.current_stream()
    h = abg.abg_create(g, stream=stream)
    for _ in range(args.warmup):
        abg.abg_cluster(h, p, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    ev0.record(stream)
    for _ in range(args.steps):
        results.append(abg.abg_cluster(h, p, stream=stream)[1])
    ev1.record(stream)
    torch.cuda.synchronize()
    el = ev0.elapsed_time(ev1) / 1e3
    h.close()
    phase = [statistics.median(r.ms_phase[i] for r in results) for i in range(6)]
    line = {"metric": "TPO solves/s and propagation rounds/s on one planted ABG",
            "value": args.steps / el, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f32+bf16",
            "data": "synthetic", "config": {"workload": label, "n_u": int(g.n_u),
                                            "n_v": int(g.n_v), "nnz": int(g.nnz),
                                            "precision": args.precision},
            "prop_rounds_per_s": pdict["gamma"] / (phase[1] / 1e3),
            "phase_ms": dict(zip(["attributes", "propagation", "features", "svd_nmf", "nci",
                                  "objective"], phase))}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = the benchmark)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="skip the batched and served measurements added to the default line")
    ap.add_argument("--sys-graphs", type=int, default=128,
                    help="default line: graphs of the batched measurement")
    ap.add_argument("--sys-requests", type=int, default=60,
                    help="default line: requests of the served measurement (fresh graph each)")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the BF16 variant timed after the FP32 steps")
    ap.add_argument("--workload", choices=["large", "batched", "serve", "config1", "config2"],
                    default="large")
    ap.add_argument("--graphs", type=int, default=512, help="batched workload: number of graphs")
    ap.add_argument("--requests", type=int, default=200, help="served workload: requests")
    ap.add_argument("--pool", type=int, default=0,
                    help="served workload: distinct graphs cycled (0 = a fresh graph per request)")
    ap.add_argument("--rate", type=float, default=200.0, help="served workload: arrivals/s")
    ap.add_argument("--workers", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--nci", choices=["procrustes", "printed"], default="procrustes",
                    help="T update of Algorithm 3 (the printed T = Phi^T Y collapses this "
                         "workload into one cluster)")
    ap.add_argument("--precision", choices=["fp32", "bf16-contract", "bf16-propagation", "bf16"],
                    default="fp32",
                    help="bf16-contract: products with R on the BF16 tensor cores; "
                         "bf16-propagation: W and Z stored in BF16 between the SpMMs; bf16: both "
                         "(accumulation is FP32 throughout)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload != "large":
        import torch
        torch.cuda.set_device(local_rank)
        {"batched": run_batched, "serve": run_serve, "config1": run_small_config,
         "config2": run_small_config}[args.workload](args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
