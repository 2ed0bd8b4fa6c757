"""Python binding of ``libabg.so`` (the C ABI declared in ``include/abg.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. Functions keep the C names. Host arrays are numpy arrays;
device buffers are PyTorch CUDA tensors (used only as device memory), and
streams are ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers.
There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libabg.so")

ABG_OK, ABG_PENDING = 0, 1
ABG_EINVAL, ABG_ENOMEM, ABG_EDEVICE = -1, -2, -3
ABG_ENOTADMITTED, ABG_ETIMEDOUT, ABG_ENOTFOUND, ABG_ECANCELLED, ABG_ENUMERIC = -4, -5, -6, -7, -8
ABG_X_DENSE_F32, ABG_X_DENSE_BF16, ABG_X_CSR_F32 = 0, 1, 2
ABG_STREAM_G, ABG_STREAM_OMEGA_R, ABG_STREAM_OMEGA_X = 1, 2, 3

_p = C.c_void_p
_i32, _i64, _u64, _f64 = C.c_int32, C.c_int64, C.c_uint64, C.c_double


class abg_graph_desc(C.Structure):
    _fields_ = [("n_u", _i64), ("n_v", _i64), ("nnz", _i64),
                ("u_ptr", _p), ("v_idx", _p), ("w", _p),
                ("v_ptr", _p), ("u_idx", _p), ("w_t", _p),
                ("d_u", _i32), ("x_kind", _i32),
                ("x", _p), ("x_ptr", _p), ("x_idx", _p), ("x_val", _p),
                ("device", _i32), ("side", _i32)]


class abg_params(C.Structure):
    _fields_ = [("k", _i32), ("gamma", _i32), ("d", _i32), ("t_f", _i32), ("t_g", _i32),
                ("oversample", _i32), ("power_iters", _i32), ("nci_flags", _i32),
                ("alpha", _f64), ("seed", _u64), ("precision", _i32), ("options", _i32)]


class abg_result(C.Structure):
    _fields_ = [("objective", _f64), ("trace_obj", _f64), ("min_margin", _f64),
                ("last_changes", _i32), ("empty_clusters", _i32), ("clamped_rows", _i32),
                ("chol_breakdowns", _i32), ("ms_phase", C.c_float * 6), ("nci_passes", _i32),
                ("reused_propagation", _i32), ("warm_started", _i32)]

    def as_dict(self) -> dict:
        return {f: (list(getattr(self, f)) if f == "ms_phase" else getattr(self, f))
                for f, _ in self._fields_}


class abg_server_opts(C.Structure):
    _fields_ = [("device", _i32), ("workers", _i32), ("hbm_budget_bytes", _i64),
                ("max_batch_graphs", _i32), ("batch_window_us", _i32), ("max_batch_rows", _i64)]


class abg_server_stats(C.Structure):
    _fields_ = [(f, _i64) for f in ("submitted", "completed", "failed", "rejected", "batches",
                                    "max_batch", "pending", "inflight_bytes", "latency_us_last",
                                    "propagations_reused")]


class AbgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (status {status})")
        self.status = status


# name -> (restype, argtypes); every symbol of include/abg.h
SIGNATURES = {
    "abg_strerror": (C.c_char_p, [C.c_int]),
    "abg_last_error": (C.c_char_p, []),
    "abg_params_default": (None, [_p]),
    "abg_launch_count": (_i64, []),
    "abg_tensor_core_launches": (_i64, []),
    "abg_spmm_tuned_shapes": (_i64, []),
    "abg_create": (C.c_int, [_p, _p, _p]),
    "abg_destroy": (None, [_p]),
    "abg_graph_footprint": (_i64, [_p]),
    "abg_solve_footprint": (_i64, [_p, _p]),
    "abg_cluster": (C.c_int, [_p, _p, _p, _p, _p]),
    "abg_batch_create": (C.c_int, [_p, _i32, _i32, _p, _p]),
    "abg_graph_segments": (_i32, [_p]),
    "abg_batch_cluster": (C.c_int, [_p, _p, _p, _p, _p]),
    "abg_server_opts_default": (None, [_p]),
    "abg_server_create": (C.c_int, [_p, _p]),
    "abg_server_destroy": (None, [_p]),
    "abg_submit_resident": (C.c_int, [_p, _p, _p, _p]),
    "abg_submit": (C.c_int, [_p, _p, _p, _p]),
    "abg_poll": (C.c_int, [_p, _u64, _i64, _p, _p]),
    "abg_server_get_stats": (C.c_int, [_p, _p]),
    "abg_reduce_attributes": (C.c_int, [_p, _i32, _i32, _i32, _u64, _p, _i64, _p]),
    "abg_propagate": (C.c_int, [_p, _p, _i64, _i32, _f64, _i32, _i32, _p, _i64, _p]),
    "abg_orthogonal_matrix": (C.c_int, [_u64, _i32, _p, _p]),
    "abg_random_features": (C.c_int, [_p, _i64, _i32, _i64, _u64, _p, _i64, _p, _p]),
    "abg_seed_factors": (C.c_int, [_p, _i64, _i32, _i64, _i32, _i32, _i32, _u64, _p, _i64, _p,
                                   _i64, _p, _i32, _p]),
    "abg_onmf": (C.c_int, [_p, _i64, _i32, _i64, _i32, _i32, _p, _i64, _p, _i64, _i32, _p]),
    "abg_nci": (C.c_int, [_p, _i64, _i32, _i64, _i32, _i32, _p, _p, _p, _p, _p, _p]),
    "abg_objective": (C.c_int, [_p, _i64, _i32, _i64, _p, _i32, _p, _p]),
    "abg_objective_noalloc": (C.c_int, [_p, _i64, _i32, _i64, _p, _i32, _p, _p]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str) -> int:
    if status < 0:
        L = lib()
        raise AbgError(status, where, f"{L.abg_strerror(status).decode()}: "
                                      f"{L.abg_last_error().decode()}")
    return status


def _ptr(a) -> int | None:
    """Address of a numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "host arrays must be C-contiguous"
        return a.ctypes.data
    return a.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ld(t) -> int:
    """Row stride (elements) of a 2-D torch tensor."""
    return int(t.stride(0))


ABG_NCI_PROCRUSTES = 1
ABG_NCI_EARLY_STOP = 2
ABG_PRECISION_FP32 = 0
ABG_BF16_CONTRACT = 1
ABG_BF16_PROPAGATION = 2
ABG_REUSE_PROPAGATION = 1
ABG_WARM_START = 2


def params(k: int, alpha: float = 0.6, gamma: int = 6, d: int = 0, t_f: int = 5, t_g: int = 20,
           oversample: int = 10, power_iters: int = 4, seed: int = 0, procrustes: bool = False,
           early_stop: bool = False, bf16_propagation: bool = False,
           bf16_contract: bool = False, reuse_propagation: bool = False,
           warm_start: bool = False) -> abg_params:
    p = abg_params()
    lib().abg_params_default(C.byref(p))
    p.k, p.alpha, p.gamma, p.d, p.t_f, p.t_g = k, alpha, gamma, d, t_f, t_g
    p.oversample, p.power_iters, p.seed = oversample, power_iters, seed
    p.nci_flags = (ABG_NCI_PROCRUSTES if procrustes else 0) | (ABG_NCI_EARLY_STOP if early_stop else 0)
    p.precision = ((ABG_BF16_PROPAGATION if bf16_propagation else 0) |
                   (ABG_BF16_CONTRACT if bf16_contract else 0))
    p.options = ((ABG_REUSE_PROPAGATION if reuse_propagation else 0) |
                 (ABG_WARM_START if warm_start else 0))
    return p


class Graph:
    """Owns an ``abg_graph*``; the host arrays are copied at creation."""

    def __init__(self, handle: int, n_u: int, n_v: int, d_u: int):
        self.handle, self.n_u, self.n_v, self.d_u = handle, n_u, n_v, d_u

    def footprint(self) -> int:
        return int(lib().abg_graph_footprint(self.handle))

    def close(self):
        if self.handle:
            lib().abg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


ABG_SIDE_U = 0
ABG_SIDE_V = 1


def abg_create(g, device: int = 0, stream=None, csc=None, side: int = ABG_SIDE_U) -> Graph:
    """Upload an ABG. ``g`` carries n_u, n_v, u_ptr, v_idx, w, d_u, x_kind, x / x_ptr,
    x_idx, x_val (see ``synth.ABG``). ``csc`` = optional (v_ptr, u_idx, w_t) host arrays.
    ``side = ABG_SIDE_V`` clusters V: the attributes in ``g`` then describe the V nodes."""
    keep = []

    def h(a, dt):
        arr = _host(a, dt)
        keep.append(arr)
        return _ptr(arr)

    d = abg_graph_desc()
    d.n_u, d.n_v, d.nnz = int(g.n_u), int(g.n_v), int(g.u_ptr[-1])
    d.u_ptr, d.v_idx = h(g.u_ptr, np.int64), h(g.v_idx, np.int32)
    d.w = h(g.w, np.float32) if g.w is not None else None
    if csc is not None:
        d.v_ptr, d.u_idx = h(csc[0], np.int64), h(csc[1], np.int32)
        d.w_t = h(csc[2], np.float32) if csc[2] is not None else None
    d.d_u = int(g.d_u)
    kind = {"dense_f32": ABG_X_DENSE_F32, "dense_bf16": ABG_X_DENSE_BF16,
            "csr_f32": ABG_X_CSR_F32}[g.x_kind]
    d.x_kind = kind
    if kind == ABG_X_DENSE_F32:
        d.x = h(g.x, np.float32)
    elif kind == ABG_X_DENSE_BF16:
        d.x = h(g.x, np.uint16)
    else:
        d.x_ptr, d.x_idx, d.x_val = h(g.x_ptr, np.int64), h(g.x_idx, np.int32), h(g.x_val, np.float32)
    d.device = device
    d.side = side
    out = C.c_void_p()
    _check(lib().abg_create(C.byref(d), _stream(stream), C.byref(out)), "abg_create")
    if side == ABG_SIDE_V:          # the clustered side comes first
        return Graph(out.value, d.n_v, d.n_u, d.d_u)
    return Graph(out.value, d.n_u, d.n_v, d.d_u)


def abg_cluster(graph: Graph, p: abg_params, labels=None, stream=None):
    """Run Algorithms 1-3. ``labels``: int32 numpy array or CUDA tensor of length n_u
    (allocated on the host when None). Returns (labels, abg_result)."""
    if labels is None:
        labels = np.empty(graph.n_u, dtype=np.int32)
    res = abg_result()
    _check(lib().abg_cluster(graph.handle, C.byref(p), _stream(stream), _ptr(labels),
                             C.byref(res)), "abg_cluster")
    return labels, res


def abg_launch_count() -> int:
    return int(lib().abg_launch_count())


def abg_tensor_core_launches() -> int:
    return int(lib().abg_tensor_core_launches())


def abg_spmm_tuned_shapes() -> int:
    return int(lib().abg_spmm_tuned_shapes())


def _desc_of(g, keep: list, side: int = ABG_SIDE_U) -> abg_graph_desc:
    def h(a, dt):
        arr = _host(a, dt)
        keep.append(arr)
        return _ptr(arr)

    d = abg_graph_desc()
    d.n_u, d.n_v, d.nnz = int(g.n_u), int(g.n_v), int(g.u_ptr[-1])
    d.u_ptr, d.v_idx = h(g.u_ptr, np.int64), h(g.v_idx, np.int32)
    d.w = h(g.w, np.float32) if g.w is not None else None
    d.d_u = int(g.d_u)
    kind = {"dense_f32": ABG_X_DENSE_F32, "dense_bf16": ABG_X_DENSE_BF16,
            "csr_f32": ABG_X_CSR_F32}[g.x_kind]
    d.x_kind = kind
    if kind == ABG_X_DENSE_F32:
        d.x = h(g.x, np.float32)
    elif kind == ABG_X_DENSE_BF16:
        d.x = h(g.x, np.uint16)
    else:
        d.x_ptr, d.x_idx, d.x_val = h(g.x_ptr, np.int64), h(g.x_idx, np.int32), h(g.x_val, np.float32)
    d.side = side
    return d


def abg_batch_create(graphs, device: int = 0, stream=None, side: int = ABG_SIDE_U) -> Graph:
    """Stack several graphs (same d_u and attribute kind) into one batch (segments)."""
    keep = []
    arr = (abg_graph_desc * len(graphs))()
    for i, g in enumerate(graphs):
        arr[i] = _desc_of(g, keep, side)
        arr[i].device = device
    out = C.c_void_p()
    _check(lib().abg_batch_create(arr, len(graphs), device, _stream(stream), C.byref(out)),
           "abg_batch_create")
    nu, nv = sum(int(g.n_u) for g in graphs), sum(int(g.n_v) for g in graphs)
    if side == ABG_SIDE_V:
        nu, nv = nv, nu
    return Graph(out.value, nu, nv, int(graphs[0].d_u))


def abg_batch_cluster(batch: Graph, params_list, labels=None, stream=None):
    """Solve every graph of a batch; returns (stacked labels, list of abg_result)."""
    n = len(params_list)
    ps = (abg_params * n)(*params_list)
    res = (abg_result * n)()
    if labels is None:
        labels = np.empty(batch.n_u, dtype=np.int32)
    _check(lib().abg_batch_cluster(batch.handle, ps, _stream(stream), _ptr(labels), res),
           "abg_batch_cluster")
    return labels, list(res)


def abg_solve_footprint(graph: Graph, p: abg_params) -> int:
    return int(lib().abg_solve_footprint(graph.handle, C.byref(p)))


def abg_reduce_attributes(graph: Graph, d: int, x_out, oversample=10, power_iters=4, seed=0,
                          stream=None):
    _check(lib().abg_reduce_attributes(graph.handle, d, oversample, power_iters, seed,
                                       _ptr(x_out), _ld(x_out), _stream(stream)),
           "abg_reduce_attributes")
    return x_out


def abg_propagate(graph: Graph, x, d: int, alpha: float, gamma: int, zhat, stream=None,
                  bf16_propagation: bool = False):
    _check(lib().abg_propagate(graph.handle, _ptr(x), _ld(x) if x is not None else 0, d, alpha,
                               gamma, ABG_BF16_PROPAGATION if bf16_propagation else 0, _ptr(zhat),
                               _ld(zhat), _stream(stream)), "abg_propagate")
    return zhat


def abg_orthogonal_matrix(seed: int, d: int, q_out, stream=None):
    _check(lib().abg_orthogonal_matrix(seed, d, _ptr(q_out), _stream(stream)),
           "abg_orthogonal_matrix")
    return q_out


def abg_random_features(zhat, n: int, d: int, seed: int, r_out, stream=None) -> int:
    cl = C.c_int32(0)
    _check(lib().abg_random_features(_ptr(zhat), n, d, _ld(zhat), seed, _ptr(r_out), _ld(r_out),
                                     C.byref(cl), _stream(stream)), "abg_random_features")
    return cl.value


def abg_seed_factors(r, n: int, m: int, k: int, phi_out, h_out, sigma_out=None, oversample=10,
                     power_iters=4, seed=0, stream=None, bf16_contract: bool = False):
    _check(lib().abg_seed_factors(_ptr(r), n, m, _ld(r), k, oversample, power_iters, seed,
                                  _ptr(phi_out), _ld(phi_out), _ptr(h_out), _ld(h_out),
                                  _ptr(sigma_out), ABG_BF16_CONTRACT if bf16_contract else 0,
                                  _stream(stream)), "abg_seed_factors")


def abg_onmf(r, n: int, m: int, k: int, t_f: int, phi, h, stream=None,
             bf16_contract: bool = False):
    _check(lib().abg_onmf(_ptr(r), n, m, _ld(r), k, t_f, _ptr(phi), _ld(phi), _ptr(h), _ld(h),
                          ABG_BF16_CONTRACT if bf16_contract else 0, _stream(stream)),
           "abg_onmf")


def abg_nci(phi, n: int, k: int, t_g: int, labels_out, margin_out=None, t_out=None, stream=None,
            nci_flags: int = 0, with_passes: bool = False):
    """Returns the label changes of the last pass (and the passes run with ``with_passes``)."""
    lc = C.c_int32(0)
    np_ = C.c_int32(0)
    _check(lib().abg_nci(_ptr(phi), n, k, _ld(phi), t_g, nci_flags, _ptr(labels_out),
                         _ptr(margin_out), _ptr(t_out), C.byref(lc), C.byref(np_),
                         _stream(stream)), "abg_nci")
    return (lc.value, np_.value) if with_passes else lc.value


def abg_objective(r, n: int, m: int, labels, k: int, stream=None) -> tuple[float, float]:
    out = (C.c_double * 2)()
    _check(lib().abg_objective(_ptr(r), n, m, _ld(r), _ptr(labels), k, out, _stream(stream)),
           "abg_objective")
    return float(out[0]), float(out[1])


def abg_objective_noalloc(r, n: int, m: int, labels, k: int, stream=None) -> tuple[float, float]:
    """abg_objective without any device allocation: its scratch is a fixed array inside the
    library (see include/abg.h for the size limit and the sharing rules)."""
    out = (C.c_double * 2)()
    _check(lib().abg_objective_noalloc(_ptr(r), n, m, _ld(r), _ptr(labels), k, out,
                                       _stream(stream)), "abg_objective_noalloc")
    return float(out[0]), float(out[1])


class Server:
    """Continuous-batching request loop (abg_server_*). Submitted graphs' host arrays are kept
    alive here until the request is polled to a final status."""

    def __init__(self, device: int = 0, workers: int = 3, hbm_budget_bytes: int = 64 << 30,
                 max_batch_graphs: int = 64, batch_window_us: int = 0,
                 max_batch_rows: int = 4 << 20):
        o = abg_server_opts()
        lib().abg_server_opts_default(C.byref(o))
        o.device, o.workers, o.hbm_budget_bytes = device, workers, hbm_budget_bytes
        o.max_batch_graphs, o.batch_window_us, o.max_batch_rows = (max_batch_graphs,
                                                                   batch_window_us, max_batch_rows)
        h = C.c_void_p()
        _check(lib().abg_server_create(C.byref(o), C.byref(h)), "abg_server_create")
        self.handle = h.value
        self._keep = {}
        self._n_u = {}

    def submit(self, g, p: abg_params, side: int = ABG_SIDE_U) -> int:
        keep = []
        d = _desc_of(g, keep, side)
        rid = C.c_uint64(0)
        st = lib().abg_submit(self.handle, C.byref(d), C.byref(p), C.byref(rid))
        if st == ABG_ENOTADMITTED:
            return -int(rid.value)
        _check(st, "abg_submit")
        self._keep[rid.value] = (keep, d)
        self._n_u[rid.value] = int(g.n_v if side == ABG_SIDE_V else g.n_u)
        return int(rid.value)

    def submit_resident(self, graph: "Graph", p: abg_params) -> int:
        """Queue a re-solve of a graph already on the device (``abg_create``); ``graph`` must
        stay open until the request is polled to completion."""
        rid = C.c_uint64(0)
        st = lib().abg_submit_resident(self.handle, graph.handle, C.byref(p), C.byref(rid))
        if st == ABG_ENOTADMITTED:
            return -int(rid.value)
        _check(st, "abg_submit_resident")
        self._n_u[rid.value] = int(graph.n_u)
        return int(rid.value)

    def poll(self, rid: int, timeout_us: int = -1):
        """(status, labels or None, abg_result or None)."""
        n = self._n_u.get(abs(rid), 0)
        labels = np.empty(max(n, 1), dtype=np.int32)
        res = abg_result()
        st = lib().abg_poll(self.handle, abs(rid), timeout_us, _ptr(labels), C.byref(res))
        if st in (ABG_PENDING, ABG_ETIMEDOUT):
            return st, None, None
        self._keep.pop(abs(rid), None)
        self._n_u.pop(abs(rid), None)
        return st, (labels[:n] if st == ABG_OK else None), (res if st == ABG_OK else None)

    def stats(self) -> dict:
        s = abg_server_stats()
        _check(lib().abg_server_get_stats(self.handle, C.byref(s)), "abg_server_get_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if self.handle:
            lib().abg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
