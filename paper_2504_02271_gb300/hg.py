"""Thin ctypes binding of libhg (include/hg.h).

Argument marshalling only: every step of the counting path runs in the CUDA
kernels of ``libhg.so``.  The functions keep the C names.  Device memory comes
from PyTorch's caching allocator (installed through ``hg_set_allocator``) and
work runs on the CUDA stream passed at load time (default: torch's current
stream).  If the library is missing the import of this module fails: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhg.so")

STATUS = {
    0: "HG_OK", 1: "HG_ERR_INVALID_ARG", 2: "HG_ERR_EMPTY_HYPEREDGE", 3: "HG_ERR_DUP_VERTEX",
    4: "HG_ERR_VERTEX_RANGE", 5: "HG_ERR_UNSORTED", 6: "HG_ERR_DUPLICATE_HYPEREDGE",
    7: "HG_ERR_OOM", 8: "HG_ERR_CUDA", 9: "HG_ERR_TIMEOUT", 10: "HG_ERR_STATE",
    11: "HG_ERR_UNSUPPORTED", 12: "HG_ERR_NO_DEVICE", 13: "HG_ERR_INTERNAL",
    14: "HG_ERR_CANCELLED",
}
HG_OK = 0

# every entry point declared in include/hg.h
EXPORTED = ("hg_set_allocator", "hg_load_csr", "hg_build_wedges", "hg_count_patterns",
            "hg_clustering_coeff", "hg_free", "hg_status_str", "hg_set_timing", "hg_kernel_times",
            "hg_pattern_table", "hg_close_stats_get", "hg_kernel_launches", "hg_wait_flag",
            "hg_wedge_degrees_noalloc", "hg_sample_estimate", "hg_load_batch",
            "hg_batch_build_wedges", "hg_batch_count_patterns", "hg_batch_clustering_coeff",
            "hg_batch_waves", "hg_batch_wave", "hg_batch_free", "hg_load_batch_members",
            "hg_server_create", "hg_server_add_graph", "hg_server_submit", "hg_server_wait",
            "hg_server_drain", "hg_server_cancel", "hg_server_stats_get", "hg_server_destroy",
            "hg_sample_estimate_adv", "hg_enumerate_pattern", "hg_sample_work_get",
            "hg_canonical_masks", "hg_mask_histogram", "hg_batch_mask_histogram",
            "hg_autotune", "hg_batch_autotune", "hg_count_owned", "hg_out_degrees")


class HgError(RuntimeError):
    """A call of the C ABI returned a status other than HG_OK; .name is the status name."""

    def __init__(self, fn: str, status: int, text: str):
        super().__init__(f"{fn}: {STATUS.get(status, status)} ({text})")
        self.status = status
        self.name = STATUS.get(status, str(status))


class _Tuning(ctypes.Structure):
    _fields_ = [("dense_min_size", ctypes.c_int32), ("dense_max_count", ctypes.c_int32),
                ("close_mode", ctypes.c_int32), ("orient_exact", ctypes.c_int32),
                ("gather_light_max", ctypes.c_int32), ("warp_team_max", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


TUNING_FIELDS = ("dense_min_size", "dense_max_count", "close_mode", "orient_exact",
                 "gather_light_max", "warp_team_max")


def _tuning(fields: dict):
    """A _Tuning from keyword fields, or None (NULL: the handle's own choice) when all are 0."""
    bad = set(fields) - set(TUNING_FIELDS)
    if bad:
        raise TypeError(f"unknown tuning fields {sorted(bad)}")
    if not any(int(v) for v in fields.values()):
        return None
    return _Tuning(*(int(fields.get(n, 0)) for n in TUNING_FIELDS))


def _tuning_dict(t) -> dict:
    return {n: int(getattr(t, n)) for n in TUNING_FIELDS}


_AUTOTUNE_MAX = 16


class _AutotuneResult(ctypes.Structure):
    _fields_ = [("best", _Tuning), ("best_ms", ctypes.c_float), ("best_index", ctypes.c_int32),
                ("num_tried", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tried", _Tuning * _AUTOTUNE_MAX), ("ms", ctypes.c_float * _AUTOTUNE_MAX),
                ("counts", (ctypes.c_uint64 * 21) * _AUTOTUNE_MAX)]


def _autotune_dict(r) -> dict:
    n = int(r.num_tried)
    return {"best": _tuning_dict(r.best), "best_ms": float(r.best_ms),
            "best_index": int(r.best_index),
            "tried": [_tuning_dict(r.tried[k]) for k in range(n)],
            "ms": [float(r.ms[k]) for k in range(n)],
            "counts": np.array([list(r.counts[k]) for k in range(n)], dtype=np.uint64)}


class _WedgeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("W", "W_t", "W_c", "connected", "max_deg",
                                                 "max_out_deg", "dense_edges", "reserved")]


class _CloseStats(ctypes.Structure):
    _fields_ = [("probes", ctypes.c_uint64), ("gathers", ctypes.c_uint64),
                ("out_entries", ctypes.c_uint64), ("teams", ctypes.c_uint64),
                ("bucket_teams", ctypes.c_uint64 * 8), ("bucket_probes", ctypes.c_uint64 * 8),
                ("bucket_gathers", ctypes.c_uint64 * 8),
                ("bucket_out_entries", ctypes.c_uint64 * 8)]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch_graphs", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("max_batch_queries", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class _Query(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("graph", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("first_sample", ctypes.c_uint64), ("num_samples", ctypes.c_uint64),
                ("eps", ctypes.c_double * 20)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("kind", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("counts", ctypes.c_uint64 * 21), ("est", ctypes.c_double * 21),
                ("cc", ctypes.c_double), ("open", ctypes.c_uint64), ("connected", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batch_queries", ctypes.c_int32),
                ("batch_graphs", ctypes.c_int32), ("worker", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "batches", "exact_batches",
                                                 "queries_batched", "max_in_flight_bytes",
                                                 "max_concurrent_batches", "budget_bytes")] + \
               [("now", ctypes.c_double)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_void_p)


def _open():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhg.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.hg_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, vp]
    lib.hg_wait_flag.argtypes = [vp, ctypes.c_int32, vp]
    lib.hg_load_csr.argtypes = [i32, i32, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.hg_build_wedges.argtypes = [vp, ctypes.POINTER(_Tuning), ctypes.POINTER(_WedgeStats)]
    lib.hg_count_patterns.argtypes = [vp, vp]
    lib.hg_clustering_coeff.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]
    lib.hg_free.argtypes = [vp]
    lib.hg_status_str.argtypes = [ctypes.c_int]
    lib.hg_status_str.restype = ctypes.c_char_p
    lib.hg_set_timing.argtypes = [vp, ctypes.c_int]
    lib.hg_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32)]
    lib.hg_pattern_table.argtypes = [vp]
    lib.hg_canonical_masks.argtypes = [vp]
    lib.hg_mask_histogram.argtypes = [vp, vp]
    lib.hg_count_owned.argtypes = [vp, vp, i32, vp, vp]
    lib.hg_out_degrees.argtypes = [vp, vp]
    lib.hg_batch_mask_histogram.argtypes = [vp, vp]
    lib.hg_autotune.argtypes = [vp, vp]
    lib.hg_batch_autotune.argtypes = [vp, i32, vp]
    lib.hg_close_stats_get.argtypes = [vp, ctypes.POINTER(_CloseStats)]
    lib.hg_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.hg_wedge_degrees_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp]
    u64 = ctypes.c_uint64
    lib.hg_sample_estimate.argtypes = [vp, u64, u64, u64, ctypes.c_double, vp, vp]
    lib.hg_sample_estimate_adv.argtypes = [vp, u64, u64, u64, ctypes.c_double, ctypes.c_uint32,
                                           vp, vp, vp]
    lib.hg_enumerate_pattern.argtypes = [vp, i32, vp, u64, ctypes.c_int, ctypes.POINTER(u64)]
    lib.hg_sample_work_get.argtypes = [vp, vp]
    lib.hg_load_batch.argtypes = [i32, vp, vp, vp, vp, ctypes.c_int, i64, vp, ctypes.POINTER(vp)]
    lib.hg_batch_build_wedges.argtypes = [vp, ctypes.POINTER(_Tuning)]
    lib.hg_batch_count_patterns.argtypes = [vp, vp, vp]
    lib.hg_batch_clustering_coeff.argtypes = [vp, vp, vp, vp, vp]
    lib.hg_batch_waves.argtypes = [vp, ctypes.POINTER(i32)]
    lib.hg_batch_wave.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32),
                                  ctypes.POINTER(i32)]
    lib.hg_batch_free.argtypes = [vp]
    lib.hg_load_batch_members.argtypes = [i32, vp, vp, vp, vp, ctypes.c_int, i64, vp,
                                          ctypes.POINTER(vp)]
    lib.hg_server_create.argtypes = [ctypes.POINTER(_ServerOptions), ctypes.POINTER(vp)]
    lib.hg_server_add_graph.argtypes = [vp, i32, i32, vp, vp, ctypes.c_int, ctypes.POINTER(i32)]
    lib.hg_server_submit.argtypes = [vp, ctypes.POINTER(_Query), ctypes.POINTER(u64)]
    lib.hg_server_wait.argtypes = [vp, u64, ctypes.POINTER(_Result)]
    lib.hg_server_drain.argtypes = [vp]
    lib.hg_server_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.hg_server_stats_get.argtypes = [vp, ctypes.POINTER(_ServerStats)]
    lib.hg_server_destroy.argtypes = [vp]
    for name in EXPORTED:
        if name != "hg_status_str":
            getattr(lib, name).restype = ctypes.c_int
    del i64
    return lib


_lib = _open()


def _check(fn: str, status: int) -> None:
    if status != HG_OK:
        raise HgError(fn, status, hg_status_str(status))


def hg_wait_flag(flag, limit_us: int, stream: int | None = None) -> None:
    """Bounded device wait on an int32 device flag (a one-element CUDA tensor or a device
    address); raises HgError HG_ERR_TIMEOUT when it is still zero after limit_us."""
    try:
        import torch
        if isinstance(flag, torch.Tensor):
            if not flag.is_cuda or flag.dtype != torch.int32:
                raise ValueError("flag must be an int32 CUDA tensor")
            flag = flag.data_ptr()
    except ImportError:
        pass
    if stream is None:
        stream = _default_stream()
    _check("hg_wait_flag", _lib.hg_wait_flag(ctypes.c_void_p(int(flag)), int(limit_us),
                                             ctypes.c_void_p(stream)))


def hg_status_str(status: int) -> str:
    """The library's one-line description of a status code."""
    return _lib.hg_status_str(int(status)).decode()


# ------------------------------------------------------------------ allocator

_torch_hooks = None


def use_torch_allocator() -> None:
    """Route libhg's device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, stream, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:  # out of memory -> NULL -> HG_ERR_OOM
            return None

    def _free(ptr, _nbytes, _stream, _ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check("hg_set_allocator", _lib.hg_set_allocator(hooks[0], hooks[1], None))
    _torch_hooks = hooks


def use_default_allocator() -> None:
    """Back to cudaMallocAsync / cudaFreeAsync on the handle's stream."""
    global _torch_hooks
    _check("hg_set_allocator", _lib.hg_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
    _torch_hooks = None


def hg_set_allocator(alloc, free, ctx=None) -> None:
    """Install raw ctypes hooks (see include/hg.h); pass None, None for the default."""
    if alloc is None and free is None:
        use_default_allocator()
        return
    _check("hg_set_allocator", _lib.hg_set_allocator(alloc, free, ctx))


# ------------------------------------------------------------------ handle API

@dataclass
class Graph:
    """An hg_graph handle plus what the binding needs to keep alive."""

    ptr: int
    stream: int
    num_vertices: int
    num_edges: int
    nnz: int
    owned: bool = True   # False for the wave handles a Batch lends out

    def __del__(self):
        if self.ptr and self.owned:
            try:
                _lib.hg_free(ctypes.c_void_p(self.ptr))
            except Exception:
                pass
            self.ptr = 0


def _as_ptr(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.int64: torch.int64, np.int32: torch.int32}[dtype]
            if x.dtype != want or not x.is_contiguous():
                x = x.to(want).contiguous()
            return x.data_ptr(), bool(x.is_cuda), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, False, a


def _default_stream() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def hg_load_csr(num_vertices: int, num_edges: int, edge_ptr, edge_vtx, stream: int | None = None
                ) -> Graph:
    """Validate and upload a hyperedge->vertex CSR; returns a Graph handle."""
    p_ptr, p_dev, keep1 = _as_ptr(edge_ptr, np.int64)
    v_ptr, v_dev, keep2 = _as_ptr(edge_vtx, np.int32)
    if p_dev != v_dev:
        raise ValueError("edge_ptr and edge_vtx must both be on the host or both on the device")
    if stream is None:
        stream = _default_stream()
    out = ctypes.c_void_p()
    st = _lib.hg_load_csr(int(num_vertices), int(num_edges), p_ptr, v_ptr, 1 if p_dev else 0,
                          ctypes.c_void_p(stream), ctypes.byref(out))
    del keep1, keep2
    _check("hg_load_csr", st)
    nnz = int(edge_ptr[-1])
    return Graph(int(out.value), int(stream), int(num_vertices), int(num_edges), nnz)


def hg_build_wedges(g: Graph, **tuning) -> dict:
    """Step one: hyperwedges, their types and the degree orientation; returns the stats.
    Keyword fields of hg_tuning (dense_min_size, dense_max_count, close_mode, orient_exact,
    gather_light_max, warp_team_max); none (or all 0) = the handle's autotuned choice if
    hg_autotune ran, else the defaults."""
    tun = _tuning(tuning)
    st = _WedgeStats()
    _check("hg_build_wedges",
           _lib.hg_build_wedges(ctypes.c_void_p(g.ptr),
                                ctypes.byref(tun) if tun is not None else None, ctypes.byref(st)))
    return {n: int(getattr(st, n)) for n, _ in _WedgeStats._fields_ if n != "reserved"}


def hg_autotune(g: Graph) -> dict:
    """Autotune the tuning of step one and two on this hypergraph (see include/hg.h); returns
    the choice and every candidate tried with its time (ms) and counts."""
    r = _AutotuneResult()
    _check("hg_autotune", _lib.hg_autotune(ctypes.c_void_p(g.ptr), ctypes.byref(r)))
    return _autotune_dict(r)


def hg_count_patterns(g: Graph) -> np.ndarray:
    """Step two: uint64[21] with [0] = total hyper-triangles and [p] = H[p]."""
    out = np.zeros(21, dtype=np.uint64)
    _check("hg_count_patterns", _lib.hg_count_patterns(ctypes.c_void_p(g.ptr), out.ctypes.data))
    return out


def hg_mask_histogram(g: Graph) -> np.ndarray:
    """uint64[128]: hyper-triangles of the last count per canonical region mask."""
    out = np.zeros(128, dtype=np.uint64)
    _check("hg_mask_histogram", _lib.hg_mask_histogram(ctypes.c_void_p(g.ptr), out.ctypes.data))
    return out


def hg_count_owned(g: Graph, owners) -> tuple[np.ndarray, np.ndarray]:
    """Step two over the hyper-triangles owned by `owners` (their lowest-ranked member):
    (counts uint64[21], canonical masks uint64[128])."""
    own = np.ascontiguousarray(np.asarray(owners, dtype=np.int32))
    counts = np.zeros(21, dtype=np.uint64)
    masks = np.zeros(128, dtype=np.uint64)
    _check("hg_count_owned", _lib.hg_count_owned(ctypes.c_void_p(g.ptr), own.ctypes.data,
                                                 len(own), counts.ctypes.data,
                                                 masks.ctypes.data))
    return counts, masks


def hg_out_degrees(g: Graph) -> np.ndarray:
    """int32[|E|]: each hyperedge's neighbours ranked above it in (|N(e)|, id)."""
    out = np.zeros(max(g.num_edges, 1), dtype=np.int32)
    _check("hg_out_degrees", _lib.hg_out_degrees(ctypes.c_void_p(g.ptr), out.ctypes.data))
    return out[:g.num_edges]


def hg_sample_estimate(g: Graph, seed: int, first_sample: int, num_samples: int,
                       sigma: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Hyperwedge-sampling estimate (Algorithm 6): (raw uint64[21], est float64[21])."""
    raw = np.zeros(21, dtype=np.uint64)
    est = np.zeros(21, dtype=np.float64)
    _check("hg_sample_estimate",
           _lib.hg_sample_estimate(ctypes.c_void_p(g.ptr), int(seed) & (2**64 - 1),
                                   int(first_sample), int(num_samples), float(sigma),
                                   raw.ctypes.data, est.ctypes.data))
    return raw, est


def hg_sample_estimate_adv(g: Graph, seed: int, first_sample: int, num_samples: int,
                           sigma: float = 1.0, class_mask: int = 15) -> tuple[np.ndarray, np.ndarray, dict]:
    """Appro-adv (Algorithm 7): (raw uint64[21], est float64[21], info)."""
    raw = np.zeros(21, dtype=np.uint64)
    est = np.zeros(21, dtype=np.float64)
    info = np.zeros(8, dtype=np.uint64)
    _check("hg_sample_estimate_adv",
           _lib.hg_sample_estimate_adv(ctypes.c_void_p(g.ptr), int(seed) & (2**64 - 1),
                                       int(first_sample), int(num_samples), float(sigma),
                                       int(class_mask), raw.ctypes.data, est.ctypes.data,
                                       info.ctypes.data))
    keys = ("W", "W_t", "W_c", "alpha_1", "alpha_2", "alpha_3", "alpha_4", "edges")
    return raw, est, {k: int(v) for k, v in zip(keys, info)}


def hg_enumerate_pattern(g: Graph, pattern: int, capacity: int | None = None, out=None):
    """(triples, total): the hyper-triangles of `pattern` (0 = all) as (i, j, k) rows.

    With `out` (a contiguous int32 torch tensor of shape [capacity, 3] on the device) the
    triples are written there; otherwise into a numpy array of `capacity` rows (default:
    the total, found by a first call with capacity 0)."""
    total = ctypes.c_uint64()
    if out is not None:
        _check("hg_enumerate_pattern",
               _lib.hg_enumerate_pattern(ctypes.c_void_p(g.ptr), int(pattern),
                                         ctypes.c_void_p(out.data_ptr()), out.shape[0], 1,
                                         ctypes.byref(total)))
        return out, int(total.value)
    if capacity is None:
        _check("hg_enumerate_pattern",
               _lib.hg_enumerate_pattern(ctypes.c_void_p(g.ptr), int(pattern), None, 0, 0,
                                         ctypes.byref(total)))
        capacity = int(total.value)
    arr = np.zeros((int(capacity), 3), dtype=np.int32)
    _check("hg_enumerate_pattern",
           _lib.hg_enumerate_pattern(ctypes.c_void_p(g.ptr), int(pattern),
                                     arr.ctypes.data if capacity else None, int(capacity), 0,
                                     ctypes.byref(total)))
    return arr[:min(int(capacity), int(total.value))], int(total.value)


def hg_clustering_coeff(g: Graph, eps) -> tuple[float, int, int]:
    """(cc, open hyper-triangles, connected triples) for weights eps[20] (Def. 5.1)."""
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    if e.shape != (20,):
        raise ValueError("eps must have 20 entries")
    cc = ctypes.c_double()
    op = ctypes.c_uint64()
    co = ctypes.c_uint64()
    _check("hg_clustering_coeff",
           _lib.hg_clustering_coeff(ctypes.c_void_p(g.ptr), e.ctypes.data, ctypes.byref(cc),
                                    ctypes.byref(op), ctypes.byref(co)))
    return float(cc.value), int(op.value), int(co.value)


def hg_close_stats_get(g: Graph) -> dict:
    """Work of the last hg_count_patterns or hg_count_owned: probes, gathers, out_entries,
    teams, bucket_teams."""
    st = _CloseStats()
    _check("hg_close_stats_get", _lib.hg_close_stats_get(ctypes.c_void_p(g.ptr), ctypes.byref(st)))
    return {"probes": int(st.probes), "gathers": int(st.gathers),
            "out_entries": int(st.out_entries), "teams": int(st.teams),
            "bucket_teams": [int(x) for x in st.bucket_teams],
            "bucket_probes": [int(x) for x in st.bucket_probes],
            "bucket_gathers": [int(x) for x in st.bucket_gathers],
            "bucket_out_entries": [int(x) for x in st.bucket_out_entries]}


def hg_kernel_launches() -> int:
    """Process-wide count of kernel launches issued by libhg."""
    n = ctypes.c_uint64()
    _check("hg_kernel_launches", _lib.hg_kernel_launches(ctypes.byref(n)))
    return int(n.value)


def hg_wedge_degrees_noalloc(num_edges: int, edge_ptr, edge_vtx, vertex_ptr, vertex_edge,
                             degrees, inclusion_wedges, stream: int | None = None) -> None:
    """Line-graph degrees and the inclusion-wedge count into caller-owned device tensors.

    For callers that cannot allocate device memory while they run: every argument
    is a device tensor the caller already holds (int64 edge_ptr / vertex_ptr,
    int32 edge_vtx / vertex_edge / degrees[|E|], one int64 for inclusion_wedges);
    the library uses only its own fixed 32 MiB device array.  See include/hg.h.
    """
    if stream is None:
        stream = _default_stream()
    _check("hg_wedge_degrees_noalloc",
           _lib.hg_wedge_degrees_noalloc(int(num_edges), edge_ptr.data_ptr(), edge_vtx.data_ptr(),
                                         vertex_ptr.data_ptr(), vertex_edge.data_ptr(),
                                         degrees.data_ptr(), inclusion_wedges.data_ptr(),
                                         ctypes.c_void_p(stream)))


def hg_pattern_table() -> np.ndarray:
    """uint8[128]: pattern (1..20, 0 = none) of each labelled 7-bit region mask."""
    out = np.zeros(128, dtype=np.uint8)
    _check("hg_pattern_table", _lib.hg_pattern_table(out.ctypes.data))
    return out


def hg_canonical_masks() -> np.ndarray:
    """uint8[128]: canonical form (smallest relabelling) of each labelled region mask."""
    out = np.zeros(128, dtype=np.uint8)
    _check("hg_canonical_masks", _lib.hg_canonical_masks(out.ctypes.data))
    return out


def hg_free(g: Graph) -> None:
    """Release the handle and its device memory; calling it again does nothing."""
    if g.ptr:
        p, g.ptr = g.ptr, 0
        _check("hg_free", _lib.hg_free(ctypes.c_void_p(p)))


def hg_set_timing(g: Graph, enable: bool) -> None:
    """Turn per-kernel-group event timing of the handle on or off (read by hg_kernel_times)."""
    _check("hg_set_timing", _lib.hg_set_timing(ctypes.c_void_p(g.ptr), 1 if enable else 0))


def hg_kernel_times(g: Graph) -> dict[str, tuple[float, int]]:
    """{kernel group: (summed ms, launches)} since the last read."""
    cap = 64
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_float * cap)()
    launches = (ctypes.c_int32 * cap)()
    n = ctypes.c_int32(cap)
    _check("hg_kernel_times", _lib.hg_kernel_times(ctypes.c_void_p(g.ptr), names, ms, launches,
                                                   ctypes.byref(n)))
    return {names[k].decode(): (float(ms[k]), int(launches[k])) for k in range(n.value)}


# ------------------------------------------------------------------ batches

@dataclass
class Batch:
    """An hg_batch handle: many hypergraphs counted in the same launches."""

    ptr: int
    stream: int
    num_graphs: int
    keep: object = None

    def __del__(self):
        if self.ptr:
            try:
                _lib.hg_batch_free(ctypes.c_void_p(self.ptr))
            except Exception:
                pass
            self.ptr = 0


def concat_members(members):
    """Member CSRs [(num_vertices, edge_ptr, edge_vtx), ...] -> the concatenated
    (num_vertices[G], edge_off[G+1], edge_ptr, edge_vtx) layout of hg_load_batch
    (vertex ids stay member-local)."""
    nv = np.array([int(m[0]) for m in members], dtype=np.int32)
    ne = np.array([len(m[1]) - 1 for m in members], dtype=np.int64)
    edge_off = np.zeros(len(members) + 1, dtype=np.int64)
    np.cumsum(ne, out=edge_off[1:])
    nnz = np.array([int(m[1][-1]) for m in members], dtype=np.int64)
    base = np.zeros(len(members) + 1, dtype=np.int64)
    np.cumsum(nnz, out=base[1:])
    edge_ptr = np.empty(int(edge_off[-1]) + 1, dtype=np.int64)
    for k, m in enumerate(members):
        edge_ptr[edge_off[k]:edge_off[k + 1]] = np.asarray(m[1][:-1], dtype=np.int64) + base[k]
    edge_ptr[-1] = base[-1]
    edge_vtx = (np.concatenate([np.asarray(m[2], dtype=np.int32) for m in members])
                if len(members) else np.zeros(0, dtype=np.int32))
    return nv, edge_off, edge_ptr, edge_vtx


def hg_load_batch(num_vertices, edge_off, edge_ptr, edge_vtx, max_wave_edges: int = 0,
                  stream: int | None = None) -> Batch:
    """Upload a batch (layout of concat_members); edge_ptr/edge_vtx on host or device."""
    nv = np.ascontiguousarray(num_vertices, dtype=np.int32)
    eo = np.ascontiguousarray(edge_off, dtype=np.int64)
    if len(eo) != len(nv) + 1:
        raise ValueError("edge_off must have num_graphs + 1 entries")
    p_ptr, p_dev, keep1 = _as_ptr(edge_ptr, np.int64)
    v_ptr, v_dev, keep2 = _as_ptr(edge_vtx, np.int32)
    if p_dev != v_dev:
        raise ValueError("edge_ptr and edge_vtx must both be on the host or both on the device")
    if stream is None:
        stream = _default_stream()
    out = ctypes.c_void_p()
    st = _lib.hg_load_batch(len(nv), nv.ctypes.data, eo.ctypes.data, ctypes.c_void_p(p_ptr),
                            ctypes.c_void_p(v_ptr), 1 if p_dev else 0, int(max_wave_edges),
                            ctypes.c_void_p(stream), ctypes.byref(out))
    del keep1, keep2
    _check("hg_load_batch", st)
    return Batch(int(out.value), int(stream), len(nv))


def hg_batch_build_wedges(b: Batch, **tuning) -> None:
    """Step one on every wave of the batch; the tuning fields are those of hg_build_wedges."""
    tun = _tuning(tuning)
    _check("hg_batch_build_wedges",
           _lib.hg_batch_build_wedges(ctypes.c_void_p(b.ptr),
                                      ctypes.byref(tun) if tun is not None else None))


def hg_batch_autotune(b: Batch, wave: int = -1) -> dict:
    """hg_autotune on one wave (-1: the one with the most hyperedges); every wave keeps the
    choice for hg_batch_build_wedges without tuning fields."""
    r = _AutotuneResult()
    _check("hg_batch_autotune",
           _lib.hg_batch_autotune(ctypes.c_void_p(b.ptr), int(wave), ctypes.byref(r)))
    return _autotune_dict(r)


def hg_batch_count_patterns(b: Batch) -> tuple[np.ndarray, dict]:
    """(counts uint64[G, 21], per-member wedge stats as uint64 arrays of length G)."""
    counts = np.zeros((b.num_graphs, 21), dtype=np.uint64)
    stats = (_WedgeStats * b.num_graphs)()
    _check("hg_batch_count_patterns",
           _lib.hg_batch_count_patterns(ctypes.c_void_p(b.ptr), counts.ctypes.data,
                                        ctypes.cast(stats, ctypes.c_void_p)))
    arr = np.ctypeslib.as_array(ctypes.cast(stats, ctypes.POINTER(ctypes.c_uint64)),
                                shape=(b.num_graphs, 8)).copy()
    names = [n for n, _ in _WedgeStats._fields_]
    return counts, {n: arr[:, k] for k, n in enumerate(names) if n != "reserved"}


def hg_batch_mask_histogram(b: Batch) -> np.ndarray:
    """uint64[G, 128]: each member's hyper-triangles per canonical region mask."""
    out = np.zeros((b.num_graphs, 128), dtype=np.uint64)
    _check("hg_batch_mask_histogram",
           _lib.hg_batch_mask_histogram(ctypes.c_void_p(b.ptr), out.ctypes.data))
    return out


def hg_batch_clustering_coeff(b: Batch, eps) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Per member (cc, open hyper-triangles, connected triples) for weights eps[20]."""
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    if e.shape != (20,):
        raise ValueError("eps must have 20 entries")
    cc = np.zeros(b.num_graphs, dtype=np.float64)
    op = np.zeros(b.num_graphs, dtype=np.uint64)
    co = np.zeros(b.num_graphs, dtype=np.uint64)
    _check("hg_batch_clustering_coeff",
           _lib.hg_batch_clustering_coeff(ctypes.c_void_p(b.ptr), e.ctypes.data, cc.ctypes.data,
                                          op.ctypes.data, co.ctypes.data))
    return cc, op, co


def hg_batch_waves(b: Batch) -> list[tuple[Graph, int, int]]:
    """[(wave handle (borrowed), first member, member count), ...]."""
    n = ctypes.c_int32()
    _check("hg_batch_waves", _lib.hg_batch_waves(ctypes.c_void_p(b.ptr), ctypes.byref(n)))
    out = []
    for k in range(n.value):
        w = ctypes.c_void_p()
        f = ctypes.c_int32()
        c = ctypes.c_int32()
        _check("hg_batch_wave", _lib.hg_batch_wave(ctypes.c_void_p(b.ptr), k, ctypes.byref(w),
                                                   ctypes.byref(f), ctypes.byref(c)))
        out.append((Graph(int(w.value), b.stream, 0, 0, 0, owned=False), f.value, c.value))
    return out


def hg_batch_free(b: Batch) -> None:
    """Release the batch and every wave's handle; calling it again does nothing."""
    if b.ptr:
        p, b.ptr = b.ptr, 0
        _check("hg_batch_free", _lib.hg_batch_free(ctypes.c_void_p(p)))


def hg_load_batch_members(members, max_wave_edges: int = 0, stream: int | None = None) -> Batch:
    """Batch of members stored apart: [(num_vertices, edge_ptr, edge_vtx), ...], each CSR
    with offsets from 0 (numpy on the host or torch tensors on the device, not mixed)."""
    keep, ptrs, idxs, devs = [], [], [], set()
    for _, p, i in members:
        pp, pd, k1 = _as_ptr(p, np.int64)
        ip, idv, k2 = _as_ptr(i, np.int32)
        devs.update((pd, idv))
        keep += [k1, k2]
        ptrs.append(pp)
        idxs.append(ip)
    if len(devs) > 1:
        raise ValueError("member CSRs must all be on the host or all on the device")
    nv = np.array([int(m[0]) for m in members], dtype=np.int32)
    ne = np.array([len(m[1]) - 1 for m in members], dtype=np.int32)
    pa = (ctypes.c_void_p * len(members))(*ptrs)
    ia = (ctypes.c_void_p * len(members))(*idxs)
    if stream is None:
        stream = _default_stream()
    out = ctypes.c_void_p()
    st = _lib.hg_load_batch_members(len(members), nv.ctypes.data, ne.ctypes.data,
                                    ctypes.cast(pa, ctypes.c_void_p), ctypes.cast(ia, ctypes.c_void_p),
                                    1 if devs == {True} else 0, int(max_wave_edges),
                                    ctypes.c_void_p(stream), ctypes.byref(out))
    del keep
    _check("hg_load_batch_members", st)
    return Batch(int(out.value), int(stream), len(members))


# ------------------------------------------------------------------ serving

HG_Q_COUNTS, HG_Q_CLUSTERING, HG_Q_ESTIMATE = 0, 1, 2


class Server:
    """hg_server: queries on resident hypergraphs with continuous batching."""

    def __init__(self, workers: int = 0, max_batch_graphs: int = 0, memory_budget: int = 0,
                 max_batch_queries: int = 0):
        opt = _ServerOptions(int(workers), int(max_batch_graphs), int(memory_budget),
                             int(max_batch_queries))
        out = ctypes.c_void_p()
        _check("hg_server_create", _lib.hg_server_create(ctypes.byref(opt), ctypes.byref(out)))
        self.ptr = int(out.value)

    def add_graph(self, num_vertices: int, edge_ptr, edge_vtx) -> int:
        """Register a hypergraph (host or device CSR, validated and copied); returns its id."""
        p_ptr, p_dev, k1 = _as_ptr(edge_ptr, np.int64)
        v_ptr, v_dev, k2 = _as_ptr(edge_vtx, np.int32)
        if p_dev != v_dev:
            raise ValueError("edge_ptr and edge_vtx must both be on the host or both on the device")
        gid = ctypes.c_int32()
        _check("hg_server_add_graph",
               _lib.hg_server_add_graph(ctypes.c_void_p(self.ptr), int(num_vertices),
                                        len(edge_ptr) - 1, ctypes.c_void_p(p_ptr),
                                        ctypes.c_void_p(v_ptr), 1 if p_dev else 0,
                                        ctypes.byref(gid)))
        del k1, k2
        return int(gid.value)

    def submit(self, kind: int, graph: int, seed: int = 0, first_sample: int = 0,
               num_samples: int = 0, eps=None) -> int:
        """Queue a query (HG_Q_COUNTS, HG_Q_CLUSTERING with eps[20], HG_Q_ESTIMATE with seed
        and sample range) on a registered hypergraph; returns its ticket."""
        q = _Query(int(kind), int(graph), int(seed) & (2**64 - 1), int(first_sample),
                   int(num_samples))
        if eps is not None:
            for k, x in enumerate(eps):
                q.eps[k] = float(x)
        t = ctypes.c_uint64()
        _check("hg_server_submit", _lib.hg_server_submit(ctypes.c_void_p(self.ptr), ctypes.byref(q),
                                                         ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int) -> dict:
        """Block until the ticket's query is answered and return the answer (once per ticket)."""
        r = _Result()
        _check("hg_server_wait", _lib.hg_server_wait(ctypes.c_void_p(self.ptr), int(ticket),
                                                     ctypes.byref(r)))
        return {"status": int(r.status), "kind": int(r.kind), "graph": int(r.graph),
                "counts": np.array(list(r.counts), dtype=np.uint64),
                "est": np.array(list(r.est), dtype=np.float64), "cc": float(r.cc),
                "open": int(r.open), "connected": int(r.connected), "t_submit": r.t_submit,
                "t_start": r.t_start, "t_done": r.t_done, "batch_queries": int(r.batch_queries),
                "batch_graphs": int(r.batch_graphs), "worker": int(r.worker)}

    def cancel(self, ticket: int) -> None:
        """Cancel a query no worker has taken yet; its wait() then has status HG_ERR_CANCELLED.
        Raises HgError HG_ERR_STATE when it is already running or answered."""
        _check("hg_server_cancel", _lib.hg_server_cancel(ctypes.c_void_p(self.ptr), int(ticket)))

    def drain(self) -> None:
        """Block until every queued query has been answered."""
        _check("hg_server_drain", _lib.hg_server_drain(ctypes.c_void_p(self.ptr)))

    def stats(self) -> dict:
        """Counters of the server: queries, batches, concurrency and memory in flight."""
        st = _ServerStats()
        _check("hg_server_stats_get", _lib.hg_server_stats_get(ctypes.c_void_p(self.ptr),
                                                               ctypes.byref(st)))
        return {n: (float(getattr(st, n)) if n == "now" else int(getattr(st, n)))
                for n, _ in _ServerStats._fields_}

    def close(self) -> None:
        """Answer what is queued, stop the workers and free the resident hypergraphs."""
        if self.ptr:
            p, self.ptr = self.ptr, 0
            _check("hg_server_destroy", _lib.hg_server_destroy(ctypes.c_void_p(p)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hg_sample_work_get(g: Graph) -> dict:
    """Reads of the last hg_sample_estimate: row-pointer reads, entries, vertex ids."""
    w = np.zeros(3, dtype=np.uint64)
    _check("hg_sample_work_get", _lib.hg_sample_work_get(ctypes.c_void_p(g.ptr), w.ctypes.data))
    return {"ptr_reads": int(w[0]), "entry_reads": int(w[1]), "vertex_reads": int(w[2])}
