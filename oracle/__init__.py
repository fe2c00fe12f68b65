"""Oracle for exact hyper-triangle counting: plain, slow, obviously correct.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code,
table, header or constant generator with the CUDA library under
``paper_2504_02271_gb300/``, and it never imports that package.

The native part (``oracle.cpp``, built by ``build()`` with plain g++ and
OpenMP) enumerates triples the way Exact-bs does (Algorithm 1) or by brute
force, and classifies each hyper-triangle from its seven Venn regions
(Def. 2.4).  This module adds the fine-grained clustering coefficient of
Def. 5.1, evaluated in IEEE double on the host.

Parity status of each function:
  * counts, totals, wedge statistics, open triples: pinned by the paper's worked
    examples (Sec. 6.2), Algorithm 5's O(1) rules, closed forms and brute force;
  * the canonical region-mask histogram (128 bins; the pattern of each
    hyper-triangle before any numbering): pinned by closed forms (sunflowers,
    chains, ordinary graphs), a pure-Python brute force written from the region
    definitions of Sec. 2, brute force vs Exact-bs, and relabelling invariance;
  * the numbering of patterns 9, 11 and 13-20 inside the TTT class: parity
    unpinned (the paper prints that part of the numbering only in a figure
    that is not available); class membership of every pattern is pinned;
  * the samplers (Algorithms 6 and 7): pinned by their every-hyperwedge-once
    special cases (equal to the exact counts), split ranges, uniformity and
    unbiasedness; the Philox4x32-10 block function by the generator's published
    known-answer vectors (tests/golden/philox_kat.json).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

# pattern classes (Sec. 2): CCC = 1, TCC = 2-5, TTC = 6-8, TTT = 9-20;
# DenseTTT = 9-16, SparseTTT = 17-20 (Sec. 3.2)
CLASS_OF_PATTERN = {1: "CCC", **{p: "TCC" for p in range(2, 6)}, **{p: "TTC" for p in range(6, 9)},
                    **{p: "TTT" for p in range(9, 21)}}
DENSE_TTT = tuple(range(9, 17))
SPARSE_TTT = tuple(range(17, 21))

_ERR = {-2: "empty hyperedge", -3: "vertex id out of range", -4: "repeated vertex in a hyperedge",
        -5: "duplicate hyperedge", -6: "bad argument", -7: "pattern table inconsistent",
        -8: "unclassifiable triple"}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++ -O2 -fopenmp)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.c_void_p
        lib.oracle_count.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        lib.oracle_count.restype = ctypes.c_int
        lib.oracle_degrees.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_degrees.restype = ctypes.c_int
        lib.oracle_count_owned.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_count_owned.restype = ctypes.c_int
        lib.oracle_canonical_mask.argtypes = [ctypes.c_int]
        lib.oracle_canonical_mask.restype = ctypes.c_int
        for f in (lib.oracle_classify, lib.oracle_region_mask):
            f.argtypes = [i32p, ctypes.c_int, i32p, ctypes.c_int, i32p, ctypes.c_int]
            f.restype = ctypes.c_int
        lib.oracle_pattern_of_mask.argtypes = [ctypes.c_int]
        lib.oracle_pattern_of_mask.restype = ctypes.c_int
        lib.oracle_pattern_table_ok.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_sample_estimate.argtypes = [
            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_sample_estimate.restype = ctypes.c_int
        lib.oracle_subgraph.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.c_void_p]
        lib.oracle_subgraph.restype = ctypes.c_int32
        lib.oracle_sample_estimate_adv.argtypes = [
            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_sample_estimate_adv.restype = ctypes.c_int
        lib.oracle_enumerate.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_enumerate.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class OracleResult:
    counts: np.ndarray          # uint64[21]: [0] = T, [p] = H[p]
    W: int                      # hyperwedges (Def. 2.2)
    W_t: int                    # intersection type (Def. 2.3)
    W_c: int                    # inclusion type
    connected: int              # sum_i C(|N(e_i)|, 2)
    open: int                   # open hyper-triangles (Def. 5.1)
    max_deg: int                # max |N(e_i)|
    seconds: float
    threads: int
    # uint64[128]: masks[m] = hyper-triangles whose region mask in canonical form
    # (canonical_mask) is m (Sec. 2; independent of the pattern numbering)
    masks: np.ndarray = None

    @property
    def T(self) -> int:
        return int(self.counts[0])

    def H(self, p: int) -> int:
        return int(self.counts[p])


def count(e_ptr, e_idx, num_vertices: int, mode: str = "exact_bs", threads: int = 0,
          i_range: tuple[int, int] | None = None) -> OracleResult:
    """Exact per-pattern counts of the hypergraph given as a hyperedge->vertex CSR.

    mode ``exact_bs`` enumerates like Algorithm 1; ``brute`` tries every triple.
    ``i_range`` restricts counting to triangles whose smallest hyperedge id lies
    in [lo, hi) (a bounded sample of the same workload).
    """
    lib = _load()
    e_ptr = np.ascontiguousarray(e_ptr, dtype=np.int64)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    ne = len(e_ptr) - 1
    lo, hi = (0, ne) if i_range is None else i_range
    counts = np.zeros(21, dtype=np.uint64)
    stats = np.zeros(8, dtype=np.uint64)
    masks = np.zeros(128, dtype=np.uint64)
    secs = ctypes.c_double(0.0)
    m = {"exact_bs": 0, "brute": 1}[mode]
    rc = lib.oracle_count(int(num_vertices), int(ne), e_ptr.ctypes.data, e_idx.ctypes.data, m,
                          int(threads), int(lo), int(hi), counts.ctypes.data, stats.ctypes.data,
                          masks.ctypes.data, ctypes.byref(secs))
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    return OracleResult(counts, int(stats[0]), int(stats[1]), int(stats[2]), int(stats[3]),
                        int(stats[4]), int(stats[5]), float(secs.value),
                        int(threads) if threads > 0 else int(lib.oracle_max_threads()), masks)


def degrees(e_ptr, e_idx, num_vertices: int) -> np.ndarray:
    """int32[|E|]: |N(e_i)|, the number of other hyperedges sharing a vertex with e_i."""
    e_ptr = np.ascontiguousarray(e_ptr, dtype=np.int64)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    out = np.zeros(max(len(e_ptr) - 1, 1), dtype=np.int32)
    rc = _load().oracle_degrees(int(num_vertices), len(e_ptr) - 1, e_ptr.ctypes.data,
                                e_idx.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    return out[:len(e_ptr) - 1]


def count_owned(e_ptr, e_idx, num_vertices: int, owners, threads: int = 0):
    """Hyper-triangles by owner, the member ranked lowest in the order (|N(e)|, id).

    Returns (masks, above): masks uint64[n][128], masks[k][m] = hyper-triangles owned by
    owners[k] whose canonical region mask is m; above int32[n], the neighbours of
    owners[k] ranked above it."""
    e_ptr = np.ascontiguousarray(e_ptr, dtype=np.int64)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    own = np.ascontiguousarray(np.asarray(owners, dtype=np.int32))
    n = len(own)
    masks = np.zeros((max(n, 1), 128), dtype=np.uint64)
    above = np.zeros(max(n, 1), dtype=np.int32)
    rc = _load().oracle_count_owned(int(num_vertices), len(e_ptr) - 1, e_ptr.ctypes.data,
                                    e_idx.ctypes.data, own.ctypes.data, n, int(threads),
                                    above.ctypes.data, masks.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    return masks[:n], above[:n]


def _arr(x):
    a = np.ascontiguousarray(np.asarray(sorted(x), dtype=np.int32))
    return a, a.ctypes.data, len(a)


def classify(a, b, c) -> int:
    """Pattern (1..20) of three vertex sets; 0 if not a hyper-triangle; -1 if two are equal."""
    A, B, C = _arr(a), _arr(b), _arr(c)
    return int(_load().oracle_classify(A[1], A[2], B[1], B[2], C[1], C[2]))


def region_mask(a, b, c) -> int:
    """7-bit non-emptiness mask of regions (a)..(g) (bit 0 = region a) of (e_i, e_j, e_k)."""
    A, B, C = _arr(a), _arr(b), _arr(c)
    return int(_load().oracle_region_mask(A[1], A[2], B[1], B[2], C[1], C[2]))


def pattern_of_mask(mask: int) -> int:
    return int(_load().oracle_pattern_of_mask(int(mask)))


def canonical_mask(mask: int) -> int:
    """Smallest of the six relabellings of a labelled region mask (Sec. 2)."""
    return int(_load().oracle_canonical_mask(int(mask)))


def table_ok() -> bool:
    return bool(_load().oracle_pattern_table_ok())


def philox4x32_10(counter, key):
    """Philox4x32-10 block (Salmon et al., SC'11): 4 output words of a counter and key."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return [int(x) for x in out]


@dataclass
class SampleEstimate:
    raw: np.ndarray      # uint64[21]: triangles counted for the drawn hyperwedges ([0] = total)
    est: np.ndarray      # float64[21]: raw * (W / samples) / sigma^3
    W: int


def sample_estimate(e_ptr, e_idx, num_vertices: int, seed: int, first: int, num: int,
                    sigma: float = 1.0, identity_draws: bool = False, threads: int = 0
                    ) -> SampleEstimate:
    """Hyperwedge-sampling estimate of Algorithm 6 (Appro-bs) for samples first .. first+num-1."""
    lib = _load()
    e_ptr = np.ascontiguousarray(e_ptr, dtype=np.int64)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    raw = np.zeros(21, dtype=np.uint64)
    est = np.zeros(21, dtype=np.float64)
    W = ctypes.c_uint64(0)
    rc = lib.oracle_sample_estimate(int(num_vertices), len(e_ptr) - 1, e_ptr.ctypes.data,
                                    e_idx.ctypes.data, seed & (2**64 - 1), int(first), int(num),
                                    float(sigma), 1 if identity_draws else 0, int(threads),
                                    raw.ctypes.data, est.ctypes.data, ctypes.byref(W))
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    return SampleEstimate(raw, est, int(W.value))


def enumerate_pattern(e_ptr, e_idx, num_vertices: int, pattern: int, mode: str = "exact_bs",
                      threads: int = 0) -> np.ndarray:
    """int32[T_p, 3]: the hyper-triangles of `pattern` (0 = all) as i < j < k, sorted."""
    lib = _load()
    e_ptr = np.ascontiguousarray(e_ptr, dtype=np.int64)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    m = {"exact_bs": 0, "brute": 1}[mode]
    total = ctypes.c_uint64(0)
    rc = lib.oracle_enumerate(int(num_vertices), len(e_ptr) - 1, e_ptr.ctypes.data, e_idx.ctypes.data,
                              m, int(pattern), int(threads), None, 0, ctypes.byref(total))
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    out = np.zeros((int(total.value), 3), dtype=np.int32)
    rc = lib.oracle_enumerate(int(num_vertices), len(e_ptr) - 1, e_ptr.ctypes.data, e_idx.ctypes.data,
                              m, int(pattern), int(threads), out.ctypes.data, int(total.value),
                              ctypes.byref(total))
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    return out


def subgraph(num_edges: int, seed: int, sigma: float) -> np.ndarray:
    """Ids (ascending) of the hyperedges kept in G' for sampling proportion sigma
    (Algorithms 6-7, the sigma|E| draw): the ceil(sigma |E|) smallest Philox priorities."""
    kept = np.zeros(max(num_edges, 1), dtype=np.int32)
    n = _load().oracle_subgraph(int(num_edges), seed & (2**64 - 1), float(sigma), kept.ctypes.data)
    if n < 0:
        raise ValueError("oracle: bad argument")
    return kept[:n].copy()


@dataclass
class AdvEstimate:
    raw: np.ndarray       # uint64[21]
    est: np.ndarray       # float64[21]
    W: int
    W_t: int
    W_c: int
    alphas: tuple         # samples of the TTT, CCC, TTC, TCC sets
    edges: int            # |E'|


CLASS_BITS = {"CCC": 1, "TCC": 2, "TTC": 4, "TTT": 8}


def sample_estimate_adv(e_ptr, e_idx, num_vertices: int, seed: int, first: int, num: int,
                        sigma: float = 1.0, class_mask: int = 15, identity_draws: bool = False,
                        threads: int = 0) -> AdvEstimate:
    """Appro-adv (Algorithm 7): per-class hyperwedge sampling from W^t and W^c."""
    lib = _load()
    e_ptr = np.ascontiguousarray(e_ptr, dtype=np.int64)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    raw = np.zeros(21, dtype=np.uint64)
    est = np.zeros(21, dtype=np.float64)
    info = np.zeros(8, dtype=np.uint64)
    rc = lib.oracle_sample_estimate_adv(int(num_vertices), len(e_ptr) - 1, e_ptr.ctypes.data,
                                        e_idx.ctypes.data, seed & (2**64 - 1), int(first), int(num),
                                        float(sigma), int(class_mask), 1 if identity_draws else 0,
                                        int(threads), raw.ctypes.data, est.ctypes.data,
                                        info.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")
    return AdvEstimate(raw, est, int(info[0]), int(info[1]), int(info[2]),
                       tuple(int(x) for x in info[3:7]), int(info[7]))


def clustering_coeff(counts, open_triples: int, eps) -> float:
    """Fine-grained hypergraph clustering coefficient (Def. 5.1).

    3 * sum_p eps_p |triangles of pattern p| / |open hyper-triangles|, summed
    over p = 1..20 in that order in IEEE double; NaN when there is no open
    hyper-triangle.
    """
    s = 0.0
    for p in range(1, 21):
        s += float(eps[p - 1]) * float(int(counts[p]))
    if open_triples == 0:
        return math.nan
    return 3.0 * s / float(open_triples)


def pattern_wise_cc(counts, open_triples: int) -> list[float]:
    """CC_p with eps = one-hot(p), p = 1..20 (the per-pattern view of Sec. 5)."""
    out = []
    for p in range(1, 21):
        eps = [0.0] * 20
        eps[p - 1] = 1.0
        out.append(clustering_coeff(counts, open_triples, eps))
    return out
