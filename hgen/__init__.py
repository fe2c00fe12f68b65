"""Seeded synthetic hypergraph generator (shared input of the oracle and the CUDA path).

This package holds no part of the counting method: it draws hyperedges and
returns a hyperedge->vertex CSR (``e_ptr`` int64 [|E|+1], ``e_idx`` int32 [nnz],
rows sorted ascending, no repeated vertex inside a hyperedge, no two equal
hyperedges).  The native part is ``gen.c``; ``build()`` compiles it with plain
gcc and ``-ffp-contract=off`` so that x86-64 and AArch64 produce byte-identical
output.

The workloads below are shaped after the paper's data (Table 3: co-authorship,
tags, email ...).  Their recipe, one per named workload, is:

* ``tiny_plain``  |V|=1,000  |E|=2,000  sizes U{2..6}           Zipf(1.1) seed 0
* ``coauthor``    |V|=1e5    |E|=5e5    sizes power law 2.5 [2,25] Zipf(1.0) seed 1, vertex degree cap 100
* ``tag_heavy``   |V|=2e4    |E|=2e6    sizes log-normal(1.5,1.0) [2,200] Zipf(1.2) seed 2, degree cap 1000
* ``batched(s)``  |E| log-uniform [100, 2e5], |V|=|E|/4, power law 2.2 [2,50], Zipf(1.0), seed s, cap 100
* ``served(m)``   |E| log-uniform [1e3, 1e6], |V|=|E|/5, otherwise as ``coauthor``, seed 5000+m
* ``dense_core``  |V|=24     |E|=2,600  sizes U{3..6}         uniform popularity, seed 7

The degree cap withdraws a vertex from later draws once it is in that many
hyperedges; without it the Zipf head puts a single vertex in ~8% of all
hyperedges and the exact count needs >1e14 classified triples.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libhgen.so")

SIZE_UNIFORM, SIZE_POWERLAW, SIZE_LOGNORMAL = 0, 1, 2


class _Params(ctypes.Structure):
    _fields_ = [
        ("num_vertices", ctypes.c_int64),
        ("num_edges", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("size_dist", ctypes.c_int32),
        ("size_lo", ctypes.c_int32),
        ("size_hi", ctypes.c_int32),
        ("degree_cap", ctypes.c_int32),
        ("size_p1", ctypes.c_double),
        ("size_p2", ctypes.c_double),
        ("zipf_s", ctypes.c_double),
        ("dedup", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


@dataclass(frozen=True)
class HypergraphSpec:
    """Parameters of one synthetic hypergraph."""

    num_vertices: int
    num_edges: int
    seed: int
    size_dist: int = SIZE_UNIFORM
    size_lo: int = 2
    size_hi: int = 6
    size_p1: float = 0.0
    size_p2: float = 0.0
    zipf_s: float = 1.0
    degree_cap: int = 0
    dedup: bool = True
    name: str = "custom"

    def _c(self) -> _Params:
        return _Params(
            int(self.num_vertices), int(self.num_edges), int(self.seed) & (2**64 - 1),
            int(self.size_dist), int(self.size_lo), int(min(self.size_hi, self.num_vertices)),
            int(self.degree_cap), float(self.size_p1), float(self.size_p2), float(self.zipf_s),
            1 if self.dedup else 0, 0,
        )


def build(force: bool = False) -> str:
    """Compile gen.c into libhgen.so next to it (plain gcc, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.hgen_sizes.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p]
        lib.hgen_sizes.restype = ctypes.c_int
        lib.hgen_fill.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]
        lib.hgen_fill.restype = ctypes.c_int
        lib.hgen_loguniform_int.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                            ctypes.c_int64]
        lib.hgen_loguniform_int.restype = ctypes.c_int64
        lib.hgen_det_log.argtypes = [ctypes.c_double]
        lib.hgen_det_log.restype = ctypes.c_double
        lib.hgen_det_exp.argtypes = [ctypes.c_double]
        lib.hgen_det_exp.restype = ctypes.c_double
        _lib = lib
    return _lib


_ERRORS = {-1: "bad argument", -2: "out of memory", -3: "not enough available vertices",
           -4: "could not draw a fresh hyperedge"}


class DedupExhausted(RuntimeError):
    """The generator found no fresh hyperedge after many redraws."""


def generate(spec: HypergraphSpec) -> tuple[np.ndarray, np.ndarray]:
    """Return (e_ptr int64[|E|+1], e_idx int32[nnz]) for the spec."""
    lib = _load()
    p = spec._c()
    sizes = np.empty(spec.num_edges, dtype=np.int32)
    rc = lib.hgen_sizes(ctypes.byref(p), sizes.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"hgen_sizes: {_ERRORS.get(rc, rc)}")
    e_ptr = np.zeros(spec.num_edges + 1, dtype=np.int64)
    np.cumsum(sizes, out=e_ptr[1:])
    e_idx = np.empty(int(e_ptr[-1]), dtype=np.int32)
    rc = lib.hgen_fill(ctypes.byref(p), sizes.ctypes.data, e_ptr.ctypes.data, e_idx.ctypes.data)
    if rc == -4:
        raise DedupExhausted(f"hgen_fill ({spec.name}): {_ERRORS.get(rc, rc)}")
    if rc != 0:
        raise RuntimeError(f"hgen_fill: {_ERRORS.get(rc, rc)}")
    return e_ptr, e_idx


def generate_batch(specs: list[HypergraphSpec], threads: int = 0, redraw=None
                   ) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray, list[HypergraphSpec]]:
    """Generate many hypergraphs into one concatenated layout:
    (num_vertices int32[G], edge_off int64[G+1], edge_ptr int64[sum |E|+1],
    edge_vtx int32[sum nnz], specs used), member m's hyperedges at edge_off[m] ..
    edge_off[m+1]-1 with member-local vertex ids.  A member whose draw runs out of
    fresh hyperedges is drawn again from redraw(spec, r), r = 1, 2, ... (first that
    succeeds) when `redraw` is given.  Members are drawn in parallel threads (the C
    generator keeps no shared state and ctypes releases the GIL); the output does not
    depend on the thread count."""
    from concurrent.futures import ThreadPoolExecutor

    workers = threads if threads > 0 else (os.cpu_count() or 1)

    def run(sp0):
        sp, r = sp0, 0
        while True:
            try:
                return (sp, *generate(sp))
            except DedupExhausted:
                r += 1
                if redraw is None or r > 64:
                    raise
                sp = redraw(sp0, r)

    with ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(run, specs))
    G = len(parts)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    np.cumsum([len(p[1]) - 1 for p in parts], out=edge_off[1:])
    nnz = np.zeros(G + 1, dtype=np.int64)
    np.cumsum([int(p[1][-1]) for p in parts], out=nnz[1:])
    edge_ptr = np.empty(int(edge_off[-1]) + 1, dtype=np.int64)
    edge_vtx = np.empty(int(nnz[-1]), dtype=np.int32)

    def place(m):
        sp, e_ptr, e_idx = parts[m]
        edge_ptr[edge_off[m]:edge_off[m + 1]] = e_ptr[:-1] + nnz[m]
        edge_vtx[nnz[m]:nnz[m + 1]] = e_idx

    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(place, range(G)))
    edge_ptr[-1] = nnz[-1]
    nv = np.array([p[0].num_vertices for p in parts], dtype=np.int32)
    return nv, edge_off, edge_ptr, edge_vtx, [p[0] for p in parts]


def loguniform_int(seed: int, tag: int, lo: int, hi: int) -> int:
    return int(_load().hgen_loguniform_int(seed & (2**64 - 1), tag, lo, hi))


def csr_hash(e_ptr: np.ndarray, e_idx: np.ndarray) -> str:
    """Content hash of a CSR (little-endian int64 offsets then int32 ids)."""
    h = hashlib.blake2b(digest_size=16)
    h.update(np.ascontiguousarray(e_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(e_idx, dtype="<i4").tobytes())
    return h.hexdigest()


def prefix(e_ptr: np.ndarray, e_idx: np.ndarray, num_edges: int) -> tuple[np.ndarray, np.ndarray]:
    """The sub-hypergraph made of the first `num_edges` hyperedges of a CSR."""
    p = np.ascontiguousarray(e_ptr[: num_edges + 1])
    return p, np.ascontiguousarray(e_idx[: int(p[-1])])


# ---------------------------------------------------------------- named workloads

TINY_PLAIN = HypergraphSpec(1000, 2000, 0, SIZE_UNIFORM, 2, 6, zipf_s=1.1, name="tiny_plain")
COAUTHOR = HypergraphSpec(100_000, 500_000, 1, SIZE_POWERLAW, 2, 25, size_p1=2.5, zipf_s=1.0,
                          degree_cap=100, name="coauthor")
TAG_HEAVY = HypergraphSpec(20_000, 2_000_000, 2, SIZE_LOGNORMAL, 2, 200, size_p1=1.5,
                           size_p2=1.0, zipf_s=1.2, degree_cap=1000, name="tag_heavy")


def batched(seed: int) -> HypergraphSpec:
    """One member of the 4,096-hypergraph batch (seeds 100..4195)."""
    ne = loguniform_int(seed, 0, 100, 200_000)
    nv = max(ne // 4, 2)
    return HypergraphSpec(nv, ne, seed, SIZE_POWERLAW, 2, 50, size_p1=2.2, zipf_s=1.0,
                          degree_cap=100, name=f"batched_{seed}")


def batched_redraw(spec: HypergraphSpec, r: int) -> HypergraphSpec:
    """Batch member drawn again from seed + r * 2^32 (same sizes of |V| and |E|) when its
    own seed runs out of fresh hyperedges under the degree cap."""
    return replace(spec, seed=spec.seed + (r << 32))


def served(member: int) -> HypergraphSpec:
    """One of the 64 resident hypergraphs of the serving workload."""
    seed = 5000 + member
    ne = loguniform_int(seed, 0, 1000, 1_000_000)
    return replace(COAUTHOR, num_vertices=max(ne // 5, 2), num_edges=ne, seed=seed,
                   name=f"served_{member}")


# a dense core: every hyperedge meets most others, so hyperedges close with out-degrees
# up to ~1,200 after degree ordering (test input for the block-sized closure teams)
DENSE_CORE = HypergraphSpec(24, 2600, 7, SIZE_UNIFORM, 3, 6, zipf_s=0.0, name="dense_core")

WORKLOADS = {"tiny_plain": TINY_PLAIN, "coauthor": COAUTHOR, "tag_heavy": TAG_HEAVY,
             "dense_core": DENSE_CORE}


def hub(num_spokes: int, num_extra: int, seed: int) -> tuple[int, np.ndarray, np.ndarray]:
    """A hub vertex 0 in `num_spokes` hyperedges ({0, a, b}, every third one {0, a}, with
    fresh a, b), plus `num_extra` random pairs over the spoke vertices (duplicates
    dropped); hyperedges sorted lexicographically.  Returns (num_vertices, e_ptr, e_idx)."""
    rng = np.random.default_rng(seed)
    edges = [[0, 1 + 2 * k, 2 + 2 * k] if k % 3 else [0, 1 + 2 * k] for k in range(num_spokes)]
    for _ in range(num_extra):
        a, b = rng.choice(2 * num_spokes, 2, replace=False) + 1
        edges.append([int(a), int(b)])
    uniq = sorted({tuple(sorted(set(e))) for e in edges})
    e_ptr = np.zeros(len(uniq) + 1, dtype=np.int64)
    e_ptr[1:] = np.cumsum([len(e) for e in uniq])
    e_idx = np.array([v for e in uniq for v in e], dtype=np.int32)
    return 2 * num_spokes + 1, e_ptr, e_idx
