"""Write the stored expected values of the generated workloads.

Every number written here comes from the oracle (``oracle/``) run on the
seeded generator's output (``hgen/``); nothing comes from the CUDA path.  The
CSR content hash is stored with each entry so a test can check that the
generator reproduced the same hypergraph before comparing counts.  ``masks``
maps each canonical region mask (the smallest of its six relabellings) to the
number of hyper-triangles that have it; absent masks have none.

Usage:  python tests/golden/make_golden.py [name ...]   (default: all)
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import hgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")

# name -> (spec, number of leading hyperedges or None for the whole hypergraph)
CASES = {
    "tiny_plain": (hgen.TINY_PLAIN, None),
    "tiny_plain_prefix200": (hgen.TINY_PLAIN, 200),
    "coauthor": (hgen.COAUTHOR, None),
    "coauthor_prefix50k": (hgen.COAUTHOR, 50_000),
    "tag_heavy_prefix1000": (hgen.TAG_HEAVY, 1_000),
    "tag_heavy_prefix2000": (hgen.TAG_HEAVY, 2_000),
    "dense_core": (hgen.DENSE_CORE, None),
}
# hub hypergraphs (hgen.hub): name -> (spokes, extra pairs, seed)
HUBS = {
    "hub6000": (6000, 200, 3),
    "hub3000": (3000, 0, 0),
}


def run(name: str) -> dict:
    if name in HUBS:
        nv, e_ptr, e_idx = hgen.hub(*HUBS[name])
        workload, pre = "hub", None
    else:
        spec, pre = CASES[name]
        nv, workload = spec.num_vertices, spec.name
        e_ptr, e_idx = hgen.generate(spec)
        if pre is not None:
            e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, pre)
    t0 = time.time()
    r = oracle.count(e_ptr, e_idx, nv)
    entry = {
        "workload": workload, "prefix_edges": pre, "num_vertices": nv,
        "num_edges": len(e_ptr) - 1, "nnz": int(e_ptr[-1]),
        "csr_hash": hgen.csr_hash(e_ptr, e_idx),
        "counts": [int(x) for x in r.counts],
        "masks": {str(m): int(r.masks[m]) for m in range(128) if r.masks[m]},
        "W": r.W, "W_t": r.W_t, "W_c": r.W_c,
        "connected": r.connected, "open": r.open, "max_deg": r.max_deg,
        "oracle_seconds": round(r.seconds, 2), "oracle_threads": r.threads,
    }
    if name in HUBS:
        entry["hub"] = list(HUBS[name])
    if pre is not None and pre <= 300:
        b = oracle.count(e_ptr, e_idx, nv, mode="brute")
        assert [int(x) for x in b.counts] == entry["counts"] and b.open == r.open
        assert b.masks.tolist() == r.masks.tolist()
        entry["brute_force_agrees"] = True
    print(f"{name}: T={r.T} W={r.W} {time.time() - t0:.1f}s", flush=True)
    return entry


def main(names: list[str]) -> None:
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for n in names or list(CASES) + list(HUBS):
        data[n] = run(n)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
