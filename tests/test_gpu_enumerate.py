"""Single-pattern enumeration (Sec. 2 problem statement) on the GPU vs the oracle.

The order of the found triples is not fixed, so the lists are compared sorted; with a
capacity below the total, what is unique (the total) is compared and every written
triple is checked to be a distinct hyper-triangle of the pattern."""
import numpy as np
import pytest

from conftest import csr_of, load_json

pytestmark = pytest.mark.gpu


def handle(hg, nv, e_ptr, e_idx):
    import torch

    stream = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    hg.hg_build_wedges(g)
    return g


def sorted_rows(a):
    a = np.asarray(a, dtype=np.int64).reshape(-1, 3)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))].tolist()


def test_every_pattern_matches_the_oracle(hglib):
    import hgen
    import oracle

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 250)
    g = handle(hglib, 1000, e_ptr, e_idx)
    try:
        counts = hglib.hg_count_patterns(g)
        for p in range(0, 21):
            got, total = hglib.hg_enumerate_pattern(g, p)
            want = oracle.enumerate_pattern(e_ptr, e_idx, 1000, p)
            assert total == len(want) == int(counts[p]), p
            assert sorted_rows(got) == want.tolist(), p
    finally:
        hglib.hg_free(g)


def test_paper_case_studies(hglib):
    for name in ("email", "coauthorship"):
        d = load_json("paper_examples.json")[name]
        e_ptr, e_idx = csr_of(d["hyperedges"])
        nv = 1 + max(v for e in d["hyperedges"] for v in e)
        g = handle(hglib, nv, e_ptr, e_idx)
        try:
            for tri, p in d["printed_triangles"]:
                got, _ = hglib.hg_enumerate_pattern(g, p)
                assert [x - 1 for x in tri] in sorted_rows(got), (name, tri)
            if name == "email":
                got, total = hglib.hg_enumerate_pattern(g, 5)
                assert total == 3
                assert sorted_rows(got) == sorted([x - 1 for x in t] for t, _ in d["printed_triangles"])
        finally:
            hglib.hg_free(g)


def test_capacity_and_device_output(hglib):
    import torch

    import hgen
    import oracle

    gold = load_json("workloads.json")["coauthor_prefix50k"]
    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.COAUTHOR), 50_000)
    g = handle(hglib, gold["num_vertices"], e_ptr, e_idx)
    try:
        # a rare pattern in full, on the device
        p = min(range(1, 21), key=lambda q: gold["counts"][q] if gold["counts"][q] else 1 << 62)
        out = torch.zeros((gold["counts"][p], 3), dtype=torch.int32, device="cuda")
        got, total = hglib.hg_enumerate_pattern(g, p, out=out)
        assert total == gold["counts"][p]
        want = oracle.enumerate_pattern(e_ptr, e_idx, gold["num_vertices"], p)
        assert sorted_rows(got.cpu().numpy()) == want.tolist()
        # a common pattern truncated to 1000 rows: exact total, valid distinct rows
        q = max(range(1, 21), key=lambda x: gold["counts"][x])
        got, total = hglib.hg_enumerate_pattern(g, q, capacity=1000)
        assert total == gold["counts"][q] and len(got) == 1000
        rows = got.tolist()
        assert len({tuple(r) for r in rows}) == 1000
        for i, j, k in rows[:200]:
            assert i < j < k
            sets = [set(e_idx[e_ptr[x]:e_ptr[x + 1]].tolist()) for x in (i, j, k)]
            assert oracle.classify(*sets) == q
        _, total0 = hglib.hg_enumerate_pattern(g, 0, capacity=0)
        assert total0 == gold["counts"][0]
    finally:
        hglib.hg_free(g)
