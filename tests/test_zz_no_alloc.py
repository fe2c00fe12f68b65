"""The allocation-free entry point against the regular one, through the C ABI.

hg_wedge_degrees_noalloc serves callers that cannot allocate device memory while
they run (services whose device memory is a fixed arena owned by someone else):
it takes only caller-owned device buffers and a fixed library array.  Each
hyperedge's degree must equal the oracle's |N(e_i)|, and the degrees must
reproduce the wedge statistics hg_build_wedges reports for the same hypergraph,
on consecutive calls (the fixed array keeps old contents).  This file is
collected last so a stopping run has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def transpose(e_ptr, e_idx, nv):
    rows = np.repeat(np.arange(len(e_ptr) - 1, dtype=np.int32), np.diff(e_ptr))
    order = np.argsort(e_idx, kind="stable")
    v_ptr = np.zeros(nv + 1, dtype=np.int64)
    np.cumsum(np.bincount(e_idx, minlength=nv), out=v_ptr[1:])
    return v_ptr, rows[order].astype(np.int32)


def regular_stats(hg, nv, e_ptr, e_idx):
    import torch

    s = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=s.cuda_stream)
    try:
        return hg.hg_build_wedges(g)
    finally:
        hg.hg_free(g)


@pytest.mark.parametrize("name", ["tiny_plain", "coauthor_prefix50k"])
def test_noalloc_degrees_match_build_wedges(hglib, name):
    import torch

    import hgen
    import oracle
    from conftest import load_json

    gold = load_json("workloads.json")[name]
    e_ptr, e_idx = hgen.generate(hgen.WORKLOADS[gold["workload"]])
    if gold["prefix_edges"] is not None:
        e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, gold["prefix_edges"])
    nv, ne = gold["num_vertices"], len(e_ptr) - 1
    v_ptr, v_idx = transpose(e_ptr, e_idx, nv)
    want = regular_stats(hglib, nv, e_ptr, e_idx)
    want_deg = oracle.degrees(e_ptr, e_idx, nv)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (e_ptr, e_idx, v_ptr, v_idx)]
    stream = torch.cuda.Stream()
    for _ in range(2):   # the second call sees the first call's leftovers
        deg = torch.full((ne,), -1, dtype=torch.int32, device=dev)
        wc = torch.full((1,), 7, dtype=torch.int64, device=dev)
        hglib.hg.hg_wedge_degrees_noalloc(ne, *t, deg, wc, stream=stream.cuda_stream)
        d = deg.cpu().numpy().astype(np.int64)
        assert d.tolist() == want_deg.tolist()   # every |N(e_i)|, element by element
        assert int(d.sum()) == 2 * want["W"]
        assert int(d.max()) == want["max_deg"]
        assert int((d * (d - 1) // 2).sum()) == want["connected"]
        assert int(wc.item()) == want["W_c"] == gold["W_c"]


def test_noalloc_rejects_rows_beyond_its_tables(hglib):
    import torch

    # a vertex in 20,000 hyperedges: each row gathers 19,999 > 16,384 incidences
    ne = 20_000
    e_ptr = np.arange(0, 2 * ne + 1, 2, dtype=np.int64)
    e_idx = np.stack([np.zeros(ne, np.int32), np.arange(1, ne + 1, dtype=np.int32)], 1).ravel()
    v_ptr, v_idx = transpose(e_ptr, e_idx, ne + 1)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (e_ptr, e_idx, v_ptr, v_idx)]
    deg = torch.zeros(ne, dtype=torch.int32, device=dev)
    wc = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(hglib.HgError) as e:
        hglib.hg.hg_wedge_degrees_noalloc(ne, *t, deg, wc)
    assert e.value.name == "HG_ERR_UNSUPPORTED"
