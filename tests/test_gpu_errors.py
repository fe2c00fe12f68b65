"""Failure paths through the C ABI, none of which faults the GPU: a malformed CSR is
rejected with its status by the host checks or by the validation kernels (offsets are
checked before any row is read, a vertex id before it is used as an index), a duplicate
hyperedge by step one, an allocator that returns NULL gives HG_ERR_OOM before any
kernel runs; after each the context keeps working.  An empty hypergraph (no hyperedge)
is valid and has no hyper-triangle."""
import math

import numpy as np
import pytest

from conftest import csr_of

pytestmark = pytest.mark.gpu


def load(hg, nv, e_ptr, e_idx, ne=None):
    import torch

    stream = torch.cuda.Stream()
    ne = len(e_ptr) - 1 if ne is None else ne
    return hg.hg_load_csr(nv, ne, np.asarray(e_ptr, dtype=np.int64),
                          np.asarray(e_idx, dtype=np.int32), stream=stream.cuda_stream)


def still_works(hg):
    g = load(hg, 4, *csr_of([[0, 1], [1, 2], [0, 2]]))
    try:
        hg.hg_build_wedges(g)
        assert int(hg.hg_count_patterns(g)[0]) == 1
    finally:
        hg.hg_free(g)


@pytest.mark.parametrize("nv, e_ptr, e_idx, status", [
    (3, [0, 2, 2], [0, 1], "HG_ERR_EMPTY_HYPEREDGE"),
    (3, [0, 2, 1], [0], "HG_ERR_INVALID_ARG"),          # offsets decrease
    (3, [1, 2, 3], [0, 1, 2], "HG_ERR_INVALID_ARG"),    # first offset is not 0
    (3, [0, 2], [0, 3], "HG_ERR_VERTEX_RANGE"),
    (3, [0, 2], [-1, 0], "HG_ERR_VERTEX_RANGE"),
    (3, [0, 2], [1, 1], "HG_ERR_DUP_VERTEX"),
    (3, [0, 2], [2, 1], "HG_ERR_UNSORTED"),
    (0, [0, 2], [0, 1], "HG_ERR_INVALID_ARG"),          # no vertices
    (3, [0, -1], [], "HG_ERR_INVALID_ARG"),             # negative incidence count
])
def test_malformed_csr_is_rejected(hglib, nv, e_ptr, e_idx, status):
    with pytest.raises(hglib.HgError) as ei:
        load(hglib, nv, e_ptr, e_idx)
    assert ei.value.name == status
    still_works(hglib)


def test_negative_edge_count_is_rejected(hglib):
    with pytest.raises(hglib.HgError) as ei:
        load(hglib, 3, [0, 2], [0, 1], ne=-1)
    assert ei.value.name == "HG_ERR_INVALID_ARG"


def test_duplicate_hyperedge_is_rejected_by_step_one(hglib):
    g = load(hglib, 4, *csr_of([[0, 1], [1, 2], [0, 1]]))
    try:
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_build_wedges(g)
        assert ei.value.name == "HG_ERR_DUPLICATE_HYPEREDGE"
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_count_patterns(g)
        assert ei.value.name == "HG_ERR_STATE"
    finally:
        hglib.hg_free(g)
    still_works(hglib)


def test_allocator_returning_null_gives_oom(hglib):
    calls = []

    def alloc(nbytes, stream, ctx):
        calls.append(int(nbytes))
        return None

    def free(ptr, nbytes, stream, ctx):
        pass

    hooks = (hglib.hg._ALLOC_FN(alloc), hglib.hg._FREE_FN(free))
    hglib.hg_set_allocator(*hooks)
    try:
        with pytest.raises(hglib.HgError) as ei:
            load(hglib, 4, *csr_of([[0, 1], [1, 2], [0, 2]]))
        assert ei.value.name == "HG_ERR_OOM" and calls
    finally:
        hglib.use_torch_allocator()
    still_works(hglib)


def test_empty_hypergraph(hglib):
    g = load(hglib, 5, [0], [])
    try:
        st = hglib.hg_build_wedges(g)
        assert (st["W"], st["W_t"], st["W_c"], st["connected"]) == (0, 0, 0, 0)
        assert hglib.hg_count_patterns(g).tolist() == [0] * 21
        cc, open_, connected = hglib.hg_clustering_coeff(g, [1.0] * 20)
        assert (open_, connected) == (0, 0) and math.isnan(cc)
        raw, est = hglib.hg_sample_estimate(g, 1, 0, 1000)
        assert raw.tolist() == [0] * 21 and est.tolist() == [0.0] * 21
    finally:
        hglib.hg_free(g)


def test_bounded_wait_gives_up_and_the_context_survives(hglib):
    # a flag that nothing sets: the wait returns HG_ERR_TIMEOUT after its limit
    import time

    import torch

    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with pytest.raises(hglib.HgError) as ei:
        hglib.hg_wait_flag(flag, 20_000)   # 20 ms
    assert ei.value.name == "HG_ERR_TIMEOUT"
    assert 0.015 < time.perf_counter() - t0 < 5.0
    flag.fill_(1)
    torch.cuda.synchronize()
    hglib.hg_wait_flag(flag, 20_000)        # already set: returns at once
    with pytest.raises(hglib.HgError) as ei:
        hglib.hg_wait_flag(flag, -1)
    assert ei.value.name == "HG_ERR_INVALID_ARG"
    still_works(hglib)
