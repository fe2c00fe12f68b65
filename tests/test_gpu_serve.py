"""hg_server: every answer of a mixed, batched, concurrent query stream equals the
answer of the plain calls for that query alone (bit-exact counts, coefficients and
estimates), and the oracle's where it is cheap."""
import threading
import time

import numpy as np
import pytest

from conftest import csr_of

pytestmark = pytest.mark.gpu


def graphs():
    import hgen

    out = []
    base = hgen.generate(hgen.TINY_PLAIN)
    for pre in (150, 400, 900):
        out.append((1000, *hgen.prefix(*base, pre)))
    for m in (0, 3, 7):   # members of the serving workload shape, cut to stay small
        spec = hgen.served(m)
        e_ptr, e_idx = hgen.generate(spec)
        out.append((spec.num_vertices, *hgen.prefix(e_ptr, e_idx, min(len(e_ptr) - 1, 20_000))))
    out.append((6, *csr_of([[0, 1], [2, 3], [4, 5]])))   # no hyperwedge at all
    return out


def stream(n, n_graphs, seed):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.0, 1.0, 20)
    qs = []
    for k in range(n):
        kind = int(rng.integers(0, 3))
        qs.append({"kind": kind, "graph": int(rng.integers(0, n_graphs)), "seed": 77 + k,
                   "first_sample": int(rng.integers(0, 2**40)), "num_samples": 20_000,
                   "eps": eps})
    gaps = rng.exponential(1.0 / 4000.0, n)   # Poisson arrivals, 4000 per second
    return qs, np.cumsum(gaps)


def serve(hg, gs, qs, arrivals, **opt):
    srv = hg.Server(**opt)
    try:
        ids = [srv.add_graph(nv, p, i) for nv, p, i in gs]
        tickets = [None] * len(qs)

        def producer():
            t0 = time.perf_counter()
            for k, q in enumerate(qs):
                delay = arrivals[k] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets[k] = srv.submit(q["kind"], ids[q["graph"]], q["seed"], q["first_sample"],
                                        q["num_samples"], q["eps"])

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        res = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    return res, stats


def alone(hg, gs, q):
    import torch

    nv, e_ptr, e_idx = gs[q["graph"]]
    stream_ = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream_.cuda_stream)
    try:
        hg.hg_build_wedges(g)
        if q["kind"] == hg.HG_Q_ESTIMATE:
            raw, est = hg.hg_sample_estimate(g, q["seed"], q["first_sample"], q["num_samples"])
            return {"counts": raw, "est": est}
        counts = hg.hg_count_patterns(g)
        cc, open_, conn = hg.hg_clustering_coeff(g, q["eps"])
        return {"counts": counts, "cc": cc, "open": open_, "connected": conn}
    finally:
        hg.hg_free(g)


def same(hg, q, r, a):
    assert r["status"] == 0
    assert r["counts"].tolist() == a["counts"].tolist()
    if q["kind"] == hg.HG_Q_ESTIMATE:
        assert r["est"].tolist() == a["est"].tolist()
    if q["kind"] == hg.HG_Q_CLUSTERING:
        assert (np.isnan(r["cc"]) and np.isnan(a["cc"])) or r["cc"] == a["cc"]
        assert (r["open"], r["connected"]) == (a["open"], a["connected"])


def test_mixed_stream_answers_equal_alone(hglib):
    import oracle

    gs = graphs()
    qs, arr = stream(400, len(gs), 5)
    res, stats = serve(hglib, gs, qs, arr, workers=3)
    assert stats["submitted"] == len(qs)
    assert stats["batches"] < len(qs)            # queries did share batches
    cache = {}
    for q, r in zip(qs, res):
        est = q["kind"] == hglib.HG_Q_ESTIMATE
        key = (q["graph"], est) + ((q["seed"], q["first_sample"]) if est else ())
        if key not in cache:
            cache[key] = alone(hglib, gs, q)
        same(hglib, q, r, cache[key])
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    # the oracle on the small hypergraphs
    for k in (0, 1, 6):
        nv, e_ptr, e_idx = gs[k]
        ref = oracle.count(e_ptr, e_idx, nv)
        for q, r in zip(qs, res):
            if q["graph"] == k and q["kind"] != hglib.HG_Q_ESTIMATE:
                assert r["counts"].tolist() == [int(x) for x in ref.counts]
                if q["kind"] == hglib.HG_Q_CLUSTERING:
                    cc = oracle.clustering_coeff(ref.counts, ref.open, q["eps"])
                    assert (np.isnan(cc) and np.isnan(r["cc"])) or r["cc"] == cc
    checked = 0
    for q, r in zip(qs, res):
        if q["kind"] == hglib.HG_Q_ESTIMATE and q["graph"] in (0, 1) and checked < 6:
            nv, e_ptr, e_idx = gs[q["graph"]]
            ref = oracle.sample_estimate(e_ptr, e_idx, nv, seed=q["seed"], first=q["first_sample"],
                                         num=q["num_samples"])
            assert r["counts"].tolist() == ref.raw.tolist()
            assert r["est"].tolist() == ref.est.tolist()
            checked += 1
    assert checked > 0


def test_no_batching_and_tiny_budget_give_the_same_answers(hglib):
    gs = graphs()
    qs, arr = stream(120, len(gs), 9)
    base, _ = serve(hglib, gs, qs, arr, workers=3)
    plain, st1 = serve(hglib, gs, qs, arr, workers=1, max_batch_queries=1)
    tight, st2 = serve(hglib, gs, qs, arr, workers=4, memory_budget=1)
    assert st1["batches"] == len(qs) and st1["max_concurrent_batches"] == 1
    assert st2["max_concurrent_batches"] == 1    # one batch at a time fits a 1-byte budget
    for q, a, b, c in zip(qs, base, plain, tight):
        for other in (b, c):
            assert other["counts"].tolist() == a["counts"].tolist()
            assert other["est"].tolist() == a["est"].tolist()
            if q["kind"] == hglib.HG_Q_CLUSTERING:
                assert (np.isnan(a["cc"]) and np.isnan(other["cc"])) or other["cc"] == a["cc"]


def test_server_argument_errors(hglib):
    srv = hglib.Server(workers=1)
    try:
        gid = srv.add_graph(4, *csr_of([[0, 1], [1, 2], [2, 3]]))
        with pytest.raises(hglib.HgError) as ei:
            srv.add_graph(4, *csr_of([[0, 1], [0, 1]]))
        assert ei.value.name == "HG_ERR_DUPLICATE_HYPEREDGE"
        with pytest.raises(hglib.HgError) as ei:
            srv.submit(hglib.HG_Q_COUNTS, gid + 5)
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        with pytest.raises(hglib.HgError) as ei:
            srv.submit(7, gid)
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        with pytest.raises(hglib.HgError) as ei:
            srv.wait(12345)
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        t = srv.submit(hglib.HG_Q_COUNTS, gid)
        r = srv.wait(t)
        assert r["status"] == 0 and r["counts"].tolist() == [0] * 21
        with pytest.raises(hglib.HgError):
            srv.wait(t)                           # each ticket once
        srv.drain()
    finally:
        srv.close()


def test_cancel_queued_queries(hglib):
    # one worker, one query per batch: of 40 queued counts, the last ones are still queued
    # when they are cancelled; a cancelled query waits out as HG_ERR_CANCELLED, the others
    # are answered as usual
    gs = graphs()
    srv = hglib.Server(workers=1, max_batch_queries=1)
    try:
        gid = srv.add_graph(*gs[5])
        tickets = [srv.submit(hglib.HG_Q_COUNTS, gid) for _ in range(40)]
        cancelled = []
        for t in tickets[20:]:
            try:
                srv.cancel(t)
                cancelled.append(t)
            except hglib.HgError as e:
                assert e.name == "HG_ERR_STATE"   # a worker had taken it already
        assert cancelled
        with pytest.raises(hglib.HgError) as ei:
            srv.cancel(10**9)
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        answered = None
        for t in tickets:
            r = srv.wait(t)
            if t in cancelled:
                assert r["status"] == 14 and r["worker"] == -1   # HG_ERR_CANCELLED
            else:
                assert r["status"] == 0
                answered = answered or r["counts"].tolist()
                assert r["counts"].tolist() == answered
        with pytest.raises(hglib.HgError) as ei:
            srv.cancel(tickets[0])   # already collected
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        srv.drain()
    finally:
        srv.close()


def test_cancelling_a_head_that_does_not_fit_admits_the_next(hglib):
    # Two workers and a memory budget that holds a long estimate A plus a small count C,
    # but not A plus the big count B.  Queued behind A: B (head, does not fit), then C.
    # Cancelling B must let the idle worker take C while A still runs (C starts before A
    # ends), not only once A completes.
    gs = graphs()
    a_graph, b_graph, c_graph = gs[3], gs[5], gs[0]

    def alone_bytes(kind, g, **q):
        srv = hglib.Server(workers=1)
        try:
            gid = srv.add_graph(*g)
            srv.wait(srv.submit(kind, gid, **q))
            return srv.stats()["max_in_flight_bytes"]
        finally:
            srv.close()

    long_q = {"seed": 5, "first_sample": 0, "num_samples": 150_000_000}
    ma = alone_bytes(hglib.HG_Q_ESTIMATE, a_graph, **long_q)
    mb = alone_bytes(hglib.HG_Q_COUNTS, b_graph)
    mc = alone_bytes(hglib.HG_Q_COUNTS, c_graph)
    assert mb > mc > 0 and ma > 0
    srv = hglib.Server(workers=2, memory_budget=ma + mc)
    try:
        ga, gb, gc = (srv.add_graph(*g) for g in (a_graph, b_graph, c_graph))
        ta = srv.submit(hglib.HG_Q_ESTIMATE, ga, **long_q)
        deadline = time.perf_counter() + 10.0
        while srv.stats()["batches"] < 1 and time.perf_counter() < deadline:
            time.sleep(0.001)
        tb = srv.submit(hglib.HG_Q_COUNTS, gb)
        tc = srv.submit(hglib.HG_Q_COUNTS, gc)
        time.sleep(0.02)
        srv.cancel(tb)   # A still runs, so B cannot have been taken
        rc = srv.wait(tc)
        ra = srv.wait(ta)
        assert srv.wait(tb)["status"] == 14   # HG_ERR_CANCELLED
        assert ra["status"] == 0 and rc["status"] == 0
        assert rc["t_start"] < ra["t_done"], (rc["t_start"], ra["t_done"])
    finally:
        srv.close()
