"""The autotuner (hg_autotune / hg_batch_autotune): every candidate it times gives the
oracle's counts bit for bit, and builds that use its choice do too.  Through the C ABI."""
import numpy as np
import pytest

from conftest import load_json

pytestmark = pytest.mark.gpu


def stored_masks(entry):
    out = [0] * 128
    for m, n in entry["masks"].items():
        out[int(m)] = n
    return out


def workload(name):
    import hgen

    gold = load_json("workloads.json")[name]
    e_ptr, e_idx = hgen.generate(hgen.WORKLOADS[gold["workload"]])
    if gold["prefix_edges"] is not None:
        e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, gold["prefix_edges"])
    return gold, e_ptr, e_idx


@pytest.mark.parametrize("name", ["tiny_plain", "coauthor_prefix50k", "tag_heavy_prefix2000",
                                  "dense_core"])
def test_every_candidate_gives_the_oracle_counts(hglib, name):
    import torch

    gold, e_ptr, e_idx = workload(name)
    stream = torch.cuda.Stream()
    g = hglib.hg_load_csr(gold["num_vertices"], len(e_ptr) - 1, e_ptr, e_idx,
                          stream=stream.cuda_stream)
    try:
        r = hglib.hg_autotune(g)
        # the handle is left counted with the choice
        assert hglib.hg_count_patterns(g).tolist() == gold["counts"]
        # a build with no tuning fields takes the handle's choice
        st = hglib.hg_build_wedges(g)
        counts = hglib.hg_count_patterns(g)
        masks = hglib.hg_mask_histogram(g)
    finally:
        hglib.hg_free(g)
    n = len(r["tried"])
    assert n >= 6 and r["tried"][0] == {k: 0 for k in r["tried"][0]}
    for k in range(n):
        assert r["counts"][k].tolist() == gold["counts"], r["tried"][k]
    assert r["best"] == r["tried"][r["best_index"]]
    assert r["best_ms"] == min(r["ms"][k] for k in range(n) if r["tried"][k] == r["best"])
    assert masks.tolist() == stored_masks(gold) and counts.tolist() == gold["counts"]
    assert st["W"] == gold["W"] and st["W_c"] == gold["W_c"]
    if name == "tag_heavy_prefix2000":   # hyperedges of 32+ vertices: the tile path is a candidate
        assert any(t["dense_min_size"] != 0 for t in r["tried"])


def test_each_tuning_field_alone_gives_the_same_counts(hglib):
    # the values the autotuner may pick, one at a time, through hg_build_wedges
    import torch

    gold, e_ptr, e_idx = workload("coauthor_prefix50k")
    stream = torch.cuda.Stream()
    g = hglib.hg_load_csr(gold["num_vertices"], len(e_ptr) - 1, e_ptr, e_idx,
                          stream=stream.cuda_stream)
    try:
        for kw in ({"warp_team_max": 64}, {"warp_team_max": 128}, {"gather_light_max": 32},
                   {"gather_light_max": 64}, {"gather_light_max": 128}, {"orient_exact": 1}):
            hglib.hg_build_wedges(g, **kw)
            assert hglib.hg_count_patterns(g).tolist() == gold["counts"], kw
            assert hglib.hg_mask_histogram(g).tolist() == stored_masks(gold), kw
            cs = hglib.hg_close_stats_get(g)
            if kw.get("warp_team_max") == 64:   # out-degree 65-256 now on block teams
                assert cs["bucket_teams"][1] == cs["bucket_teams"][2] == 0
                assert cs["bucket_teams"][3] > 0
    finally:
        hglib.hg_free(g)


def test_batch_autotune_keeps_every_member_exact(hglib):
    import torch

    import oracle
    from test_gpu_batch import random_members

    members = random_members(6, 40)
    nv, eoff, eptr, evtx = hglib.concat_members(members)
    stream = torch.cuda.Stream()
    b = hglib.hg_load_batch(nv, eoff, eptr, evtx, max_wave_edges=3000, stream=stream.cuda_stream)
    try:
        waves = hglib.hg_batch_waves(b)
        assert len(waves) > 1
        r = hglib.hg_batch_autotune(b)
        assert len(r["tried"]) >= 6
        assert all(c.tolist() == r["counts"][0].tolist() for c in r["counts"])
        hglib.hg_batch_build_wedges(b)   # every wave with the choice
        counts, _ = hglib.hg_batch_count_patterns(b)
        masks = hglib.hg_batch_mask_histogram(b)
    finally:
        hglib.hg_batch_free(b)
    for m, (n_v, p, i) in enumerate(members):
        ref = oracle.count(p, i, n_v)
        assert masks[m].tolist() == ref.masks.tolist(), m
        assert counts[m].tolist() == [int(x) for x in ref.counts], m
