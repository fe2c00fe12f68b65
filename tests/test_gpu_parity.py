"""CUDA path vs the oracle, element by element, through the C ABI.  Integers:
bit-exact.  The canonical region-mask histogram (the pattern of every hyper-triangle
before the twenty patterns are numbered) is compared first, then the counts and the
wedge statistics."""
import numpy as np
import pytest

from conftest import csr_of, load_json

pytestmark = pytest.mark.gpu


def gpu_count(hg, nv, e_ptr, e_idx, **kw):
    import torch

    stream = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    try:
        stats = hg.hg_build_wedges(g, **kw)
        counts = hg.hg_count_patterns(g)
        stats["masks"] = hg.hg_mask_histogram(g).tolist()
        stats["close"] = hg.hg_close_stats_get(g)
        cc1, open_, connected = hg.hg_clustering_coeff(g, [1.0] * 20)
    finally:
        hg.hg_free(g)
    stats["open"] = open_
    stats["connected2"] = connected
    stats["cc1"] = cc1
    return counts, stats


def check_against_oracle(hg, nv, e_ptr, e_idx, ref=None):
    import oracle

    counts, st = gpu_count(hg, nv, e_ptr, e_idx)
    if ref is None:
        ref = oracle.count(e_ptr, e_idx, nv)
    assert st["masks"] == ref.masks.tolist()
    assert counts.tolist() == [int(x) for x in ref.counts]
    assert st["W"] == ref.W and st["W_c"] == ref.W_c and st["W_t"] == ref.W_t
    assert st["connected"] == ref.connected and st["max_deg"] == ref.max_deg
    assert st["open"] == ref.open
    return counts, st


def test_paper_email_example(hglib):
    # Sec. 6.2 (e-mail case study): three hyper-triangles, all pattern 5
    d = load_json("paper_examples.json")["email"]
    e_ptr, e_idx = csr_of(d["hyperedges"])
    counts, st = check_against_oracle(hglib, 200, e_ptr, e_idx)
    assert int(counts[5]) == 3 and int(counts[0]) == 3


def test_paper_coauthor_example(hglib):
    d = load_json("paper_examples.json")["coauthorship"]
    e_ptr, e_idx = csr_of(d["hyperedges"])
    check_against_oracle(hglib, 20, e_ptr, e_idx)


@pytest.mark.parametrize("seed", range(12))
def test_random_small(hglib, seed):
    import hgen

    # a draw that asks a small universe for more distinct hyperedges than it holds is
    # replaced by the next derived seed, so every case runs
    for attempt in range(20):
        s = seed + 1000 * attempt
        rng = np.random.default_rng(s)
        spec = hgen.HypergraphSpec(
            num_vertices=int(rng.integers(5, 60)), num_edges=int(rng.integers(3, 400)), seed=s,
            size_dist=hgen.SIZE_UNIFORM, size_lo=1, size_hi=int(rng.integers(2, 12)),
            zipf_s=float(rng.uniform(0.5, 1.5)), name="random_small")
        try:
            e_ptr, e_idx = hgen.generate(spec)
            break
        except RuntimeError:
            continue
    else:
        raise AssertionError("no drawable case among 20 derived seeds")
    check_against_oracle(hglib, spec.num_vertices, e_ptr, e_idx)


def stored_masks(entry):
    out = [0] * 128
    for m, n in entry["masks"].items():
        out[int(m)] = n
    return out


def test_wide_hyperedges(hglib):
    # lowest-ranked hyperedges with more than 32 vertices take the block kernel
    import hgen

    spec = hgen.HypergraphSpec(400, 300, 7, hgen.SIZE_UNIFORM, 20, 90, zipf_s=0.3, name="wide")
    e_ptr, e_idx = hgen.generate(spec)
    check_against_oracle(hglib, spec.num_vertices, e_ptr, e_idx)


def test_heavy_rows_and_every_team_shape_repeated(hglib):
    # A hub vertex in 6000 hyperedges: rows gather > 4096 candidates (global-scratch
    # gather blocks), and the out-degrees after degree ordering run from 0 to ~6000, so
    # every shared-table closure team shape runs - warp teams, block teams for out-degree
    # <= 1024, <= 2048 and <= 6144 (the cluster teams beyond are compared owner by owner
    # in test_gpu_owned.py).  About
    # 3.6e10 hyper-triangles, so the oracle's values are stored.  Five runs must agree
    # with the oracle every time (a schedule-dependent miscount would show as a run
    # that differs).
    import hgen

    gold = load_json("workloads.json")["hub6000"]
    nv, e_ptr, e_idx = hgen.hub(*gold["hub"])
    assert hgen.csr_hash(e_ptr, e_idx) == gold["csr_hash"]
    for run in range(5):
        counts, st = gpu_count(hglib, nv, e_ptr, e_idx)
        teams = st["close"]["bucket_teams"]
        # every shared-table shape (the hub's hyperedges have <= 3 vertices)
        assert all(teams[k] > 0 for k in (0, 1, 2, 3, 4, 5)), teams
        assert st["masks"] == stored_masks(gold), run
        assert counts.tolist() == gold["counts"], run
        for k in ("W", "W_c", "W_t", "connected", "open", "max_deg"):
            assert st[k] == gold[k], (run, k)


def test_tiny_plain_full(hglib):
    import hgen

    gold = load_json("workloads.json")["tiny_plain"]
    e_ptr, e_idx = hgen.generate(hgen.TINY_PLAIN)
    assert hgen.csr_hash(e_ptr, e_idx) == gold["csr_hash"]
    counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx)
    assert st["masks"] == stored_masks(gold)
    assert counts.tolist() == gold["counts"]
    assert st["W"] == gold["W"] and st["W_c"] == gold["W_c"] and st["open"] == gold["open"]


@pytest.mark.parametrize("name", ["coauthor_prefix50k", "tag_heavy_prefix1000",
                                  "tag_heavy_prefix2000", "coauthor", "dense_core"])
def test_workload_golden(hglib, name):
    import hgen

    data = load_json("workloads.json")
    if name not in data:
        pytest.skip(f"no stored oracle values for {name}")
    gold = data[name]
    spec = hgen.WORKLOADS[gold["workload"]]
    e_ptr, e_idx = hgen.generate(spec)
    if gold["prefix_edges"] is not None:
        e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, gold["prefix_edges"])
    assert hgen.csr_hash(e_ptr, e_idx) == gold["csr_hash"]
    counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx)
    assert st["masks"] == stored_masks(gold)
    assert counts.tolist() == gold["counts"]
    for k in ("W", "W_c", "W_t", "connected", "open", "max_deg"):
        assert st[k] == gold[k], k


@pytest.mark.parametrize("name", ["tiny_plain", "coauthor_prefix50k", "tag_heavy_prefix2000"])
def test_counts_do_not_depend_on_the_oriented_layout(hglib, name):
    # oriented rows in the exact layout (W entries) or with room for deg(i) (2W)
    import hgen

    gold = load_json("workloads.json")[name]
    e_ptr, e_idx = hgen.generate(hgen.WORKLOADS[gold["workload"]])
    if gold["prefix_edges"] is not None:
        e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, gold["prefix_edges"])
    counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx, orient_exact=1)
    assert st["masks"] == stored_masks(gold)
    assert counts.tolist() == gold["counts"]
    assert (st["W"], st["W_c"], st["connected"], st["open"]) == \
        (gold["W"], gold["W_c"], gold["connected"], gold["open"])


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["tiny_plain", "coauthor_prefix50k"])
def test_counts_do_not_depend_on_team_shape(hglib, name, mode):
    # every hyperedge through the global-table kernel (mode 1), or handed over to it
    # by the warp and block teams after they built their cuckoo tables (mode 2, the
    # path of a team whose stash overflows), gives the counts of the out-degree/size
    # buckets
    import hgen

    gold = load_json("workloads.json")[name]
    e_ptr, e_idx = hgen.generate(hgen.WORKLOADS[gold["workload"]])
    if gold["prefix_edges"] is not None:
        e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, gold["prefix_edges"])
    counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx, close_mode=mode)
    assert st["masks"] == stored_masks(gold)
    assert counts.tolist() == gold["counts"]
    probes = st["close"]["bucket_probes"]
    if mode == 2:   # the warp and block teams probed nothing; the global-table teams did it all
        assert st["close"]["bucket_teams"][:3] != [0, 0, 0]
        assert probes[:6] == [0] * 6 and probes[6] > 0
    assert sum(probes) == st["close"]["probes"]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_unpacked_rows_every_team_shape(hglib, mode):
    # three hyperedges of 300 vertices make omega exceed 8 bits, so rows are two int32
    # arrays and the warp and block teams keep 64-bit cuckoo items; the small hyperedges
    # still close in warp teams (out-degree <= 64, <= 128, <= 256) and 1024-teams
    import hgen
    import oracle

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 600)
    edges = [e_idx[e_ptr[i]:e_ptr[i + 1]].tolist() for i in range(len(e_ptr) - 1)]
    rng = np.random.default_rng(5)
    for _ in range(3):
        edges.append(rng.choice(1000, 300, replace=False).tolist())
    e_ptr, e_idx = csr_of(edges)
    counts, st = gpu_count(hglib, 1000, e_ptr, e_idx, close_mode=mode)
    ref = oracle.count(e_ptr, e_idx, 1000)
    assert st["masks"] == ref.masks.tolist()
    assert counts.tolist() == [int(x) for x in ref.counts]
    assert (st["W"], st["W_c"], st["connected"]) == (ref.W, ref.W_c, ref.connected)
    if mode == 0:
        teams = st["close"]["bucket_teams"]
        assert all(teams[k] > 0 for k in (0, 1, 2, 3, 6)), teams


def test_cuckoo_stash_and_handover(hglib):
    # Hyperedge ids that land on the same slot of both cuckoo tables of an
    # out-degree-64 warp team (the top 7 bits of x*A1 and of x*A2 mod 2^32 agree).
    # Thirteen hyperedges through one hub vertex, u = id 1 and twelve such ids, make a
    # clique ranked by id: the team of the k-th colliding id holds 11 - k of them, so
    # teams with 3..10 colliding keys scan the stash and teams with 11 or 12 overflow
    # it and are handed to the global-table teams.  Counts must equal the oracle's.
    M, A1, A2 = 0xFFFFFFFF, 0x9E3779B1, 0x85EBCA6B
    ids = [55818, 79684, 103550, 126573, 127416, 128259, 150439, 151282, 152125, 174305,
           175148, 175991]
    slots = {(((x * A1) & M) >> 25, ((x * A2) & M) >> 25) for x in ids}
    assert len(slots) == 1
    ne = 180_000
    edges = [[1000 + i] for i in range(ne)]   # singletons on private vertices
    edges[1] = [0, 1, 2, 400]
    for i, x in enumerate(ids):
        edges[x] = [0, 500 + i, 1 + i % 3]
    e_ptr, e_idx = csr_of(edges)
    counts, st = check_against_oracle(hglib, 1000 + ne, e_ptr, e_idx)
    assert int(counts[0]) == 286   # C(13, 3): every triple shares the hub
    probes = st["close"]["bucket_probes"]
    assert probes[0] > 0 and probes[6] > 0   # some teams closed in place, some handed over
    # exactly the teams with 12 and 11 colliding keys overflow (2 slots + 8 stashed)
    assert st["close"]["bucket_teams"][6] == 2


def test_rejected_tuning_leaves_the_handle_usable(hglib):
    import torch

    e_ptr, e_idx = csr_of([[0, 1], [1, 2], [0, 2], [2, 3]])
    stream = torch.cuda.Stream()
    g = hglib.hg_load_csr(4, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    try:
        hglib.hg_build_wedges(g)
        before = hglib.hg_count_patterns(g)
        for bad in ({"close_mode": 3}, {"close_mode": -1}, {"orient_exact": 2},
                    {"gather_light_max": 16}, {"gather_light_max": 600}, {"warp_team_max": 100}):
            with pytest.raises(hglib.HgError) as ei:
                hglib.hg_build_wedges(g, **bad)
            assert ei.value.name == "HG_ERR_INVALID_ARG"
        assert hglib.hg_count_patterns(g).tolist() == before.tolist()
    finally:
        hglib.hg_free(g)
    import oracle

    assert before.tolist() == [int(x) for x in oracle.count(e_ptr, e_idx, 4).counts]


def big_hyperedges(seed, ne, nv, lo, hi):
    import hgen

    spec = hgen.HypergraphSpec(nv, ne, seed, hgen.SIZE_UNIFORM, lo, hi, zipf_s=0.6, name="big")
    return spec, *hgen.generate(spec)


@pytest.mark.parametrize("seed", [1, 2])
def test_dense_tiles_match_oracle(hglib, seed):
    # every hyperedge heavy: all omega come from the tensor-core tiles
    import oracle

    spec, e_ptr, e_idx = big_hyperedges(seed, 400, 4000, 40, 100)
    counts, st = gpu_count(hglib, spec.num_vertices, e_ptr, e_idx, dense_min_size=40,
                           dense_max_count=1000)
    assert st["dense_edges"] == 400
    ref = oracle.count(e_ptr, e_idx, spec.num_vertices)
    assert st["masks"] == ref.masks.tolist()
    assert counts.tolist() == [int(x) for x in ref.counts]
    assert (st["W"], st["W_c"], st["connected"]) == (ref.W, ref.W_c, ref.connected)


def test_dense_tiles_mixed_heavy_and_light(hglib):
    # part of the hyperedges heavy: heavy x heavy from tiles, the rest hashed
    import hgen

    spec = hgen.HypergraphSpec(2000, 3000, 11, hgen.SIZE_LOGNORMAL, 2, 160, size_p1=2.5,
                               size_p2=1.0, zipf_s=0.9, name="mixed")
    e_ptr, e_idx = hgen.generate(spec)
    off, st_off = gpu_count(hglib, spec.num_vertices, e_ptr, e_idx, dense_min_size=-1)
    on, st_on = gpu_count(hglib, spec.num_vertices, e_ptr, e_idx, dense_min_size=24,
                          dense_max_count=700)
    assert st_off["dense_edges"] == 0 and 256 <= st_on["dense_edges"] <= 700
    assert on.tolist() == off.tolist()
    for k in ("W", "W_c", "connected", "max_deg", "open"):
        assert st_on[k] == st_off[k], k


def test_dense_tiles_tag_heavy_prefix(hglib):
    import hgen

    gold = load_json("workloads.json")["tag_heavy_prefix2000"]
    e_ptr, e_idx = hgen.generate(hgen.TAG_HEAVY)
    e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, 2000)
    counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx, dense_min_size=20,
                           dense_max_count=1200)
    assert st["dense_edges"] > 0
    assert st["masks"] == stored_masks(gold)
    assert counts.tolist() == gold["counts"]
    assert (st["W"], st["W_c"], st["connected"]) == (gold["W"], gold["W_c"], gold["connected"])


def test_dense_tiles_omega_above_255(hglib):
    # 96 heavy hyperedges of 350-450 vertices drawn from 600 share 190-330 vertices
    # pairwise, beyond one byte; light hyperedges on a partly overlapping range.  Every
    # heavy pair's omega comes from the tensor-core tiles (Def. 2.2), so a truncated or
    # saturated tile output would change omega, the hyperwedge types and the patterns.
    import oracle

    rng = np.random.default_rng(17)
    heavy = [sorted(rng.choice(600, int(rng.integers(350, 451)), replace=False).tolist())
             for _ in range(96)]
    light = [sorted(rng.choice(np.arange(560, 2560), int(rng.integers(2, 6)), replace=False).tolist())
             for _ in range(1500)]
    edges = heavy + light
    e_ptr, e_idx = csr_of(edges)
    assert len({tuple(e) for e in edges}) == len(edges)
    counts, st = gpu_count(hglib, 2560, e_ptr, e_idx, dense_min_size=300, dense_max_count=400)
    assert st["dense_edges"] == 96
    sets = [set(e) for e in heavy]
    assert max(len(sets[0] & sets[j]) for j in range(1, 96)) > 255
    ref = oracle.count(e_ptr, e_idx, 2560)
    assert st["masks"] == ref.masks.tolist()
    assert counts.tolist() == [int(x) for x in ref.counts]
    assert (st["W"], st["W_c"], st["connected"], st["open"]) == (ref.W, ref.W_c, ref.connected,
                                                                ref.open)


def test_block_teams_out_degree_257_to_1024_repeated(hglib):
    # 348 hyperedges of 5-10 vertices over 28: 34 hyperedges close with out-degree
    # 257-267 (block teams with shared tables); ten runs, each equal to the oracle
    import hgen
    import oracle

    spec = hgen.HypergraphSpec(28, 348, 1, hgen.SIZE_UNIFORM, 5, 10, zipf_s=0.0, name="dense28")
    e_ptr, e_idx = hgen.generate(spec)
    ref = oracle.count(e_ptr, e_idx, 28)
    for run in range(10):
        counts, st = gpu_count(hglib, 28, e_ptr, e_idx)
        assert st["close"]["bucket_teams"][3] > 0
        assert st["masks"] == ref.masks.tolist(), run
        assert counts.tolist() == [int(x) for x in ref.counts], run


def test_dense_core_block_teams_repeated(hglib):
    # 2,600 hyperedges of 3-6 vertices over 24: out-degrees up to ~1,200, so block
    # teams for out-degree <= 1024 and <= 2048 carry most of the work; every team shape
    # (0 = by out-degree, 1 = all global tables, 2 = built then handed over) and ten
    # default runs equal the stored oracle values
    import hgen

    gold = load_json("workloads.json")["dense_core"]
    e_ptr, e_idx = hgen.generate(hgen.DENSE_CORE)
    assert hgen.csr_hash(e_ptr, e_idx) == gold["csr_hash"]
    want = stored_masks(gold)
    for run in range(10):
        counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx)
        assert st["close"]["bucket_teams"][3] > 0 and st["close"]["bucket_teams"][4] > 0
        assert st["masks"] == want, run
        assert counts.tolist() == gold["counts"], run
    for mode in (1, 2):
        counts, st = gpu_count(hglib, gold["num_vertices"], e_ptr, e_idx, close_mode=mode)
        assert st["masks"] == want and counts.tolist() == gold["counts"], mode
