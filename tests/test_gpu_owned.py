"""Step two restricted to owners (hg_count_owned) against the oracle, through the C ABI.

Each hyper-triangle is found from its member ranked lowest in (|N(e)|, id), its owner.
hg_count_owned runs only the listed owners' teams with the kernels and team shapes of a
full count, so on a hypergraph too large for the oracle's full enumeration - the
tag-shaped configuration at its full 2,000,000 hyperedges - sampled owners of every team
shape are compared one by one with the oracle's per-owner histograms, and each owner's
out-degree with the oracle's count of neighbours ranked above it.  Bit-exact."""
import numpy as np
import pytest

from conftest import load_json

pytestmark = pytest.mark.gpu

WARP_MASK_BITS = 32     # |e_u| a warp or block team holds in one mask word
WIDE_LARGE_MIN = 4096   # |e_u| > 32: out-degrees above it go to the cluster-capable teams
BLOCK_MAX = 6144        # largest shared-table block team (packed rows)
BUCKET_NAMES = ("warp<=64", "warp<=128", "warp<=256", "block<=1024", "block<=2048",
                "block<=6144", "wide", "cluster")


def bucket_of(d, sz, warp_max=256):
    """The team shape of an owner with out-degree d and |e_u| = sz under the default tuning
    (packed rows)."""
    if d < 2:
        return -1
    if sz <= WARP_MASK_BITS and d <= warp_max:
        return 0 if d <= 64 else (1 if d <= 128 else 2)
    for k, lim in ((3, 1024), (4, 2048), (5, BLOCK_MAX)):
        if sz <= WARP_MASK_BITS and d <= lim:
            return k
    return 7 if d > WIDE_LARGE_MIN else 6


def loaded(hg, nv, e_ptr, e_idx):
    import torch

    stream = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    return g, stream


def test_owners_partition_the_count(hglib):
    import hgen
    import oracle

    gold = load_json("workloads.json")["coauthor_prefix50k"]
    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.COAUTHOR), gold["prefix_edges"])
    nv, ne = gold["num_vertices"], len(e_ptr) - 1
    g, _ = loaded(hglib, nv, e_ptr, e_idx)
    try:
        with pytest.raises(hglib.HgError) as e:
            hglib.hg_count_owned(g, [0])
        assert e.value.name == "HG_ERR_STATE"   # before step one
        hglib.hg_build_wedges(g)
        full = hglib.hg_count_patterns(g)
        full_masks = hglib.hg_mask_histogram(g)
        od = hglib.hg_out_degrees(g)
        # all owners at once: the whole count
        c_all, m_all = hglib.hg_count_owned(g, np.arange(ne))
        assert c_all.tolist() == full.tolist() and m_all.tolist() == full_masks.tolist()
        with pytest.raises(hglib.HgError) as e:
            hglib.hg_mask_histogram(g)
        assert e.value.name == "HG_ERR_STATE"   # the handle holds a part, not a count
        # two halves add up; an owner listed twice counts once; none listed, nothing
        ca, ma = hglib.hg_count_owned(g, np.arange(0, ne, 2))
        cb, mb = hglib.hg_count_owned(g, np.r_[np.arange(1, ne, 2), [1, 3]])
        assert (ca + cb).tolist() == full.tolist() and (ma + mb).tolist() == full_masks.tolist()
        c0, m0 = hglib.hg_count_owned(g, [])
        assert int(c0.sum()) == 0 and int(m0.sum()) == 0
        for bad in ([-1], [ne]):
            with pytest.raises(hglib.HgError) as e:
                hglib.hg_count_owned(g, bad)
            assert e.value.name == "HG_ERR_INVALID_ARG"
        # sampled owners one by one against the oracle
        rng = np.random.default_rng(5)
        owners = rng.choice(ne, 40, replace=False).tolist() + [int(np.argmax(od))]
        want, above = oracle.count_owned(e_ptr, e_idx, nv, owners)
        assert od[owners].tolist() == above.tolist()
        for k, u in enumerate(owners):
            c, m = hglib.hg_count_owned(g, [u])
            assert m.tolist() == want[k].tolist(), u
            assert int(c[0]) == int(want[k].sum())
        # the full count is still available afterwards
        assert hglib.hg_count_patterns(g).tolist() == full.tolist()
    finally:
        hglib.hg_free(g)
    assert full.tolist() == gold["counts"]


def test_tag_heavy_full_size_sampled_owners(hglib):
    """The tag-shaped configuration at full size (|E| = 2,000,000, top hyperedges through
    the tensor-core tiles): two sampled owners of every team shape it has (every block,
    global-table and cluster shape; its out-degrees are too large for one-warp teams), each
    histogram and out-degree equal to the oracle's, and each run in the team shape it was
    sampled for."""
    import hgen
    import oracle

    spec = hgen.TAG_HEAVY
    e_ptr, e_idx = hgen.generate(spec)
    nv, ne = spec.num_vertices, len(e_ptr) - 1
    size = np.diff(e_ptr)
    g, _ = loaded(hglib, nv, e_ptr, e_idx)
    try:
        st = hglib.hg_build_wedges(g)
        assert st["dense_edges"] > 0   # the tile path is part of this configuration
        od = hglib.hg_out_degrees(g)
        assert int(od.sum()) == st["W"]
        bk = np.full(ne, -1)
        bk[(od >= 2) & (size <= WARP_MASK_BITS) & (od <= 64)] = 0
        bk[(od > 64) & (size <= WARP_MASK_BITS) & (od <= 128)] = 1
        bk[(od > 128) & (size <= WARP_MASK_BITS) & (od <= 256)] = 2
        bk[(od > 256) & (size <= WARP_MASK_BITS) & (od <= 1024)] = 3
        bk[(od > 1024) & (size <= WARP_MASK_BITS) & (od <= 2048)] = 4
        bk[(od > 2048) & (size <= WARP_MASK_BITS) & (od <= BLOCK_MAX)] = 5
        bk[(od >= 2) & (size > WARP_MASK_BITS) & (od <= WIDE_LARGE_MIN)] = 6
        bk[(od > WIDE_LARGE_MIN) & ((size > WARP_MASK_BITS) | (od > BLOCK_MAX))] = 7
        rng = np.random.default_rng(11)
        owners, want_bucket = [], []
        for k in range(8):
            pool = np.flatnonzero(bk == k)
            if k < 3 and len(pool) == 0:
                continue   # dense: no out-degree is small enough for a one-warp team
            if k == 7:   # the cheapest of the large teams for the oracle
                pool = pool[np.argsort(od[pool], kind="stable")][:50]
            assert len(pool) >= 2, BUCKET_NAMES[k]
            for u in rng.choice(pool, 2, replace=False).tolist():
                assert bucket_of(int(od[u]), int(size[u])) == k
                owners.append(u)
                want_bucket.append(k)
        got = []
        for u, k in zip(owners, want_bucket):
            c, m = hglib.hg_count_owned(g, [u])
            teams = hglib.hg_close_stats_get(g)["bucket_teams"]
            # a warp or block team whose cuckoo stash overflows is handed to the wide teams
            assert [i for i, t in enumerate(teams) if t] in ([k], [k, 6]), (u, BUCKET_NAMES[k], teams)
            got.append(m)
    finally:
        hglib.hg_free(g)
    want, above = oracle.count_owned(e_ptr, e_idx, nv, owners)
    assert od[owners].tolist() == above.tolist()
    for k, u in enumerate(owners):
        assert got[k].tolist() == want[k].tolist(), (u, BUCKET_NAMES[want_bucket[k]])
    assert all(int(w.sum()) > 0 for w in want)   # every sampled owner closes triangles


def test_hub_large_teams_sampled_owners_repeated(hglib):
    """A hub vertex in 9,000 hyperedges: every pair of them intersects, so the out-degrees
    run from 0 to 8,999 and both the largest shared-table block teams (out-degree 4,097 to
    6,144) and the cluster-capable teams beyond run.  Sampled owners of each, three times
    over, against the oracle's per-owner histograms (a schedule-dependent miscount would
    show as a run that differs)."""
    import hgen
    import oracle

    nv, e_ptr, e_idx = hgen.hub(9000, 300, 4)
    ne = len(e_ptr) - 1
    size = np.diff(e_ptr)
    g, _ = loaded(hglib, nv, e_ptr, e_idx)
    try:
        hglib.hg_build_wedges(g)
        od = hglib.hg_out_degrees(g)
        rng = np.random.default_rng(21)
        owners, shape = [], []
        for k, lo, hi in ((5, 4097, BLOCK_MAX), (7, BLOCK_MAX + 1, 1 << 30)):
            pool = np.flatnonzero((od >= lo) & (od <= hi))
            assert len(pool) >= 3, BUCKET_NAMES[k]
            for u in rng.choice(pool, 3, replace=False).tolist():
                assert bucket_of(int(od[u]), int(size[u])) == k
                owners.append(u)
                shape.append(k)
        runs = []
        for _ in range(3):
            got = []
            for u, k in zip(owners, shape):
                c, m = hglib.hg_count_owned(g, [u])
                teams = hglib.hg_close_stats_get(g)["bucket_teams"]
                assert [i for i, t in enumerate(teams) if t] in ([k], [k, 6]), (u, teams)
                got.append(m.tolist())
            runs.append(got)
    finally:
        hglib.hg_free(g)
    want, above = oracle.count_owned(e_ptr, e_idx, nv, owners)
    assert od[owners].tolist() == above.tolist()
    for got in runs:
        assert got == want.tolist()


@pytest.mark.parametrize("close_mode", [1, 2])
def test_hub_large_teams_other_team_modes(hglib, close_mode):
    """The same owners under the other team modes: every team on the global-table blocks
    (1), or the shared-table teams building their tables and then handing every owner over
    to them (2); each owner's histogram equal to the oracle's."""
    import hgen
    import oracle

    nv, e_ptr, e_idx = hgen.hub(9000, 300, 4)
    g, _ = loaded(hglib, nv, e_ptr, e_idx)
    try:
        hglib.hg_build_wedges(g, close_mode=close_mode)
        od = hglib.hg_out_degrees(g)
        rng = np.random.default_rng(22)
        owners = []
        for lo, hi in ((4097, BLOCK_MAX), (BLOCK_MAX + 1, 1 << 30)):
            owners += rng.choice(np.flatnonzero((od >= lo) & (od <= hi)), 2, replace=False).tolist()
        got = [hglib.hg_count_owned(g, [u])[1].tolist() for u in owners]
    finally:
        hglib.hg_free(g)
    want, _ = oracle.count_owned(e_ptr, e_idx, nv, owners)
    assert got == want.tolist()


def test_unpacked_layout_large_teams_sampled_owners(hglib):
    """A hyperedge of 300 vertices forces the unpacked row layout (8-byte entries), whose
    shared-table block teams stop at out-degree 4,096 (24 warps); here it is an isolated
    hyperedge beside a 6,000-spoke hub, so the hub's teams keep their out-degrees.  Sampled
    owners of the unpacked block shapes and of the cluster-capable teams beyond 4,096,
    against the oracle's per-owner histograms."""
    import hgen
    import oracle

    nv0, p0, i0 = hgen.hub(6000, 200, 5)
    e_ptr = np.concatenate([p0, [p0[-1] + 300]]).astype(np.int64)
    e_idx = np.concatenate([i0, np.arange(nv0, nv0 + 300)]).astype(np.int32)
    nv = nv0 + 300
    size = np.diff(e_ptr)
    g, _ = loaded(hglib, nv, e_ptr, e_idx)
    try:
        hglib.hg_build_wedges(g)
        od = hglib.hg_out_degrees(g)
        rng = np.random.default_rng(23)
        owners, shape = [], []
        for k, lo, hi in ((3, 257, 1024), (4, 1025, 2048), (5, 2049, 4096), (7, 4097, 1 << 30)):
            pool = np.flatnonzero((od >= lo) & (od <= hi) & (size <= WARP_MASK_BITS))
            assert len(pool) >= 2, BUCKET_NAMES[k]
            for u in rng.choice(pool, 2, replace=False).tolist():
                owners.append(u)
                shape.append(k)
        got = []
        for u, k in zip(owners, shape):
            c, m = hglib.hg_count_owned(g, [u])
            teams = hglib.hg_close_stats_get(g)["bucket_teams"]
            assert [i for i, t in enumerate(teams) if t] in ([k], [k, 6]), (u, k, teams)
            got.append(m.tolist())
    finally:
        hglib.hg_free(g)
    want, above = oracle.count_owned(e_ptr, e_idx, nv, owners)
    assert od[owners].tolist() == above.tolist()
    assert got == want.tolist()
