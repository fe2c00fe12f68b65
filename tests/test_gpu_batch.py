"""Batches of hypergraphs counted in shared launches vs each member alone and vs the
oracle, through the C ABI.  Per-member counts and wedge statistics: bit-exact."""
import numpy as np
import pytest

from conftest import csr_of, load_json

pytestmark = pytest.mark.gpu


def random_members(seed, n):
    import hgen

    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nv = int(rng.integers(5, 300))
        spec = hgen.HypergraphSpec(
            num_vertices=nv, num_edges=int(rng.integers(1, 500)), seed=1000 * seed + k,
            size_dist=hgen.SIZE_UNIFORM, size_lo=1, size_hi=int(rng.integers(2, 12)),
            zipf_s=float(rng.uniform(0.5, 1.5)), name="member")
        try:
            e_ptr, e_idx = hgen.generate(spec)
        except RuntimeError:
            continue
        out.append((nv, e_ptr, e_idx))
    # degenerate members: no hyperedge, one hyperedge, no hyperwedge
    out.insert(3, (4, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32)))
    out.insert(7, (3, *csr_of([[0, 1, 2]])))
    out.append((6, *csr_of([[0, 1], [2, 3], [4, 5]])))
    return out


def run_batch(hg, members, max_wave_edges=0, device=False, **build):
    import torch

    nv, eoff, eptr, evtx = hg.concat_members(members)
    if device:
        eptr, evtx = torch.from_numpy(eptr).cuda(), torch.from_numpy(evtx).cuda()
    stream = torch.cuda.Stream()
    b = hg.hg_load_batch(nv, eoff, eptr, evtx, max_wave_edges=max_wave_edges,
                         stream=stream.cuda_stream)
    try:
        hg.hg_batch_build_wedges(b, **build)
        counts, stats = hg.hg_batch_count_patterns(b)
        cc, open_, conn = hg.hg_batch_clustering_coeff(b, [1.0] * 20)
        waves = hg.hg_batch_waves(b)
        masks = hg.hg_batch_mask_histogram(b)
    finally:
        hg.hg_batch_free(b)
    return counts, stats, cc, open_, conn, waves, masks


def stored_masks(entry):
    out = [0] * 128
    for m, n in entry["masks"].items():
        out[int(m)] = n
    return out


def check_members(members, counts, stats, open_, stored=None, masks=None):
    # stored: member index -> stored oracle entry (tests/golden/workloads.json); masks:
    # the batch's canonical region-mask histograms, compared before the counts
    import oracle

    for m, (nv, e_ptr, e_idx) in enumerate(members):
        if stored and m in stored:
            ref = stored[m]
            want_masks = stored_masks(ref)
            want = (ref["counts"], ref["W"], ref["W_c"], ref["W_t"], ref["max_deg"],
                    ref["connected"], ref["open"])
        else:
            r = oracle.count(e_ptr, e_idx, nv)
            want_masks = r.masks.tolist()
            want = ([int(x) for x in r.counts], r.W, r.W_c, r.W_t, r.max_deg, r.connected, r.open)
        if masks is not None:
            assert masks[m].tolist() == want_masks, m
        got = (counts[m].tolist(), int(stats["W"][m]), int(stats["W_c"][m]), int(stats["W_t"][m]),
               int(stats["max_deg"][m]), int(stats["connected"][m]), int(open_[m]))
        assert got == want, m


@pytest.mark.parametrize("seed", [1, 2])
def test_random_members_match_oracle(hglib, seed):
    members = random_members(seed, 60)
    counts, stats, cc, open_, conn, waves, masks = run_batch(hglib, members)
    assert len(waves) == 1 and waves[0][2] == len(members)
    check_members(members, counts, stats, open_, masks=masks)


def test_waves_and_device_inputs_give_the_same_results(hglib):
    members = random_members(3, 80)
    one = run_batch(hglib, members)
    many = run_batch(hglib, members, max_wave_edges=700)
    dev = run_batch(hglib, members, max_wave_edges=2000, device=True)
    assert len(many[5]) > 5 and len(dev[5]) > 1
    assert sum(w[2] for w in many[5]) == len(members)
    for other in (many, dev):
        assert other[0].tolist() == one[0].tolist()
        for k in one[1]:
            assert other[1][k].tolist() == one[1][k].tolist(), k
        assert other[3].tolist() == one[3].tolist()
        assert other[6].tolist() == one[6].tolist()
        np.testing.assert_array_equal(other[2], one[2])


def test_batched_workload_members_match_single_handles(hglib):
    # the first members of the 4,096-hypergraph batch (seeds 100..), each also alone
    import hgen
    import torch

    members = []
    for seed in range(100, 164):
        spec = hgen.batched(seed)
        members.append((spec.num_vertices, *hgen.generate(spec)))
    counts, stats, cc, open_, conn, waves, masks = run_batch(hglib, members)
    stream = torch.cuda.Stream()
    for m, (nv, e_ptr, e_idx) in enumerate(members):
        g = hglib.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
        try:
            st = hglib.hg_build_wedges(g)
            alone = hglib.hg_count_patterns(g)
            alone_masks = hglib.hg_mask_histogram(g)
            cc1, op1, co1 = hglib.hg_clustering_coeff(g, [1.0] * 20)
        finally:
            hglib.hg_free(g)
        assert masks[m].tolist() == alone_masks.tolist(), m
        assert counts[m].tolist() == alone.tolist(), m
        assert int(stats["W"][m]) == st["W"] and int(stats["W_c"][m]) == st["W_c"], m
        assert int(open_[m]) == op1 and int(conn[m]) == co1, m
        assert (np.isnan(cc[m]) and np.isnan(cc1)) or cc[m] == cc1, m
    small = [k for k, m in enumerate(members) if len(m[1]) - 1 <= 3000][:12]
    check_members([members[k] for k in small], counts[small], {k: v[small] for k, v in stats.items()},
                  open_[small], masks=masks[small])


def test_every_team_shape_flushes_per_member(hglib):
    # members with out-degrees for block teams with shared tables, a hub member
    # for the wide teams, and small ones between them; then all through wide teams
    import hgen

    spec = hgen.HypergraphSpec(40, 3000, 21, hgen.SIZE_UNIFORM, 3, 5, zipf_s=0.4, name="dense_small")
    members = random_members(4, 20)
    members.insert(5, (40, *hgen.generate(spec)))
    gold = load_json("workloads.json")["hub3000"]   # 4.5e9 hyper-triangles: stored
    hub = hgen.hub(*gold["hub"])
    assert hgen.csr_hash(hub[1], hub[2]) == gold["csr_hash"]
    members.insert(12, hub)
    members.insert(15, (400, *hgen.generate(
        hgen.HypergraphSpec(400, 300, 7, hgen.SIZE_UNIFORM, 20, 90, zipf_s=0.3, name="wide"))))
    base = run_batch(hglib, members)
    check_members(members, base[0], base[1], base[3], stored={12: gold}, masks=base[6])
    wide = run_batch(hglib, members, close_mode=1)
    assert wide[6].tolist() == base[6].tolist()
    assert wide[0].tolist() == base[0].tolist()


def test_member_range_and_state_errors(hglib):
    import torch

    members = [(3, *csr_of([[0, 1], [1, 2]])), (2, *csr_of([[0, 2]]))]   # id 2 >= |V_1| = 2
    nv, eoff, eptr, evtx = hglib.concat_members(members)
    with pytest.raises(hglib.HgError) as ei:
        hglib.hg_load_batch(nv, eoff, eptr, evtx)
    assert ei.value.name == "HG_ERR_VERTEX_RANGE"
    members[1] = (3, *csr_of([[0, 2]]))
    nv, eoff, eptr, evtx = hglib.concat_members(members)
    stream = torch.cuda.Stream()
    b = hglib.hg_load_batch(nv, eoff, eptr, evtx, stream=stream.cuda_stream)
    try:
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_batch_count_patterns(b)
        assert ei.value.name == "HG_ERR_STATE"
        hglib.hg_batch_build_wedges(b)
        wave = hglib.hg_batch_waves(b)[0][0]
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_sample_estimate(wave, 1, 0, 10)
        assert ei.value.name == "HG_ERR_UNSUPPORTED"
        counts, _ = hglib.hg_batch_count_patterns(b)
        assert counts.tolist() == [[0] * 21, [0] * 21]
    finally:
        hglib.hg_batch_free(b)
