"""The seeded generator: determinism, shape, and its elementary functions."""
import math

import numpy as np
import pytest

from conftest import load_json


@pytest.fixture(scope="module")
def gen(native_cpu):
    import hgen

    return hgen


def test_tiny_plain_hash_is_stable(gen):
    # the stored hash was written on another machine: byte-identical output across
    # x86-64 and AArch64 is what lets stored oracle values be reused
    gold = load_json("workloads.json")["tiny_plain"]
    e_ptr, e_idx = gen.generate(gen.TINY_PLAIN)
    assert gen.csr_hash(e_ptr, e_idx) == gold["csr_hash"]


def test_csr_is_valid(gen):
    e_ptr, e_idx = gen.generate(gen.TINY_PLAIN)
    sizes = np.diff(e_ptr)
    assert sizes.min() >= 2 and sizes.max() <= 6 and len(sizes) == 2000
    rows = {tuple(e_idx[e_ptr[i]:e_ptr[i + 1]]) for i in range(2000)}
    assert len(rows) == 2000                       # no duplicate hyperedges
    for i in range(2000):
        r = e_idx[e_ptr[i]:e_ptr[i + 1]]
        assert np.all(np.diff(r) > 0) and r.min() >= 0 and r.max() < 1000


def test_degree_cap(gen):
    spec = gen.HypergraphSpec(2000, 20000, 3, gen.SIZE_POWERLAW, 2, 25, size_p1=2.5, zipf_s=1.0,
                              degree_cap=50)
    e_ptr, e_idx = gen.generate(spec)
    assert np.bincount(e_idx).max() == 50


def test_popularity_is_zipf_like(gen):
    spec = gen.HypergraphSpec(5000, 4000, 4, gen.SIZE_UNIFORM, 2, 2, zipf_s=1.0)
    _, e_idx = gen.generate(spec)
    deg = np.bincount(e_idx, minlength=5000)
    # Zipf(1): popularity falls like 1/rank (drawing two distinct vertices per
    # hyperedge flattens the head a little)
    assert 4 < deg[0] / deg[9] < 15 and 4 < deg[9:12].sum() / deg[99:102].sum() < 15


def test_sizes_distributions(gen):
    ln = gen.HypergraphSpec(20000, 20000, 5, gen.SIZE_LOGNORMAL, 2, 200, size_p1=1.5, size_p2=1.0,
                            zipf_s=0.5)
    e_ptr, _ = gen.generate(ln)
    s = np.diff(e_ptr)
    # median of round(exp(N(1.5, 1))) is about e^1.5 = 4.48
    assert 3.5 <= np.median(s) <= 5.5 and s.min() >= 2 and s.max() <= 200


def test_det_functions_accuracy(gen):
    lib = gen._load()
    for x in (1e-8, 0.1, 0.5, 1.0, 2.0, 3.7, 1e5, 2e6):
        assert lib.hgen_det_log(x) == pytest.approx(math.log(x), rel=1e-14, abs=1e-15)
    for x in (-20.0, -1.0, 0.0, 0.3, 1.0, 5.5, 40.0):
        assert lib.hgen_det_exp(x) == pytest.approx(math.exp(x), rel=1e-14)


def test_loguniform_sizes(gen):
    xs = [gen.loguniform_int(100 + s, 0, 100, 200_000) for s in range(400)]
    assert min(xs) >= 100 and max(xs) <= 200_000
    med = float(np.median(np.log(xs)))
    assert abs(med - (math.log(100) + math.log(200_000)) / 2) < 0.6


def test_stored_hub_values_follow_the_sunflower_closed_form():
    # hub(3000, 0, 0): 3000 hyperedges meeting pairwise in exactly {0}, each with a
    # private vertex: every triple is a hyper-triangle with regions a, b, c, g
    # non-empty (pattern 9), so H[9] = C(3000, 3), W = C(3000, 2) and no hyperwedge
    # is of inclusion type.  Pins the stored oracle entry the GPU tests compare with.
    from math import comb

    import hgen

    gold = load_json("workloads.json")["hub3000"]
    nv, e_ptr, e_idx = hgen.hub(*gold["hub"])
    assert hgen.csr_hash(e_ptr, e_idx) == gold["csr_hash"] and nv == gold["num_vertices"]
    want = [0] * 21
    want[0] = want[9] = comb(3000, 3)
    assert gold["counts"] == want
    assert (gold["W"], gold["W_c"], gold["W_t"]) == (comb(3000, 2), 0, comb(3000, 2))
    assert gold["connected"] == 3000 * comb(2999, 2) and gold["open"] == 0


def test_generate_batch_layout_and_thread_independence():
    # members drawn in threads land in the concatenated layout exactly as drawn alone,
    # whatever the thread count; a member that exhausts its fresh hyperedges is redrawn
    import hgen

    specs = [hgen.batched(s) for s in (100, 101, 962, 105)]   # seed 962 needs a redraw
    nv, eoff, eptr, evtx, used = hgen.generate_batch(specs, threads=1,
                                                     redraw=hgen.batched_redraw)
    nv4, eoff4, eptr4, evtx4, used4 = hgen.generate_batch(specs, threads=4,
                                                          redraw=hgen.batched_redraw)
    assert (eoff.tolist(), nv.tolist()) == (eoff4.tolist(), nv4.tolist())
    assert hgen.csr_hash(eptr, evtx) == hgen.csr_hash(eptr4, evtx4)
    assert [u.seed for u in used] == [100, 101, 962 + (1 << 32), 105] == [u.seed for u in used4]
    for m, sp in enumerate(used):
        p, i = hgen.generate(sp)
        lo, hi = eoff[m], eoff[m + 1]
        assert (eptr[lo:hi + 1] - eptr[lo]).tolist() == p.tolist()
        assert evtx[eptr[lo]:eptr[hi]].tolist() == i.tolist()
    with pytest.raises(hgen.DedupExhausted):
        hgen.generate(specs[2])
