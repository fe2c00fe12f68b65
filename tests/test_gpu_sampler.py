"""CUDA hyperwedge sampler (Algorithm 6, Appro-bs) vs the oracle's, through the C ABI.

Both sides draw sample n from the same Philox4x32-10 counter, so for one seed and
sample range they visit the same hyperwedges: raw counts must agree bit-exactly and
the estimates, formed by the same IEEE double expression, exactly too."""
import numpy as np
import pytest

from conftest import csr_of, load_json

pytestmark = pytest.mark.gpu


def gpu_sample(hg, nv, e_ptr, e_idx, runs, **build):
    import torch

    stream = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    try:
        st = hg.hg_build_wedges(g, **build)
        out = [hg.hg_sample_estimate(g, seed, first, num) for seed, first, num in runs]
    finally:
        hg.hg_free(g)
    return st, out


def check(hg, nv, e_ptr, e_idx, runs, **build):
    import oracle

    st, out = gpu_sample(hg, nv, e_ptr, e_idx, runs, **build)
    for (seed, first, num), (raw, est) in zip(runs, out):
        ref = oracle.sample_estimate(e_ptr, e_idx, nv, seed=seed, first=first, num=num)
        assert st["W"] == ref.W
        assert raw.tolist() == ref.raw.tolist(), (seed, first, num)
        assert est.tolist() == ref.est.tolist(), (seed, first, num)
    return st, out


def workload(name):
    import hgen

    gold = load_json("workloads.json")[name]
    e_ptr, e_idx = hgen.generate(hgen.WORKLOADS[gold["workload"]])
    if gold["prefix_edges"] is not None:
        e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, gold["prefix_edges"])
    assert hgen.csr_hash(e_ptr, e_idx) == gold["csr_hash"]
    return gold, e_ptr, e_idx


def test_tiny_plain_prefix(hglib):
    import hgen

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 300)
    runs = [(99, 1000, 3000), (99, 0, 1), (7, 2**33 - 5, 4000), (2**64 - 1, 0, 2500)]
    st, out = check(hglib, 1000, e_ptr, e_idx, runs)
    assert out[0][0][0] > 0


def test_split_ranges_sum_to_the_whole(hglib):
    import hgen

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 600)
    _, out = gpu_sample(hglib, 1000, e_ptr, e_idx,
                        [(5, 100, 9000), (5, 100, 4000), (5, 4100, 5000)])
    assert (out[1][0] + out[2][0]).tolist() == out[0][0].tolist()


@pytest.mark.parametrize("name", ["tiny_plain", "coauthor_prefix50k", "tag_heavy_prefix2000"])
def test_workloads(hglib, name):
    gold, e_ptr, e_idx = workload(name)
    check(hglib, gold["num_vertices"], e_ptr, e_idx, [(2024, 0, 200_000), (31, 10**12, 50_000)])


def test_unpacked_entries(hglib):
    # hyperedges of 256+ vertices: omega does not fit 8 bits, rows use two int32 arrays
    import hgen

    spec = hgen.HypergraphSpec(3000, 300, 4, hgen.SIZE_UNIFORM, 200, 300, zipf_s=0.6, name="big")
    e_ptr, e_idx = hgen.generate(spec)
    check(hglib, spec.num_vertices, e_ptr, e_idx, [(3, 0, 20_000)])


def test_heavy_rows_and_dense_tiles(hglib):
    # hub rows through the global-scratch hyperwedge kernel; then all-heavy tensor-core omega
    rng = np.random.default_rng(3)
    edges = [[0, 1 + 2 * k, 2 + 2 * k] if k % 3 else [0, 1 + 2 * k] for k in range(6000)]
    for _ in range(200):
        a, b = rng.choice(12000, 2, replace=False) + 1
        edges.append([int(a), int(b)])
    e_ptr, e_idx = csr_of(sorted({tuple(sorted(set(e))) for e in edges}))
    check(hglib, 13000, e_ptr, e_idx, [(11, 0, 30_000)])

    import hgen

    spec = hgen.HypergraphSpec(4000, 400, 1, hgen.SIZE_UNIFORM, 40, 100, zipf_s=0.6, name="big")
    e_ptr, e_idx = hgen.generate(spec)
    st, _ = check(hglib, spec.num_vertices, e_ptr, e_idx, [(12, 0, 20_000)], dense_min_size=40,
                  dense_max_count=1000)
    assert st["dense_edges"] == 400


def test_degenerate_calls(hglib):
    import hgen

    # no hyperwedge at all: every estimate is zero
    e_ptr, e_idx = csr_of([[0, 1], [2, 3], [4]])
    _, out = gpu_sample(hglib, 5, e_ptr, e_idx, [(1, 0, 1000)])
    assert out[0][0].tolist() == [0] * 21 and out[0][1].tolist() == [0.0] * 21
    # zero samples
    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 200)
    _, out = gpu_sample(hglib, 1000, e_ptr, e_idx, [(1, 0, 0)])
    assert out[0][0].tolist() == [0] * 21 and out[0][1].tolist() == [0.0] * 21


def test_argument_and_state_errors(hglib):
    import hgen
    import torch

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 200)
    stream = torch.cuda.Stream()
    g = hglib.hg_load_csr(1000, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    try:
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_sample_estimate(g, 1, 0, 10)
        assert ei.value.name == "HG_ERR_STATE"
        hglib.hg_build_wedges(g)
        for sigma in (0.0, 1.5, -0.5):
            with pytest.raises(hglib.HgError) as ei:
                hglib.hg_sample_estimate(g, 1, 0, 10, sigma=sigma)
            assert ei.value.name == "HG_ERR_INVALID_ARG"
            with pytest.raises(hglib.HgError) as ei:
                hglib.hg_sample_estimate_adv(g, 1, 0, 10, sigma=sigma)
            assert ei.value.name == "HG_ERR_INVALID_ARG"
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_sample_estimate_adv(g, 1, 0, 10, class_mask=16)
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        with pytest.raises(hglib.HgError) as ei:
            hglib.hg_sample_estimate(g, 1, 2**64 - 5, 10)
        assert ei.value.name == "HG_ERR_INVALID_ARG"
        # the handle still works after rejected calls, and after a rebuild
        raw, _ = hglib.hg_sample_estimate(g, 1, 0, 500)
        hglib.hg_build_wedges(g)
        raw2, _ = hglib.hg_sample_estimate(g, 1, 0, 500)
        assert raw.tolist() == raw2.tolist()
    finally:
        hglib.hg_free(g)


# ------------------------------------------------------------------ Appro-adv and sigma < 1

def gpu_adv(hg, nv, e_ptr, e_idx, runs, **build):
    import torch

    stream = torch.cuda.Stream()
    g = hg.hg_load_csr(nv, len(e_ptr) - 1, e_ptr, e_idx, stream=stream.cuda_stream)
    try:
        hg.hg_build_wedges(g, **build)
        out = []
        for r in runs:
            if r[0] == "bs":
                _, seed, first, num, sigma = r
                out.append(hg.hg_sample_estimate(g, seed, first, num, sigma=sigma))
            else:
                _, seed, first, num, sigma, mask = r
                out.append(hg.hg_sample_estimate_adv(g, seed, first, num, sigma=sigma,
                                                     class_mask=mask))
    finally:
        hg.hg_free(g)
    return out


def check_adv(hg, nv, e_ptr, e_idx, runs, **build):
    import oracle

    out = gpu_adv(hg, nv, e_ptr, e_idx, runs, **build)
    for r, got in zip(runs, out):
        if r[0] == "bs":
            _, seed, first, num, sigma = r
            ref = oracle.sample_estimate(e_ptr, e_idx, nv, seed=seed, first=first, num=num,
                                         sigma=sigma)
            assert got[0].tolist() == ref.raw.tolist(), r
            assert got[1].tolist() == ref.est.tolist(), r
        else:
            _, seed, first, num, sigma, mask = r
            ref = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=seed, first=first, num=num,
                                             sigma=sigma, class_mask=mask)
            raw, est, info = got
            assert raw.tolist() == ref.raw.tolist(), r
            assert est.tolist() == ref.est.tolist(), r
            assert (info["W"], info["W_t"], info["W_c"], info["edges"]) == \
                (ref.W, ref.W_t, ref.W_c, ref.edges), r
            assert (info["alpha_1"], info["alpha_2"], info["alpha_3"], info["alpha_4"]) == ref.alphas
    return out


def test_adv_tiny_plain(hglib):
    import hgen

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 300)
    runs = [("adv", 9, 0, 30_000, 1.0, 15), ("adv", 9, 0, 30_000, 1.0, 8),
            ("adv", 9, 0, 30_000, 1.0, 1 | 2 | 4), ("adv", 2**64 - 3, 2**36, 5_000, 1.0, 15),
            ("adv", 4, 0, 1, 1.0, 15)]
    out = check_adv(hglib, 1000, e_ptr, e_idx, runs)
    assert out[0][0][0] > 0


@pytest.mark.parametrize("name", ["tiny_plain", "coauthor_prefix50k", "tag_heavy_prefix2000"])
def test_adv_workloads(hglib, name):
    gold, e_ptr, e_idx = workload(name)
    check_adv(hglib, gold["num_vertices"], e_ptr, e_idx,
              [("adv", 2024, 0, 100_000, 1.0, 15), ("adv", 3, 10**9, 20_000, 1.0, 2 | 4)])


def test_adv_unpacked_and_dense_tiles(hglib):
    import hgen

    spec = hgen.HypergraphSpec(3000, 300, 4, hgen.SIZE_UNIFORM, 200, 300, zipf_s=0.6, name="big")
    e_ptr, e_idx = hgen.generate(spec)
    check_adv(hglib, spec.num_vertices, e_ptr, e_idx, [("adv", 3, 0, 10_000, 1.0, 15)])
    spec = hgen.HypergraphSpec(4000, 400, 1, hgen.SIZE_UNIFORM, 40, 100, zipf_s=0.6, name="big")
    e_ptr, e_idx = hgen.generate(spec)
    check_adv(hglib, spec.num_vertices, e_ptr, e_idx, [("adv", 12, 0, 10_000, 1.0, 15)],
              dense_min_size=40, dense_max_count=1000)


@pytest.mark.parametrize("sigma", [0.5, 0.3, 0.05])
def test_sigma_sub_hypergraph(hglib, sigma):
    # Algorithms 6 and 7 on G' (the ceil(sigma |E|) smallest Philox priorities)
    import hgen

    e_ptr, e_idx = hgen.prefix(*hgen.generate(hgen.TINY_PLAIN), 1500)
    runs = [("bs", 31, 0, 40_000, sigma), ("adv", 31, 0, 40_000, sigma, 15),
            ("bs", 32, 7, 40_000, sigma), ("bs", 31, 7, 10_000, 1.0), ("adv", 32, 0, 20_000, sigma, 8)]
    check_adv(hglib, 1000, e_ptr, e_idx, runs)


def test_sigma_on_coauthor_prefix(hglib):
    gold, e_ptr, e_idx = workload("coauthor_prefix50k")
    check_adv(hglib, gold["num_vertices"], e_ptr, e_idx,
              [("bs", 5, 0, 200_000, 0.4), ("adv", 5, 0, 200_000, 0.4, 15)])
