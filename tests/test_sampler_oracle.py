"""Pins of the oracle's hyperwedge-sampling estimator (Algorithm 6, Appro-bs).  CPU only.

The draws come from Philox4x32-10 counters (the sample number is the counter), so a
sample's wedge does not depend on which range it is drawn in; when the draws are
replaced by every wedge once the estimate must equal the exact count; and over many
seeds the estimate is unbiased (Lemma 4.1)."""
import numpy as np
import pytest

from conftest import load_json


@pytest.fixture(scope="module")
def small(native_cpu):
    import hgen

    e_ptr, e_idx = hgen.generate(hgen.TINY_PLAIN)
    return hgen.prefix(e_ptr, e_idx, 300) + (1000,)


def test_every_wedge_once_gives_the_exact_count(small):
    import oracle

    e_ptr, e_idx, nv = small
    exact = oracle.count(e_ptr, e_idx, nv)
    s = oracle.sample_estimate(e_ptr, e_idx, nv, seed=0, first=0, num=exact.W, identity_draws=True)
    assert s.W == exact.W
    assert s.raw.tolist() == exact.counts.tolist()
    assert s.est.tolist() == [float(x) for x in exact.counts]


def test_counter_based_draws_split_over_ranges(small):
    import oracle

    e_ptr, e_idx, nv = small
    whole = oracle.sample_estimate(e_ptr, e_idx, nv, seed=99, first=1000, num=3000)
    a = oracle.sample_estimate(e_ptr, e_idx, nv, seed=99, first=1000, num=1700)
    b = oracle.sample_estimate(e_ptr, e_idx, nv, seed=99, first=2700, num=1300)
    assert (a.raw + b.raw).tolist() == whole.raw.tolist()
    other = oracle.sample_estimate(e_ptr, e_idx, nv, seed=100, first=1000, num=3000)
    assert other.raw.tolist() != whole.raw.tolist()


def test_philox_known_answers():
    # the block function against the generator's published known-answer vectors
    import oracle

    for v in load_json("philox_kat.json")["vectors"]:
        got = oracle.philox4x32_10([int(x, 16) for x in v["counter"]],
                                   [int(x, 16) for x in v["key"]])
        assert [int(x) for x in got] == [int(x, 16) for x in v["out"]]


def test_draws_are_uniform_over_wedges():
    # Philox words mapped to [0, W) by a 64x64 multiply-high: chi-square over 64 cells
    import oracle

    cells = np.zeros(64, dtype=np.int64)
    for n in range(64 * 400):
        x = oracle.philox4x32_10([n & 0xFFFFFFFF, n >> 32, 0, 0], [12345, 0])
        r = (x[1] << 32) | x[0]
        cells[(r * 64) >> 64] += 1
    chi2 = float(((cells - 400) ** 2 / 400).sum())
    assert chi2 < 120   # 63 degrees of freedom; the 0.9999 quantile is about 113


def test_estimate_is_unbiased(small):
    # Lemma 4.1: E[est] = H.  400 seeds x 300 samples, mean within 4 standard errors
    import oracle

    e_ptr, e_idx, nv = small
    exact = oracle.count(e_ptr, e_idx, nv)
    ests = np.array([oracle.sample_estimate(e_ptr, e_idx, nv, seed=s, first=0, num=300).est
                     for s in range(400)])
    for p in [0] + [p for p in range(1, 21) if exact.counts[p] > exact.T // 50]:
        mean, se = ests[:, p].mean(), ests[:, p].std(ddof=1) / np.sqrt(len(ests))
        assert abs(mean - float(exact.counts[p])) < 4 * se + 1e-9, p


def test_block_function_avalanche():
    # flipping any one of the 128 counter bits changes about half of the 128 output
    # bits (a dropped round or a wrong word order would leave many bits unchanged)
    import oracle

    rng = np.random.default_rng(7)
    flips = []
    for _ in range(24):
        c = [int(x) for x in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        k = [int(x) for x in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        y0 = oracle.philox4x32_10(c, k)
        for bit in range(128):
            c2 = list(c)
            c2[bit // 32] ^= 1 << (bit % 32)
            y1 = oracle.philox4x32_10(c2, k)
            flips.append(sum(bin(a ^ b).count("1") for a, b in zip(y0, y1)))
    flips = np.array(flips)
    assert abs(flips.mean() - 64.0) < 1.0 and flips.min() >= 30


# ------------------------------------------------------------------ Appro-adv (Algorithm 7)

CLASS_OF = {1: "CCC", **{p: "TCC" for p in range(2, 6)}, **{p: "TTC" for p in range(6, 9)},
            **{p: "TTT" for p in range(9, 21)}}


def test_adv_every_wedge_once_gives_the_exact_class_counts(small):
    # every hyperwedge of each type drawn once: each triangle of a class is counted by
    # exactly one of its hyperwedges of the drawn type, so the estimate is the count
    import oracle

    e_ptr, e_idx, nv = small
    exact = oracle.count(e_ptr, e_idx, nv)
    a = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=0, first=0, num=1, identity_draws=True)
    assert (a.W, a.W_t, a.W_c) == (exact.W, exact.W_t, exact.W_c)
    assert a.alphas == (exact.W_t, exact.W_c, exact.W_t, exact.W_c)
    assert a.raw.tolist() == exact.counts.tolist()
    assert a.est.tolist() == [float(x) for x in exact.counts]
    # one class at a time: that class's counts, zeros elsewhere
    for cls, bit in oracle.CLASS_BITS.items():
        b = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=0, first=0, num=1, class_mask=bit,
                                       identity_draws=True)
        want = [int(exact.counts[p]) if CLASS_OF[p] == cls else 0 for p in range(1, 21)]
        assert b.raw[1:].tolist() == want, cls


def test_adv_sample_split_and_targeted_classes(small):
    import oracle

    e_ptr, e_idx, nv = small
    full = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=5, first=100, num=20_000)
    W, Wt, Wc = full.W, full.W_t, full.W_c
    a1, a2, a3, a4 = full.alphas
    assert a3 == a4 and a1 * W * W <= Wt * Wt * 20_000 < (a1 + 1) * W * W
    assert a2 * W * W <= Wc * Wc * 20_000 < (a2 + 1) * W * W
    assert 20_000 - 4 <= a1 + a2 + a3 + a4 <= 20_000   # (W_t + W_c)^2 = W^2
    for cls, bit in oracle.CLASS_BITS.items():
        one = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=5, first=100, num=20_000,
                                         class_mask=bit)
        for p in range(1, 21):
            want = full.est[p] if CLASS_OF[p] == cls else 0.0
            assert one.est[p] == want, (cls, p)


def test_adv_estimate_is_unbiased(small):
    import oracle

    e_ptr, e_idx, nv = small
    exact = oracle.count(e_ptr, e_idx, nv)
    ests = np.array([oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=s, first=0, num=400).est
                     for s in range(300)])
    for p in [0] + [p for p in range(1, 21) if exact.counts[p] > exact.T // 50]:
        mean, se = ests[:, p].mean(), ests[:, p].std(ddof=1) / np.sqrt(len(ests))
        assert abs(mean - float(exact.counts[p])) < 4 * se + 1e-9, p


# ------------------------------------------------------------------ sigma < 1 (the sigma|E| draw)

def test_subgraph_selection(small):
    import math

    import oracle

    e_ptr, e_idx, nv = small
    ne = len(e_ptr) - 1
    assert oracle.subgraph(ne, 3, 1.0).tolist() == list(range(ne))
    seen = np.zeros(ne)
    for seed in range(400):
        k = oracle.subgraph(ne, seed, 0.3)
        assert len(k) == math.ceil(0.3 * ne) and np.all(np.diff(k) > 0)
        seen[k] += 1
    assert oracle.subgraph(ne, 1, 0.3).tolist() != oracle.subgraph(ne, 2, 0.3).tolist()
    # each hyperedge kept with probability ceil(0.3 |E|) / |E|: binomial(400, q) per edge
    q = math.ceil(0.3 * ne) / ne
    z = (seen - 400 * q) / math.sqrt(400 * q * (1 - q))
    assert abs(z.mean()) < 0.3 and np.abs(z).max() < 5.0


def test_sigma_estimates_run_on_the_sub_hypergraph(small):
    # every hyperwedge of G' once: raw = the exact counts of the explicitly built G',
    # est = raw / sigma^3 (Algorithms 6 and 7: the sigma|E| draw and the final scaling)
    import oracle

    e_ptr, e_idx, nv = small
    sigma = 0.5
    kept = oracle.subgraph(len(e_ptr) - 1, 77, sigma)
    rows = [e_idx[e_ptr[i]:e_ptr[i + 1]] for i in kept]
    sp = np.zeros(len(rows) + 1, dtype=np.int64)
    sp[1:] = np.cumsum([len(r) for r in rows])
    si = np.concatenate(rows).astype(np.int32)
    sub = oracle.count(sp, si, nv)
    bs = oracle.sample_estimate(e_ptr, e_idx, nv, seed=77, first=0, num=sub.W, sigma=sigma,
                                identity_draws=True)
    assert bs.W == sub.W and bs.raw.tolist() == sub.counts.tolist()
    assert bs.est.tolist() == [float(x) / sigma ** 3 for x in sub.counts]
    adv = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=77, first=0, num=1, sigma=sigma,
                                     identity_draws=True)
    assert adv.edges == len(kept) and adv.raw.tolist() == sub.counts.tolist()
