"""Pins of the oracle's hyperwedge-sampling estimator (Algorithm 6, Appro-bs).  CPU only.

The draws come from Philox4x32-10 counters (the sample number is the counter), so a
sample's wedge does not depend on which range it is drawn in; when the draws are
replaced by every wedge once the estimate must equal the exact count; and over many
seeds the estimate is unbiased (Lemma 4.1)."""
import numpy as np
import pytest


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
