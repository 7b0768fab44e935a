"""Seeded input generators: determinism and the structure the workloads need
(time order, no self-loops where promised, power-law skew, bursts, the
clique-reduction construction of Theorem 3.1)."""
import numpy as np

from paper_1810_00980_gb300 import synth


def test_uniform_graph_is_seeded_and_sorted():
    a = synth.uniform_graph(1000, 20_000, 1_000_000, 1)
    b = synth.uniform_1k_graph(1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    src, dst, t = a
    assert src.dtype == np.int32 and dst.dtype == np.int32 and t.dtype == np.int64
    assert np.all(np.diff(t) >= 0) and np.all(src != dst)
    assert src.min() >= 0 and max(src.max(), dst.max()) < 1000 and t.max() < 1_000_000


def test_chung_lu_hawkes_structure():
    src, dst, t = synth.chung_lu_hawkes(5000, 200_000, 2.1, seed=9, horizon=10_000_000)
    assert len(t) == 200_000 and np.all(np.diff(t) >= 0) and np.all(src != dst)
    assert t.min() >= 0 and t.max() < 10_000_000
    deg = np.bincount(src, minlength=5000)
    # heavy tail: the top node has far more than the mean out-degree
    assert deg.max() > 50 * deg.mean()
    # self-excitation: counts per 10-minute bin are overdispersed (a Poisson
    # process has variance / mean = 1)
    c = np.bincount(t // 600)
    assert c.var() / c.mean() > 1.5
    # replies (b -> a right after a -> b) are common
    again = synth.chung_lu_hawkes(5000, 200_000, 2.1, seed=9, horizon=10_000_000)
    assert all(np.array_equal(x, y) for x, y in zip((src, dst, t), again))


def test_hub_bursts_and_degree_cap():
    src, dst, t = synth.chung_lu_hawkes(3000, 100_000, 1.8, seed=4, horizon=5_000_000,
                                        max_degree=20_000, hub_bursts=4, burst_max=3000)
    assert len(t) == 100_000 and np.all(np.diff(t) >= 0)
    # a burst puts >= 1500 edges of one source inside 60 s
    best = 0
    for h in np.argsort(-np.bincount(src))[:4]:
        th = np.sort(t[src == h])
        j = np.searchsorted(th, th + 60, side="right")
        best = max(best, int((j - np.arange(len(th))).max()))
    assert best >= 1500


def test_clique_reduction_construction():
    src, dst, t, ms, md, delta = synth.clique_reduction(4, [(1, 2), (2, 3), (1, 3)], 3)
    assert len(t) == 2 * 3 + 2 * 4 and np.all(np.diff(t) > 0)    # block timestamps are distinct
    assert len(ms) == 3 * 4 and delta >= t.max() - t.min()
    assert set(src[dst == 0].tolist()) == {1, 2, 3, 4} and set(src[dst != 0].tolist()) == {0}
