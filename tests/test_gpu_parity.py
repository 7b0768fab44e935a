"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts are compared bit-exactly as int64; estimates within 1e-12 relative
(the weights are exact Q64 integer sums on the device and exactly rounded
rationals in the oracle, so both sit within a few fp64 ulps of the true
value).  Per-window weights W_j are compared against the oracle's correctly
rounded value with the same 1e-12 relative bound plus the device's documented
floor error of at most 2^-64 per instance.
"""
import math

import numpy as np
import pytest

from paper_1810_00980_gb300 import synth

pytestmark = pytest.mark.gpu

EST_RTOL = 1e-12

MOTIFS = [
    ([0], [1]),
    ([0, 1], [1, 0]),
    ([0, 0], [1, 1]),
    ([0, 1], [1, 2]),
    ([1, 0], [0, 2]),
    ([0, 2], [1, 1]),
    ([0, 1, 2], [1, 2, 0]),
    ([0, 2, 2], [1, 1, 0]),          # a->b, c->b, c->a: closes from the last edge's side too
    ([0, 1, 0], [1, 2, 2]),          # a->b, b->c, a->c
    ([0, 0, 1], [1, 2, 2]),          # a->b, a->c, b->c
    ([2, 2, 2], [0, 1, 0]),
    ([0, 2, 0], [1, 1, 1]),          # b->a, c->a, b->a: closing pair fixed, second edge into a
    ([0, 0, 1], [1, 2, 0]),          # c->a, c->b, a->c: closing pair is the reverse pair
    ([0, 1, 0], [1, 0, 1]),
    ([0, 2, 1], [1, 3, 2]),
    ([0, 1, 2, 3], [1, 2, 3, 0]),
    ([0, 0, 0, 0], [1, 2, 1, 2]),
    ([1, 0, 2, 0], [0, 2, 1, 1]),
    ([0, 1, 2, 3, 4], [1, 2, 3, 4, 0]),
    ([0, 1, 0, 1, 0, 1], [1, 0, 1, 0, 1, 0]),
    ([0, 1, 2, 3, 4, 5, 6, 0], [1, 2, 3, 4, 5, 6, 7, 7]),
]


@pytest.fixture(scope="module")
def tm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_1810_00980_gb300 import tm as _tm
    return _tm


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.core.build()
    return oracle


def _graph(tm, src, dst, t, device=True, n_nodes=-1):
    import torch
    if device and len(t):
        return tm.Graph(torch.from_numpy(np.ascontiguousarray(src)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(dst)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(t)).cuda(), n_nodes)
    return tm.Graph(src, dst, t, n_nodes)


def _close(a, b, rtol=EST_RTOL):
    return abs(a - b) <= rtol * max(abs(b), 1e-300) or (a == 0 and b == 0)


# ------------------------------------------------------------------ exact ---
def test_exact_random_tiny_graphs(tm, orc):
    """Many tiny graphs with ties, duplicates and self-loops, every motif shape."""
    rng = np.random.default_rng(2024)
    for trial in range(60):
        n = int(rng.integers(2, 7))
        m = int(rng.integers(0, 60))
        src, dst, t = synth.random_small_graph(rng, n, m, int(rng.integers(1, 80)), self_loops=trial % 4 == 0)
        g = _graph(tm, src, dst, t, device=trial % 2 == 0)
        for ms, md in MOTIFS:
            mo = tm.Motif(ms, md)
            for delta in (0, 3, 17, 1000):
                want = orc.count_exact(src, dst, t, ms, md, delta)
                assert tm.count_exact(g, mo, delta) == want, (trial, ms, md, delta)
                if trial % 5 == 0:
                    assert tm.count_exact_plain(g, mo, delta) == want


def test_exact_bruteforce_small(tm, orc):
    """Def. 2.2 by exhaustive subsets on <= 12 edges, directly against the device."""
    rng = np.random.default_rng(12)
    for trial in range(40):
        src, dst, t = synth.random_small_graph(rng, 4, int(rng.integers(0, 13)), 15, self_loops=trial % 3 == 0)
        g = _graph(tm, src, dst, t)
        for ms, md in MOTIFS[:13]:
            want, _ = orc.count_bruteforce(src, dst, t, ms, md, 9)
            assert tm.count_exact(g, tm.Motif(ms, md), 9) == want


def test_exact_mid_graph_all_config_motifs(tm, orc):
    """A bursty power-law graph spanning many matcher chunks and ragged tails."""
    src, dst, t = synth.chung_lu_hawkes(3000, 300_000, 2.1, seed=21, horizon=6_000_000)
    g = _graph(tm, src, dst, t)
    for name in ("cycle3", "outstar3", "pingpong", "cycle4", "instar3"):
        ms, md = synth.MOTIFS[name] if name in synth.MOTIFS else ([0, 2, 0], [1, 1, 1])
        mo = tm.Motif(ms, md)
        for delta in (600, 3600, 86400):
            want = orc.count_exact(src, dst, t, ms, md, delta, threads=8)
            got = tm.count_exact(g, mo, delta)
            assert got == want, (name, delta, got, want)


def test_hub_heavy_graph(tm, orc):
    """Hub bursts: thousands of edges from one node inside one delta."""
    src, dst, t = synth.chung_lu_hawkes(2000, 120_000, 1.8, seed=5, horizon=3_000_000,
                                        max_degree=40_000, hub_bursts=6, burst_max=4000)
    g = _graph(tm, src, dst, t)
    for name in ("outstar3", "cycle3", "cycle4"):
        ms, md = synth.MOTIFS[name]
        mo = tm.Motif(ms, md)
        want = orc.count_exact(src, dst, t, ms, md, 1800, threads=8)
        assert tm.count_exact(g, mo, 1800) == want
    # the subtraction path of the last level (one endpoint new, long ranges)
    for thr in (1, 1 << 20):
        tm.set_tuning(enum_threshold=thr)
        for ms, md in (([0, 0], [1, 2]), ([1, 2], [0, 0]), ([0, 1, 1], [1, 2, 3])):
            want = orc.count_exact(src, dst, t, ms, md, 600, threads=8)
            assert tm.count_exact(g, tm.Motif(ms, md), 600) == want
    tm.set_tuning(enum_threshold=48)


def test_edge_cases(tm, orc):
    tmm = tm
    cyc = tmm.Motif([0, 1, 2], [1, 2, 0])
    # empty graph
    e32 = np.zeros(0, np.int32)
    g = tmm.Graph(e32, e32, np.zeros(0, np.int64), 5)
    assert tmm.count_exact(g, cyc, 10) == 0
    assert tmm.estimate(g, cyc, 10, 3, 0.5, 1) == 0.0
    # one edge, l = 1
    g = _graph(tm, np.array([0], np.int32), np.array([1], np.int32), np.array([7], np.int64))
    assert tmm.count_exact(g, tmm.Motif([0], [1]), 0) == 1
    # all timestamps equal: nothing with l >= 2
    s = np.array([0, 1, 2, 0, 1], np.int32)
    d = np.array([1, 2, 0, 2, 0], np.int32)
    t = np.full(5, 42, np.int64)
    g = _graph(tm, s, d, t)
    assert tmm.count_exact(g, cyc, 100) == 0
    assert tmm.count_exact(g, tmm.Motif([0], [1]), 0) == 5
    # unsorted and out-of-range inputs are rejected on the host
    with pytest.raises(tmm.TmError) as ei:
        tmm.Graph(np.array([0, 1], np.int32), np.array([1, 0], np.int32), np.array([5, 4], np.int64))
    assert ei.value.status == tmm.TM_EUNSORTED
    with pytest.raises(tmm.TmError) as ei:
        tmm.Graph(np.array([0, 3], np.int32), np.array([1, 0], np.int32), np.array([4, 5], np.int64), 3)
    assert ei.value.status == tmm.TM_ERANGE
    with pytest.raises(tmm.TmError) as ei:
        tmm.Graph(np.array([0, -1], np.int32), np.array([1, 0], np.int32), np.array([4, 5], np.int64))
    assert ei.value.status == tmm.TM_ERANGE
    # bad query arguments
    g = _graph(tm, s, d, np.arange(5, dtype=np.int64))
    for args in ((10, 0, 0.5, 1), (10, 3, 0.0, 1), (10, 3, 1.5, 1), (0, 3, 0.5, 1)):
        with pytest.raises(tmm.TmError) as ei:
            tmm.estimate(g, cyc, *args)
        assert ei.value.status == tmm.TM_EINVAL
    with pytest.raises(tmm.TmError):
        tmm.count_exact(g, cyc, -1)
    # negative and huge timestamps: normalisation t - t_min
    t2 = np.array([-(1 << 40), -(1 << 40) + 1, -(1 << 40) + 2], np.int64)
    g = _graph(tm, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), t2)
    assert tmm.count_exact(g, cyc, 2) == 1
    assert g.info().t_min == -(1 << 40) and g.info().t_max == 2


def test_device_and_host_load_agree(tm):
    src, dst, t = synth.uniform_1k_graph()
    a = _graph(tm, src, dst, t, device=True)
    b = _graph(tm, src, dst, t, device=False)
    ia, ib = a.info(), b.info()
    assert (ia.m, ia.n_nodes, ia.n_pairs, ia.t_max) == (ib.m, ib.n_nodes, ib.n_pairs, ib.t_max)
    assert ia.n_pairs == len(set(zip(src.tolist(), dst.tolist())))
    mo = tm.Motif([0, 1], [1, 0])
    assert tm.count_exact(a, mo, 50_000) == tm.count_exact(b, mo, 50_000)


# ---------------------------------------------------------------- estimate ---
def _check_windows(tm, orc, g, src, dst, t, ms, md, delta, c, p, seed, k=0):
    mo = tm.Motif(ms, md)
    shift, recs = tm.estimate_windows(g, mo, delta, c, p, seed, k=k, all_windows=True)
    s_or, rec_or = orc.window_records(src, dst, t, ms, md, delta, c, seed, k=k, p=p, only_kept=False,
                                      threads=4)
    assert shift == s_or
    assert len(recs) == len(rec_or)
    for a, b in zip(recs, rec_or):
        assert (a["j"], a["start"], a["lo"], a["hi"], a["kept"]) == (b["j"], b["a"], b["lo"], b["hi"], b["kept"])
        assert a["count"] == b["count"], (a, b)
        w = a["w_int"] + a["w_frac"] * 2.0 ** -64
        assert abs(w - b["W"]) <= EST_RTOL * b["W"] + b["count"] * 2.0 ** -64 + 1e-300
    return recs


def test_uniform_20k_exact_and_estimate(tm, orc):
    """Uniform graph in full: N=1,000, M=20,000; cycle, delta=3,600;
    estimate with c=30, p=0.1, seed 1."""
    src, dst, t = synth.uniform_1k_graph()
    g = _graph(tm, src, dst, t)
    ms, md = synth.MOTIFS["cycle3"]
    mo = tm.Motif(ms, md)
    assert tm.count_exact(g, mo, 3600) == orc.count_exact(src, dst, t, ms, md, 3600)
    z = tm.estimate(g, mo, 3600, 30, 0.1, 1)
    assert _close(z, orc.estimate(src, dst, t, ms, md, 3600, 30, 0.1, 1))
    _check_windows(tm, orc, g, src, dst, t, ms, md, 3600, 30, 0.1, 1)
    # wider spans so that windows hold instances
    for delta in (20_000, 100_000):
        assert tm.count_exact(g, mo, delta) == orc.count_exact(src, dst, t, ms, md, delta)
        for (c, p, seed) in ((2, 0.5, 3), (3, 1.0, 4), (1, 0.7, 5)):
            z = tm.estimate(g, mo, delta, c, p, seed)
            zo = orc.estimate(src, dst, t, ms, md, delta, c, p, seed)
            assert _close(z, zo), (delta, c, p, seed, z, zo)
        _check_windows(tm, orc, g, src, dst, t, ms, md, delta, 2, 0.5, 3)


def test_estimate_mid_graph_parity(tm, orc):
    src, dst, t = synth.chung_lu_hawkes(3000, 300_000, 2.1, seed=22, horizon=6_000_000)
    g = _graph(tm, src, dst, t)
    for name in ("cycle3", "outstar3", "pingpong", "cycle4", "feedfwd3"):
        ms, md = synth.MOTIFS[name] if name in synth.MOTIFS else ([0, 1, 0], [1, 2, 2])
        mo = tm.Motif(ms, md)
        for (delta, c, p, seed) in ((600, 10, 0.1, 1), (3600, 30, 0.3, 2), (3600, 2, 1.0, 3)):
            z = tm.estimate(g, mo, delta, c, p, seed)
            zo = orc.estimate(src, dst, t, ms, md, delta, c, p, seed, threads=8)
            assert _close(z, zo), (name, delta, c, p, seed, z, zo)
    _check_windows(tm, orc, g, src, dst, t, *synth.MOTIFS["outstar3"], 3600, 10, 0.2, 9, k=2)


def test_batch_mixed_queries_match_single(tm, orc):
    """One batched launch of exact and estimate queries (several motifs, deltas,
    c, p, b and both q_j rules) gives each query's single-query answer and the
    oracle's."""
    src, dst, t = synth.chung_lu_hawkes(2000, 150_000, 2.1, seed=23, horizon=4_000_000)
    g = _graph(tm, src, dst, t)
    motifs = {n: tm.Motif(*synth.MOTIFS[n]) for n in ("cycle3", "outstar3", "pingpong", "cycle4")}
    qs, want = [], []
    for i, (n, mo) in enumerate(motifs.items()):
        ms, md = synth.MOTIFS[n]
        qs.append(tm.exact_query(mo, 3600))
        want.append(("exact", orc.count_exact(src, dst, t, ms, md, 3600, threads=8)))
        qs.append(tm.estimate_query(mo, 3600, 10, 0.25, 100 + i))
        want.append(("est", orc.estimate(src, dst, t, ms, md, 3600, 10, 0.25, 100 + i, threads=8)))
        qs.append(tm.estimate_query(mo, 600, 30, 0.5, 200 + i, b=3))
        want.append(("est", orc.estimate(src, dst, t, ms, md, 600, 30, 0.5, 200 + i, b=3, threads=8)))
        r = 20.0
        qfun = lambda j, a, e, _t=t, _r=r: min(1.0, _r * float(np.sum((_t - _t.min() >= a) & (_t - _t.min() <= e))) / len(_t))
        qs.append(tm.estimate_query(mo, 3600, 10, r, 300 + i, q_mode=tm.TM_Q_EDGES))
        want.append(("est", orc.estimate(src, dst, t, ms, md, 3600, 10, None, 300 + i, q=qfun, threads=8)))
    res = tm.run_batch(g, qs)
    for q, r, (kind, w) in zip(qs, res, want):
        assert r["status"] == 0
        if kind == "exact":
            assert r["count"] == w
        else:
            assert _close(r["estimate"], w), (r, w)
    # alone == in the mix
    for q, r in zip(qs, res):
        alone = tm.run_batch(g, [q])[0]
        assert alone["count"] == r["count"] and alone["estimate"] == r["estimate"]


def test_variance_estimate_is_lemma44(tm, orc):
    """var_hat = sum over kept windows of Y_j^2 (1 - p) / p^2, an unbiased
    estimate of Var[Z | s] = sum_j Y_j^2 (1 - p)/p (Lemma 4.4)."""
    src, dst, t = synth.chung_lu_hawkes(2000, 150_000, 2.1, seed=24, horizon=4_000_000)
    g = _graph(tm, src, dst, t)
    ms, md = synth.MOTIFS["outstar3"]
    mo = tm.Motif(ms, md)
    p = 0.3
    r = tm.run_batch(g, [tm.estimate_query(mo, 3600, 10, p, 7)])[0]
    s, recs = orc.window_records(src, dst, t, ms, md, 3600, 10, 7, p=p, threads=8)
    want = math.fsum(x["W"] ** 2 * (1 - p) / p ** 2 for x in recs if x["kept"])
    assert abs(r["var_hat"] - want) <= 1e-9 * want


# --------------------------------------------------- full size, sampled -----
@pytest.mark.slow
def test_bursty_10m_full_size_sampled_windows(tm, orc):
    """Full size N=1e5, M=1e7 (Chung-Lu 2.1 + Hawkes): the batched path in
    the benchmark's launch configuration; per-window exact counts and weights of
    sampled kept windows checked one by one against the oracle, and one full
    exact count."""
    src, dst, t = synth.bursty_100k_10m_graph()
    g = _graph(tm, src, dst, t)
    tn = t - t.min()
    for name in ("cycle3", "outstar3", "pingpong"):
        ms, md = synth.MOTIFS[name]
        mo = tm.Motif(ms, md)
        for delta in (600, 3600):
            shift, recs = tm.estimate_windows(g, mo, delta, 30, 0.1, 11)
            nz = [r for r in recs if r["hi"] > r["lo"]]
            rng = np.random.default_rng(delta)
            pick = rng.choice(len(nz), size=min(6, len(nz)), replace=False)
            cd = 30 * delta
            for i in pick:
                r = nz[int(i)]
                lo, hi = r["lo"], r["hi"]
                assert np.all(tn[lo:hi] >= r["start"]) and np.all(tn[lo:hi] <= r["start"] + cd - 1)
                cnt, hist, _ = orc.count_exact_hist(src[lo:hi], dst[lo:hi], tn[lo:hi], ms, md, delta,
                                                    threads=8, n_nodes=100_000)
                assert r["count"] == cnt
                wo = math.fsum((int(hist[d]) * cd) / (cd - d) for d in np.nonzero(hist)[0])
                w = r["w_int"] + r["w_frac"] * 2.0 ** -64
                assert abs(w - wo) <= EST_RTOL * wo + cnt * 2.0 ** -64
    ms, md = synth.MOTIFS["pingpong"]
    want = orc.count_exact(src, dst, t, ms, md, 600, threads=16)
    res = tm.run_batch(g, [tm.exact_query(tm.Motif(ms, md), 600)])[0]
    assert res["count"] == want


@pytest.mark.slow
def test_bursty_10m_full_size_benchmark_batch(tm, orc):
    """The benchmark's own 18-query batch on the full-size graph (N=1e5, M=1e7,
    Chung-Lu 2.1 + Hawkes), in one tm_run_batch as the benchmark times it: the
    three exact queries at delta = 86,400 that the rest of the batch rides on,
    the smaller spans counted inside their enumeration, and the nine estimates
    riding along, each against the oracle over the whole graph (counts
    bit-exact as int64, estimates within 1e-12)."""
    import os
    import bench
    src, dst, t = synth.bursty_100k_10m_graph()
    g = _graph(tm, src, dst, t)
    _, qs, meta = bench.make_queries(tm)
    res = tm.run_batch(g, qs)
    threads = os.cpu_count() or 8
    for q, r, (name, delta, kind) in zip(qs, res, meta):
        ms, md = synth.MOTIFS[name]
        assert r["status"] == 0
        if kind == "exact":
            want = orc.count_exact(src, dst, t, ms, md, delta, threads=threads)
            assert r["count"] == want, (name, delta, r["count"], want)
        else:
            want = orc.estimate(src, dst, t, ms, md, delta, q.c, q.p, q.seed, b=q.b, threads=threads)
            assert _close(r["estimate"], want), (name, delta, r["estimate"], want)


def test_fold_more_shifts_than_grid_y_and_many_slices(tm, orc):
    """The fold loops over shifts beyond the grid's y limit (65,535) and gives every
    query its own partial records: an estimate averaged over b = 66,000 shifts and
    one with more than 2,048 windows per shift (folded in several slices), in one
    batch and alone, against Algorithm 1 in the oracle."""
    rng = np.random.default_rng(65536)
    src, dst, t = synth.random_small_graph(rng, 5, 1000, 5000)
    g = _graph(tm, src, dst, t)
    ms, md = [0, 1], [1, 2]
    mo = tm.Motif(ms, md)
    qa = tm.estimate_query(mo, 50, 3, 0.05, 8, b=66_000)
    qb = tm.estimate_query(mo, 2, 1, 0.5, 9, b=3)
    want_a = orc.estimate(src, dst, t, ms, md, 50, 3, 0.05, 8, b=66_000)
    want_b = orc.estimate(src, dst, t, ms, md, 2, 1, 0.5, 9, b=3)
    assert want_a > 0 and want_b > 0
    for batch in ([qa, qb], [qb, qa], [qa], [qb]):
        for q, r in zip(batch, tm.run_batch(g, batch)):
            assert r["status"] == 0
            assert _close(r["estimate"], want_a if q is qa else want_b), (r, want_a, want_b)


def test_prepared_batch_cuda_graph_matches_run_batch(tm, orc):
    """The captured CUDA graph of a batch gives the same results as tm_run_batch,
    replay after replay (scratch re-zeroed inside the graph)."""
    import torch
    src, dst, t = synth.chung_lu_hawkes(2000, 150_000, 2.1, seed=25, horizon=4_000_000)
    g = _graph(tm, src, dst, t)
    qs = []
    for n in ("cycle3", "outstar3", "pingpong", "cycle4"):
        mo = tm.Motif(*synth.MOTIFS[n])
        qs += [tm.exact_query(mo, 3600), tm.estimate_query(mo, 3600, 10, 0.3, 5, b=2),
               tm.estimate_query(mo, 600, 5, 20.0, 6, q_mode=tm.TM_Q_EDGES)]
    qs.append(tm.Query(tm.Motif([0, 1], [1, 0]), -5))         # rejected: its status only
    want = tm.run_batch(g, qs, check=False)
    pb = tm.PreparedBatch(g, qs)
    st = torch.cuda.Stream()
    keys = ("status", "count", "estimate", "windows", "windows_kept", "var_hat", "shift_var", "p_used")
    for rep in range(3):
        pb.launch(st.cuda_stream)
        got = pb.results(st.cuda_stream, check=False)
        for a, b in zip(got, want):
            # (the work counters differ: in tm_run_batch, queries that ride along with another
            # query's enumeration report none of their own)
            assert {k: a[k] for k in keys} == {k: b[k] for k in keys}
    assert want[-1]["status"] == tm.TM_EINVAL
    assert want[0]["count"] == orc.count_exact(src, dst, t, *synth.MOTIFS["cycle3"], 3600, threads=8)
    pb.free()


def test_autotune_keeps_results(tm):
    src, dst, t = synth.chung_lu_hawkes(2000, 100_000, 2.1, seed=26, horizon=3_000_000)
    g = _graph(tm, src, dst, t)
    qs = [tm.exact_query(tm.Motif(*synth.MOTIFS[n]), 3600) for n in ("cycle3", "outstar3", "cycle4")]
    before = [r["count"] for r in tm.run_batch(g, qs)]
    best = tm.autotune(g, qs)
    assert best["block_threads"] in (128, 256) and best["chunk_items"] % 32 == 0
    assert tm.get_tuning() == best
    assert [r["count"] for r in tm.run_batch(g, qs)] == before
    tm.set_tuning(block_threads=256, blocks_per_sm=4, chunk_items=256, enum_threshold=48)


def test_wide_time_span_uses_64_bit_times(tm, orc):
    """Normalised spans >= 2^31 keep 64-bit time arrays; shorter spans use 32-bit
    ones.  Both give the oracle's counts and estimates."""
    rng = np.random.default_rng(31)
    for span, burst, est in (((1 << 40), (1 << 34), ((1 << 20), 3, 0.01)),
                             ((1 << 30), (1 << 20), ((1 << 18), 3, 0.5))):
        n, m = 50, 6000
        src = rng.integers(0, n, m)
        dst = (src + 1 + rng.integers(0, n - 1, m)) % n
        base = rng.integers(0, span, m // 20)
        t = np.sort((np.repeat(base, 20) + rng.integers(0, burst, m)) % span).astype(np.int64)
        src, dst = src.astype(np.int32), dst.astype(np.int32)
        g = _graph(tm, src, dst, t)
        delta = burst // 4
        for name in ("cycle3", "outstar3", "pingpong", "cycle4"):
            ms, md = synth.MOTIFS[name]
            mo = tm.Motif(ms, md)
            assert tm.count_exact(g, mo, delta) == orc.count_exact(src, dst, t, ms, md, delta)
            d2, c2, p2 = est
            z = tm.estimate(g, mo, d2, c2, p2, 17)
            assert _close(z, orc.estimate(src, dst, t, ms, md, d2, c2, p2, 17))


@pytest.mark.slow
def test_bursty_100m_full_size_sampled_windows(tm, orc):
    """Full size N=1e6, M=1e8 (Chung-Lu 2.0 + Hawkes): the 4-cycle at
    delta=3600 in the batched launch the benchmark times (all c x p x seed
    combinations of one shift each in one batch); per-window exact counts and
    weights of sampled kept windows checked one by one against the oracle."""
    import torch
    src, dst, t = synth.bursty_1m_100m_graph()
    g = _graph(tm, src, dst, t)
    tn = t - t.min()
    ms, md = synth.MOTIFS["cycle4"]
    mo = tm.Motif(ms, md)
    qs = [tm.estimate_query(mo, 3600, c, p, seed=9000 + s) for c in (10, 30, 100) for p in (0.01, 0.1)
          for s in range(4)]
    res = tm.run_batch(g, qs)
    assert all(r["status"] == 0 for r in res)
    rng = np.random.default_rng(3)
    for (c, p, seed) in ((10, 0.01, 9000), (100, 0.1, 9002)):
        shift, recs = tm.estimate_windows(g, mo, 3600, c, p, seed)
        nz = [r for r in recs if r["hi"] > r["lo"]]
        cd = c * 3600
        for i in rng.choice(len(nz), size=min(3, len(nz)), replace=False):
            r = nz[int(i)]
            lo, hi = r["lo"], r["hi"]
            cnt, hist, _ = orc.count_exact_hist(src[lo:hi], dst[lo:hi], tn[lo:hi], ms, md, 3600,
                                                threads=16, n_nodes=1_000_000)
            assert r["count"] == cnt
            wo = math.fsum((int(hist[d]) * cd) / (cd - d) for d in np.nonzero(hist)[0])
            w = r["w_int"] + r["w_frac"] * 2.0 ** -64
            assert abs(w - wo) <= EST_RTOL * wo + cnt * 2.0 ** -64
        # the single-query estimate equals the batched one for the same seed
        z = tm.estimate(g, mo, 3600, c, p, seed)
        k = [i for i, q in enumerate(qs) if (q.c, q.p, q.seed) == (c, p, seed)][0]
        assert z == res[k]["estimate"]


@pytest.mark.slow
def test_hubs_1b_full_size_sampled_windows(tm, orc):
    """Full size N=1e7, M=1e9 (Chung-Lu 1.8 capped at degree 5e6, Hawkes
    times plus 1,000 hub bursts of up to 1e4 edges in 60 s), drawn on the GPU:
    the out-star at delta=1800 estimated with c=30, p=0.01 for 8 seeds in one
    batched launch; sampled kept windows checked one by one against the oracle.
    Windows holding a hub burst are not sampled (the oracle's enumeration is
    cubic in a burst; bursts are checked at smaller scale in test_hub_heavy_graph)."""
    import torch
    d_src, d_dst, d_t = synth.hub_bursty_10m_1b_graph_gpu()
    g = tm.Graph(d_src, d_dst, d_t)
    ms, md = synth.MOTIFS["outstar3"]
    mo = tm.Motif(ms, md)
    res = tm.run_batch(g, [tm.estimate_query(mo, 1800, 30, 0.01, seed=500 + s) for s in range(8)])
    assert all(r["status"] == 0 and r["windows_kept"] > 0 for r in res)
    # per-window detail at p = 0.1 (about 117 kept windows, some 40 % of them burst-free)
    shift, recs = tm.estimate_windows(g, mo, 1800, 30, 0.1, 500)
    t_min = int(d_t[0])
    cd = 30 * 1800
    checked = 0
    for r in recs:
        if checked == 3:
            break
        lo, hi = r["lo"], r["hi"]
        if hi <= lo:
            continue
        src = d_src[lo:hi].cpu().numpy()
        tn = d_t[lo:hi].cpu().numpy() - t_min
        # a hub burst: one source with > 1,000 edges in one 10-minute bin
        # (the heaviest hubs average about 50 per bin)
        binned = src.astype(np.int64) * (1 << 20) + (tn - tn.min()) // 600
        if np.unique(binned, return_counts=True)[1].max() > 1000:
            continue
        dst = d_dst[lo:hi].cpu().numpy()
        cnt, hist, _ = orc.count_exact_hist(src, dst, tn, ms, md, 1800, threads=16, n_nodes=10_000_000)
        assert r["count"] == cnt
        wo = math.fsum((int(hist[d]) * cd) / (cd - d) for d in np.nonzero(hist)[0])
        w = r["w_int"] + r["w_frac"] * 2.0 ** -64
        assert abs(w - wo) <= EST_RTOL * wo + cnt * 2.0 ** -64
        checked += 1
    assert checked >= 2
    g.free()
    del d_src, d_dst, d_t
    torch.cuda.empty_cache()
    tm.release_cached_memory()


def test_dense_sampling_node_grouped_windows(tm, orc):
    """Estimates that keep most windows, with windows holding many edges per
    node, enumerate each window's first edges grouped by node (a per-shift
    partition of the adjacency view by window); same results as the oracle,
    window by window."""
    src, dst, t = synth.chung_lu_hawkes(200, 50_000, 2.1, seed=27, horizon=1_000_000)
    g = _graph(tm, src, dst, t)
    for name in ("cycle3", "outstar3", "pingpong", "cycle4"):
        ms, md = synth.MOTIFS[name]
        mo = tm.Motif(ms, md)
        for (c, p, seed, b) in ((10, 0.3, 1, 2), (10, 1.0, 2, 1), (30, 0.6, 3, 1)):
            r = tm.run_batch(g, [tm.estimate_query(mo, 3600, c, p, seed, b=b)])[0]
            zo = orc.estimate(src, dst, t, ms, md, 3600, c, p, seed, b=b, threads=8)
            assert _close(r["estimate"], zo), (name, c, p, seed, b, r["estimate"], zo)
        _check_windows(tm, orc, g, src, dst, t, ms, md, 3600, 10, 0.5, 4)


TWO_NODE = [([0, 0, 0], [1, 1, 1]), ([0, 0, 1], [1, 1, 0]), ([0, 1, 0], [1, 0, 1]), ([0, 1, 1], [1, 0, 0])]


def test_two_node_motifs_exact_tiny_and_bruteforce(tm, orc):
    """The four two-node three-edge motifs (Algorithm 2's family, counted from
    the pair prefix tables) on tiny graphs with ties, multi-edges and
    self-loops: against the oracle's enumerator and Def. 2.2 by brute force."""
    rng = np.random.default_rng(77)
    for trial in range(50):
        n = int(rng.integers(2, 5))
        m = int(rng.integers(0, 40))
        src, dst, t = synth.random_small_graph(rng, n, m, int(rng.integers(1, 30)), self_loops=trial % 3 == 0)
        g = _graph(tm, src, dst, t, device=trial % 2 == 0)
        for ms, md in TWO_NODE:
            mo = tm.Motif(ms, md)
            for delta in (0, 2, 9, 1000):
                want = orc.count_exact(src, dst, t, ms, md, delta)
                assert tm.count_exact(g, mo, delta) == want, (trial, ms, md, delta)
            if m <= 12:
                want, _ = orc.count_bruteforce(src, dst, t, ms, md, 7)
                assert tm.count_exact(g, mo, 7) == want


def test_two_node_motifs_mid_graph_exact_estimate(tm, orc):
    """A bursty graph with reply edges: exact counts against the enumerator and
    (ping-pong) Algorithm 2; estimates in time order and node-grouped (dense)
    windows against the oracle, window by window."""
    src, dst, t = synth.chung_lu_hawkes(500, 120_000, 2.1, seed=31, horizon=3_000_000)
    g = _graph(tm, src, dst, t)
    # Algorithm 2 takes distinct timestamps: the first edge of every timestamp
    _, first = np.unique(t, return_index=True)
    gu = _graph(tm, src[first], dst[first], t[first])
    for delta in (600, 3600, 86400):
        want = orc.ex23(src[first], dst[first], t[first], delta)[0]
        assert tm.count_exact(gu, tm.Motif([0, 1, 0], [1, 0, 1]), delta) == want
    for ms, md in TWO_NODE:
        mo = tm.Motif(ms, md)
        for delta in (600, 3600, 86400):
            want = orc.count_exact(src, dst, t, ms, md, delta, threads=8)
            assert tm.count_exact(g, mo, delta) == want, (ms, md, delta)
        for (c, p, seed, b) in ((10, 0.1, 1, 1), (30, 0.9, 2, 2), (3, 0.5, 3, 1)):
            r = tm.run_batch(g, [tm.estimate_query(mo, 3600, c, p, seed, b=b)])[0]
            zo = orc.estimate(src, dst, t, ms, md, 3600, c, p, seed, b=b, threads=8)
            assert _close(r["estimate"], zo), (ms, md, c, p, seed, b, r["estimate"], zo)
        _check_windows(tm, orc, g, src, dst, t, ms, md, 3600, 10, 0.5, 4)
    # mixed with three-node queries in one batch, and as a prepared (captured) batch
    qs = [tm.exact_query(tm.Motif(ms, md), 3600) for ms, md in TWO_NODE]
    qs += [tm.estimate_query(tm.Motif(ms, md), 3600, 10, 0.3, 9) for ms, md in TWO_NODE]
    qs.append(tm.exact_query(tm.Motif(*synth.MOTIFS["cycle3"]), 3600))
    alone = [tm.run_batch(g, [q])[0] for q in qs]
    mixed = tm.run_batch(g, qs)
    pb = tm.PreparedBatch(g, qs)
    pb.launch()
    prep = pb.results()
    for a, b_, c_ in zip(alone, mixed, prep):
        assert a["count"] == b_["count"] == c_["count"]
        assert a["estimate"] == b_["estimate"] == c_["estimate"]
    pb.free()


def _auto_p(pilot, target, b):
    """The pilot rule stated for TM_Q_AUTO, in the same floating-point steps."""
    z, p0 = 1.96, 0.05
    z0 = pilot["estimate"]
    s2 = pilot["var_hat"] * p0 / (1.0 - p0)
    if not z0 > 0.0:
        return 1.0
    if not s2 > 0.0:
        return p0
    r = float(b) * (target * z0 / z) * (target * z0 / z) / s2
    return min(1.0, max(p0, 1.0 / (1.0 + r)))


def test_auto_p_from_pilot_variance(tm, orc):
    """TM_Q_AUTO: p chosen from a pilot's Lemma 4.4 variance estimate; the result is
    the plain uniform estimate at that p (checked against the oracle), and
    shift_var is the sample variance of the per-shift estimates."""
    src, dst, t = synth.chung_lu_hawkes(3000, 300_000, 2.1, seed=61, horizon=6_000_000)
    g = _graph(tm, src, dst, t)
    for name in ("cycle3", "outstar3", "pingpong"):
        ms, md = synth.MOTIFS[name]
        mo = tm.Motif(ms, md)
        exact = tm.count_exact(g, mo, 3600)
        for seed in (3, 4):
            q = tm.estimate_query(mo, 3600, 10, 0.05, seed, b=2, q_mode=tm.TM_Q_AUTO)
            r = tm.run_batch(g, [q])[0]
            pilot = tm.run_batch(g, [tm.estimate_query(mo, 3600, 10, tm.TM_AUTO_PILOT_P,
                                                       seed ^ tm.TM_AUTO_PILOT_SEED_XOR, b=2)])[0]
            p = _auto_p(pilot, 0.05, 2)
            assert r["p_used"] == p and 0.05 <= p <= 1.0
            plain = tm.run_batch(g, [tm.estimate_query(mo, 3600, 10, p, seed, b=2)])[0]
            assert r["estimate"] == plain["estimate"] and r["shift_var"] == plain["shift_var"]
            zo = orc.estimate(src, dst, t, ms, md, 3600, 10, p, seed, b=2, threads=8)
            assert _close(r["estimate"], zo)
            # shift_var: sample variance of the two per-shift estimates
            zk = []
            for k in range(2):
                _, recs = tm.estimate_windows(g, mo, 3600, 10, p, seed, k=k)
                zk.append(sum(x["w_int"] + x["w_frac"] * 2.0 ** -64 for x in recs) / p)
            sv = (zk[0] - zk[1]) ** 2 / 2.0
            assert abs(r["shift_var"] - sv) <= 1e-9 * max(sv, 1.0)
        assert exact > 0
    # not available where p cannot be chosen at run time
    q = tm.estimate_query(mo, 3600, 10, 0.05, 1, q_mode=tm.TM_Q_AUTO)
    pb = tm.PreparedBatch(g, [q])
    pb.launch()
    assert pb.results(check=False)[0]["status"] == tm.TM_EINVAL
    pb.free()
    res, _ = tm.stream_run(src, dst, t, [q], 100_000, int(max(src.max(), dst.max())) + 1, check=False)
    assert res[0]["status"] == tm.TM_EINVAL


def test_auto_p_meets_target_on_most_seeds(tm):
    """With target 5 % the sampling error stays near the target (the shift variance
    is not part of the rule, so the bound is loose: 80 % of seeds within 10 %)."""
    src, dst, t = synth.chung_lu_hawkes(3000, 300_000, 2.1, seed=62, horizon=6_000_000)
    g = _graph(tm, src, dst, t)
    mo = tm.Motif(*synth.MOTIFS["cycle3"])
    exact = tm.count_exact(g, mo, 3600)
    qs = [tm.estimate_query(mo, 3600, 30, 0.05, 100 + s, b=2, q_mode=tm.TM_Q_AUTO) for s in range(20)]
    res = tm.run_batch(g, qs)
    errs = [abs(r["estimate"] - exact) / exact for r in res]
    assert sum(e <= 0.10 for e in errs) >= 16, errs


def test_exact_spans_ride_along_in_one_enumeration(tm, orc):
    """Exact three-edge queries of one motif at several spans share the largest span's
    enumeration (each instance also counted for every span its duration fits): counts
    equal the single-query counts and the oracle's; the members report no work."""
    src, dst, t = synth.chung_lu_hawkes(2000, 100_000, 2.1, seed=7, horizon=3_000_000,
                                        max_degree=20_000, hub_bursts=6, burst_max=400)
    g = _graph(tm, src, dst, t)
    names = ("cycle3", "outstar3", "pingpong", "cycle4")
    qs, want = [], []
    for n in names:
        ms, md = synth.MOTIFS[n]
        mo = tm.Motif(ms, md)
        for d in (86400, 600, 3600, 3600, 0, 7):
            qs.append(tm.exact_query(mo, d))
            want.append(orc.count_exact(src, dst, t, ms, md, d, threads=8))
    mo2 = tm.Motif([2, 2, 2], [0, 1, 0])          # the same motif through another handle
    qs.append(tm.exact_query(mo2, 1800))
    want.append(orc.count_exact(src, dst, t, [2, 2, 2], [0, 1, 0], 1800, threads=8))
    res = tm.run_batch(g, qs)
    for q, r, w in zip(qs, res, want):
        assert r["status"] == 0 and r["count"] == w, (q.delta, r["count"], w)
        assert r["count"] == tm.run_batch(g, [q])[0]["count"]
    # per motif at most one query did the work (the largest span); four-edge motifs are alone
    for k, n in enumerate(names[:3]):
        worked = [r["first_edges"] > 0 for r in res[6 * k:6 * k + 6]]
        assert sum(worked) <= 2 and worked[0]   # groups of at most four queries


def test_all_windows_kept_uses_whole_graph_pass(tm, orc):
    """p = 1 keeps every window: the batch then takes every edge as a first edge in node
    order, clamped to its own window, with one accumulator per shift.  Same estimate as the
    per-window path of a prepared batch (bit for bit) and as the oracle."""
    src, dst, t = synth.chung_lu_hawkes(2000, 150_000, 2.1, seed=29, horizon=4_000_000)
    g = _graph(tm, src, dst, t)
    qs, want = [], []
    for n in ("cycle3", "outstar3", "pingpong", "cycle4"):
        ms, md = synth.MOTIFS[n]
        mo = tm.Motif(ms, md)
        for (d, c, seed, b) in ((3600, 10, 5, 2), (600, 3, 6, 1), (86400, 30, 7, 1)):
            qs.append(tm.estimate_query(mo, d, c, 1.0, seed, b=b))
            want.append(orc.estimate(src, dst, t, ms, md, d, c, 1.0, seed, b=b, threads=8))
    res = tm.run_batch(g, qs)
    pb = tm.PreparedBatch(g, qs)
    pb.launch()
    prep = pb.results()
    pb.free()
    for q, r, p_, w in zip(qs, res, prep, want):
        assert r["status"] == 0 and _close(r["estimate"], w), (q.delta, r["estimate"], w)
        assert r["estimate"] == p_["estimate"] and r["count"] == p_["count"]
        assert r["windows"] == p_["windows"] and r["windows_kept"] == p_["windows_kept"] == r["windows"]
        assert r["var_hat"] == 0.0


def test_estimates_ride_along_exact_queries(tm, orc):
    """An estimate of the same three-edge motif as an exact query of at least its span takes
    its instances from that query's enumeration (any p, b or q_j rule): results equal the
    estimate run alone (bit for bit: counts, estimates, variance estimates, kept windows)
    and the oracle's."""
    src, dst, t = synth.chung_lu_hawkes(2000, 150_000, 2.1, seed=33, horizon=4_000_000,
                                        max_degree=20_000, hub_bursts=4, burst_max=300)
    g = _graph(tm, src, dst, t)
    qs, want = [], []
    for n in ("cycle3", "outstar3", "pingpong"):
        ms, md = synth.MOTIFS[n]
        mo = tm.Motif(ms, md)
        qs += [tm.exact_query(mo, 86400), tm.exact_query(mo, 3600)]
        want += [("exact", orc.count_exact(src, dst, t, ms, md, 86400, threads=8)),
                 ("exact", orc.count_exact(src, dst, t, ms, md, 3600, threads=8))]
        for (d, c, p, seed, b) in ((86400, 30, 1.0, 3, 1), (3600, 10, 1.0, 4, 1), (600, 5, 1.0, 5, 1),
                                   (3600, 10, 0.3, 6, 2), (600, 5, 0.5, 7, 1), (3600, 4, 1.0, 9, 2)):
            qs.append(tm.estimate_query(mo, d, c, p, seed, b=b))
            want.append(("est", orc.estimate(src, dst, t, ms, md, d, c, p, seed, b=b, threads=8)))
        qs.append(tm.estimate_query(mo, 3600, 5, 20.0, 8, q_mode=tm.TM_Q_EDGES))
        r_ = 20.0
        qfun = lambda j, a, e, _t=t, _r=r_: min(1.0, _r * float(np.sum((_t - _t.min() >= a) & (_t - _t.min() <= e))) / len(_t))
        want.append(("est", orc.estimate(src, dst, t, ms, md, 3600, 5, None, 8, q=qfun, threads=8)))
    res = tm.run_batch(g, qs)
    for q, r, (kind, w) in zip(qs, res, want):
        assert r["status"] == 0
        if kind == "exact":
            assert r["count"] == w
        else:
            assert _close(r["estimate"], w), (q.delta, r["estimate"], w)
        alone = tm.run_batch(g, [q])[0]
        assert alone["count"] == r["count"] and alone["estimate"] == r["estimate"]
        assert alone["windows"] == r["windows"] and alone["windows_kept"] == r["windows_kept"]
        assert alone["var_hat"] == r["var_hat"] and alone["shift_var"] == r["shift_var"]


def test_deferred_rider_records_overflow_reruns(tm, orc):
    """The matcher leaves riders and smaller spans to a second pass through a record buffer; a
    batch that needs more records than the buffer holds runs again with room for all of them.
    With the capacity set to 16 records the results equal those at the default capacity bit for
    bit, and the oracle's."""
    src, dst, t = synth.chung_lu_hawkes(1500, 80_000, 2.1, seed=41, horizon=3_000_000)
    g = _graph(tm, src, dst, t)
    ms, md = synth.MOTIFS["cycle3"]
    mo = tm.Motif(ms, md)
    ms2, md2 = synth.MOTIFS["pingpong"]
    mo2 = tm.Motif(ms2, md2)
    qs = [tm.exact_query(mo, 86400), tm.exact_query(mo, 3600),
          tm.estimate_query(mo, 86400, 30, 1.0, 3), tm.estimate_query(mo, 3600, 10, 0.5, 4, b=2),
          tm.exact_query(mo2, 86400), tm.estimate_query(mo2, 3600, 10, 0.5, 5)]
    ref = tm.run_batch(g, qs)
    tm.profile_enable(True)
    try:
        tm.set_ride_capacity(16)
        res = tm.run_batch(g, qs)
        records = tm.profile_last()["ride_records"]
    finally:
        tm.profile_enable(False)
        tm.set_ride_capacity(1 << 23)
    assert records > 16, records
    for r, w in zip(res, ref):
        assert r["status"] == 0
        assert r["count"] == w["count"] and r["estimate"] == w["estimate"]
        assert r["var_hat"] == w["var_hat"] and r["windows_kept"] == w["windows_kept"]
    assert res[0]["count"] == orc.count_exact(src, dst, t, ms, md, 86400, threads=8)
    assert res[1]["count"] == orc.count_exact(src, dst, t, ms, md, 3600, threads=8)
    assert _close(res[3]["estimate"], orc.estimate(src, dst, t, ms, md, 3600, 10, 0.5, 4, b=2, threads=8))
    assert _close(res[5]["estimate"], orc.estimate(src, dst, t, ms2, md2, 3600, 10, 0.5, 5, threads=8))
    with pytest.raises(tm.TmError):
        tm.set_ride_capacity(0)


def test_sharing_limits_and_mixes(tm, orc):
    """Batches that stretch the sharing rules: more spans than one leader carries, more
    estimates than riders allowed, equal spans, a rejected query, automatic p and q_j rules
    side by side -- every result equals the query run alone."""
    src, dst, t = synth.chung_lu_hawkes(1500, 80_000, 2.1, seed=37, horizon=3_000_000)
    g = _graph(tm, src, dst, t)
    mo = tm.Motif(*synth.MOTIFS["cycle3"])
    mo2 = tm.Motif(*synth.MOTIFS["outstar3"])
    qs = [tm.exact_query(mo, d) for d in (86400, 600, 3600, 3600, 7200, 100, 0)]
    qs += [tm.estimate_query(mo, d, c, p, s, b=b) for (d, c, p, s, b) in
           ((3600, 10, 0.4, 1, 1), (3600, 10, 0.4, 2, 3), (600, 30, 0.9, 3, 1), (86400, 2, 0.2, 4, 1),
            (7200, 5, 1.0, 5, 1), (100, 10, 0.5, 6, 2), (3600, 3, 0.7, 7, 1), (120000, 10, 0.5, 8, 1))]
    qs.append(tm.estimate_query(mo, 3600, 10, 0.05, 9, b=2, q_mode=tm.TM_Q_AUTO))
    qs.append(tm.estimate_query(mo, 3600, 10, 15.0, 10, q_mode=tm.TM_Q_EDGES))
    qs.append(tm.Query(mo, -3))                                  # rejected
    qs += [tm.exact_query(mo2, 3600), tm.estimate_query(mo2, 3600, 10, 0.5, 11),
           tm.estimate_query(mo2, 600, 10, 0.5, 12, b=2)]
    res = tm.run_batch(g, qs, check=False)
    keys = ("status", "count", "estimate", "windows", "windows_kept", "var_hat", "shift_var", "p_used")
    for q, r in zip(qs, res):
        alone = tm.run_batch(g, [q], check=False)[0]
        assert {k: r[k] for k in keys} == {k: alone[k] for k in keys}, (q.mode, q.delta, q.p, r, alone)
    assert res[17]["status"] == tm.TM_EINVAL
    ms, md = synth.MOTIFS["cycle3"]
    for q, r in zip(qs[:7], res[:7]):
        assert r["count"] == orc.count_exact(src, dst, t, ms, md, q.delta, threads=8)
