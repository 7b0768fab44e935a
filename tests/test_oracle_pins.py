"""Pins that tie the CPU oracle to the paper and to mathematics, not to itself.

Runs on CPU (no GPU marker).  Citations: Liu, Benson & Charikar, "A sampling
framework for counting temporal motifs" (WSDM 2019).
"""
import itertools
import json
import math
import os
from collections import Counter

import numpy as np
import pytest

from paper_1810_00980_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

RANDOM_MOTIFS = [
    ([0], [1]),
    ([0, 1], [1, 0]),
    ([0, 0], [1, 1]),
    ([0, 1], [1, 2]),
    ([0, 2], [1, 1]),
    ([0, 1, 2], [1, 2, 0]),          # cycle
    ([2, 2, 2], [0, 1, 0]),          # out-star c->a, c->b, c->a
    ([0, 1, 0], [1, 0, 1]),          # ping-pong
    ([0, 2, 1], [1, 3, 2]),          # second edge shares no node with the first
    ([0, 1, 2, 3], [1, 2, 3, 0]),    # 4-cycle
    ([0, 0, 0, 0], [1, 2, 1, 2]),
    ([1, 0, 2, 0], [0, 2, 1, 1]),
]


def _arr(edges):
    e = sorted(edges, key=lambda x: x[2])
    return (np.array([x[0] for x in e], np.int32), np.array([x[1] for x in e], np.int32),
            np.array([x[2] for x in e], np.int64))


# ---------------------------------------------------------------- P1 --------
def test_hand_counted_graphs(oracle_mod):
    """Hand-worked counts and duration histograms (Defs. 2.2, 2.3, Fig. 1 caption)."""
    cases = json.load(open(os.path.join(GOLDEN, "hand_counted.json")))["cases"]
    for c in cases:
        src, dst, t = _arr(c["edges"])
        mu = [e[0] for e in c["motif"]]
        mv = [e[1] for e in c["motif"]]
        want_hist = {int(k): v for k, v in c["hist"].items()}
        cnt, hist = oracle_mod.count_bruteforce(src, dst, t, mu, mv, c["delta"])
        assert cnt == c["count"], c["name"]
        assert dict(hist) == want_hist, c["name"]
        cnt2, hist2, _ = oracle_mod.count_exact_hist(src, dst, t, mu, mv, c["delta"])
        assert cnt2 == c["count"], c["name"]
        assert {d: int(x) for d, x in enumerate(hist2) if x} == want_hist, c["name"]


# ---------------------------------------------------------------- P2 --------
@pytest.mark.parametrize("motif", RANDOM_MOTIFS)
def test_exhaustive_vs_enumerator(oracle_mod, motif):
    """Def. 2.2 by exhaustive subsets vs the pruned enumerator on graphs of <= 12
    edges with repeated pairs, ties, self-loops and windows."""
    rng = np.random.default_rng(1000 + len(motif[0]) * 17 + sum(motif[1]))
    for trial in range(120):
        n = int(rng.integers(2, 6))
        m = int(rng.integers(0, 13))
        src, dst, t = synth.random_small_graph(rng, n, m, int(rng.integers(1, 25)),
                                               self_loops=bool(trial % 3 == 0))
        delta = int(rng.integers(0, 20))
        w = None
        if trial % 4 == 1 and m:
            a = int(rng.integers(0, 12))
            w = (a, a + int(rng.integers(0, 15)))
        kw = {} if w is None else dict(w_lo=w[0], w_hi=w[1])
        c1, h1 = oracle_mod.count_bruteforce(src, dst, t, *motif, delta, **kw)
        c2, h2, _ = oracle_mod.count_exact_hist(src, dst, t, *motif, delta, **kw)
        assert c1 == c2, (trial, src, dst, t, delta, w)
        assert dict(h1) == {d: int(x) for d, x in enumerate(h2) if x}


def test_enumerator_threads_agree(oracle_mod):
    src, dst, t = synth.chung_lu_hawkes(300, 20_000, 2.1, seed=5, horizon=400_000)
    for motif in ([0, 1, 2], [1, 2, 0]), ([2, 2, 2], [0, 1, 0]):
        c1, h1, _ = oracle_mod.count_exact_hist(src, dst, t, *motif, 3600, threads=1)
        c4, h4, _ = oracle_mod.count_exact_hist(src, dst, t, *motif, 3600, threads=4)
        assert c1 == c4 and np.array_equal(h1, h4)


# ---------------------------------------------------------------- P10 -------
def test_closed_forms(oracle_mod):
    """l = 1: every non-loop edge is an instance.  One pair with m edges at
    distinct times inside delta and motif a->b x3: C(m, 3) instances, and
    a->b x2 has (m - d) instances of duration d."""
    rng = np.random.default_rng(7)
    src, dst, t = synth.random_small_graph(rng, 6, 40, 100, self_loops=True)
    assert oracle_mod.count_exact(src, dst, t, [0], [1], 0) == int(np.sum(src != dst))
    for m in range(0, 9):
        s = np.zeros(m, np.int32)
        d = np.ones(m, np.int32)
        tt = np.arange(m, dtype=np.int64) * 3
        assert oracle_mod.count_exact(s, d, tt, [0, 0, 0], [1, 1, 1], 10 ** 6) == math.comb(m, 3)
        _, h, _ = oracle_mod.count_exact_hist(s, d, tt, [0, 0], [1, 1], 3 * m)
        for dd in range(len(h)):
            want = (m - dd // 3) if (dd % 3 == 0 and 0 < dd // 3 < m) else 0
            assert h[dd] == want


# ---------------------------------------------------------------- P8 --------
def _cliques(n, edges, k):
    adj = {frozenset(e) for e in edges}
    return sum(all(frozenset((a, b)) in adj for a, b in itertools.combinations(c, 2))
               for c in itertools.combinations(range(1, n + 1), k))


@pytest.mark.parametrize("k", [2, 3, 4])
def test_clique_reduction(oracle_mod, k):
    """Theorem 3.1: the star motif S has as many delta-instances in T (delta
    unbounded) as the static graph G has k-cliques."""
    rng = np.random.default_rng(k)
    for trial in range(6 if k < 4 else 3):
        n = int(rng.integers(k, 7))
        pairs = [e for e in itertools.combinations(range(1, n + 1), 2) if rng.random() < 0.6]
        src, dst, t, ms, md, delta = synth.clique_reduction(n, pairs, k)
        want = _cliques(n, pairs, k)
        got = oracle_mod.count_exact(src, dst, t, ms, md, delta)
        assert got == want, (n, pairs, k)
        if k == 2 and len(t) <= 24:
            assert oracle_mod.count_bruteforce(src, dst, t, ms, md, delta)[0] == want


# ---------------------------------------------------------------- P9 --------
def test_ex23_matches_enumerator(oracle_mod):
    """Algorithm 2 (EX23, inner loop from j = i + 1) is an independent exact
    counter for (u,v),(v,u),(u,v); it must agree with Def. 2.2 counting,
    durations included."""
    rng = np.random.default_rng(23)
    for trial in range(40):
        n = int(rng.integers(2, 5))
        m = int(rng.integers(0, 40))
        src = rng.integers(0, n, m)
        dst = (src + 1 + rng.integers(0, n - 1, m)) % n
        t = rng.permutation(200)[:m].astype(np.int64)        # distinct times
        order = np.argsort(t)
        src, dst, t = src[order].astype(np.int32), dst[order].astype(np.int32), t[order]
        delta = int(rng.integers(0, 120))
        c1, h1 = oracle_mod.ex23(src, dst, t, delta)
        c2, h2, _ = oracle_mod.count_exact_hist(src, dst, t, [0, 1, 0], [1, 0, 1], delta)
        assert c1 == c2
        assert dict(h1) == {d: int(x) for d, x in enumerate(h2) if x}
        if m <= 12:
            assert oracle_mod.count_bruteforce(src, dst, t, [0, 1, 0], [1, 0, 1], delta)[0] == c1


# ---------------------------------------------------------------- RNG -------
def test_splitmix64_known_answers(oracle_mod):
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, n, val = (int(x) for x in line.split())
        assert oracle_mod.rng.splitmix64_output(seed, n) == val


def test_rng_draws_ranges(oracle_mod):
    r = oracle_mod.rng
    us = [r.uniform(9, 0, j) for j in range(1, 4001)]
    assert all(0.0 <= u < 1.0 for u in us)
    # uniformity: each decile near 400 (loose 6-sigma band)
    hist = np.histogram(us, bins=10, range=(0, 1))[0]
    assert np.all(np.abs(hist - 400) < 6 * math.sqrt(400 * 0.9))
    for cd in (1, 2, 7, 36000):
        ss = [r.shift(s, k, cd) for s in range(20) for k in range(5)]
        assert all(-cd + 1 <= s <= 0 for s in ss)


# ---------------------------------------------------------------- P3 --------
def test_eq2_containment_by_shift(oracle_mod):
    """Eq. 2: an instance of duration Delta lies inside one interval of I_s for
    exactly c*delta - Delta of the c*delta shifts s (so with probability
    1 - Delta/(c delta)).  Brute force over every shift, every placement, and
    the window range j = 1 .. 1 + ceil(t_max/(c delta)) of Algorithm 1."""
    for cd in (1, 2, 3, 5, 8):
        t_max = 3 * cd + 2
        for t1 in range(0, t_max + 1):
            for tl in range(t1, min(t_max, t1 + cd - 1) + 1):
                hits = 0
                for s in range(-cd + 1, 1):
                    wins = oracle_mod.windows_of_shift(t_max, cd, s)
                    hits += any(a <= t1 and tl <= e for (_, a, e) in wins)
                assert hits == cd - (tl - t1), (cd, t1, tl)


def _all_shift_records(oracle_mod, src, dst, t, motif, delta, c):
    """Per-window exact histograms for every shift s, all windows kept."""
    import oracle.core as core
    cd = c * delta
    tn = t - t.min()
    out = {}
    for s in range(-cd + 1, 1):
        rows = []
        for (j, a, e) in core.windows_of_shift(int(tn.max()), cd, s):
            lo = int(np.searchsorted(tn, a, "left"))
            hi = int(np.searchsorted(tn, e, "right"))
            if hi > lo:
                cnt, h, _ = oracle_mod.count_exact_hist(src[lo:hi], dst[lo:hi], tn[lo:hi], *motif,
                                                        delta, n_nodes=int(max(src.max(), dst.max())) + 1)
            else:
                cnt, h = 0, np.zeros(delta + 1, np.int64)
            rows.append((j, h))
        out[s] = rows
    return out


# ---------------------------------------------------------------- P4, P6 ----
def test_lemma41_and_42_over_all_shifts(oracle_mod):
    """Lemma 4.1 in integers: summed over all c*delta shifts, the per-window
    duration histograms give (c delta - Delta) * H[Delta], hence the mean of
    ||Y_s||_1 over shifts is exactly C_M.  Lemma 4.2: the variance of
    ||Y_s||_1 over shifts is at most C_M^2 / (c - 1)."""
    rng = np.random.default_rng(41)
    src, dst, t = synth.random_small_graph(rng, 5, 160, 400)
    motif = ([0, 1, 2], [1, 2, 0])
    delta = 9
    for c in (2, 3):
        cd = c * delta
        C, H, _ = oracle_mod.count_exact_hist(src, dst, t, *motif, delta)
        assert C > 0
        recs = _all_shift_records(oracle_mod, src, dst, t, motif, delta, c)
        tot = np.zeros(delta + 1, np.int64)
        norms = []
        for s, rows in recs.items():
            y1 = 0.0
            for j, h in rows:
                tot += h
                y1 += sum(int(h[d]) * cd / (cd - d) for d in range(delta + 1))
            norms.append(y1)
        assert np.array_equal(tot, np.array([(cd - d) * H[d] for d in range(delta + 1)]))
        assert abs(np.mean(norms) - C) <= 1e-9 * C
        assert np.var(norms) <= C * C / (c - 1)


# ---------------------------------------------------------------- P5 --------
def test_thm43_lemma44_exhaustive_keep_sets(oracle_mod):
    """Theorem 4.3 / Lemma 4.4 conditional on a shift: over all 2^J keep sets
    (each window kept independently with probability p), E[Z | s] = ||Y_s||_1
    and Var[Z | s] = sum_j Y_j^2 (1 - p) / p.  Z is formed by the oracle's own
    combination step of Algorithm 1."""
    import oracle.core as core
    rng = np.random.default_rng(44)
    src, dst, t = synth.random_small_graph(rng, 4, 120, 300)
    motif = ([0, 1, 0], [1, 0, 1])
    delta, c, p = 12, 3, 0.3
    cd = c * delta
    s, recs = core.window_records(src, dst, t, *motif, delta, c, seed=5, p=1.0)
    J = len(recs)
    assert 4 <= J <= 14
    Y = [r["W"] for r in recs]
    assert sum(1 for y in Y if y > 0) >= 3
    EZ = 0.0
    EZ2 = 0.0
    for mask in range(1 << J):
        sel = [dict(r, q=p, kept=True) for i, r in enumerate(recs) if mask >> i & 1]
        z = core.z_from_records(sel, cd)
        kk = bin(mask).count("1")
        pr = p ** kk * (1 - p) ** (J - kk)
        EZ += pr * z
        EZ2 += pr * z * z
    y1 = sum(Y)
    var_want = sum(y * y for y in Y) * (1 - p) / p
    assert abs(EZ - y1) <= 1e-10 * y1
    assert abs((EZ2 - EZ * EZ) - var_want) <= 1e-7 * var_want


# ---------------------------------------------------------------- P7 --------
def test_estimator_unbiased_over_seeds(oracle_mod):
    """Theorem 4.3: E[Z] = C_M.  Over n fixed seeds the sample mean lies within
    4 standard errors of the exact count (deterministic: seeds are fixed)."""
    src, dst, t = synth.chung_lu_hawkes(60, 4000, 2.1, seed=11, horizon=60_000)
    motif = ([0, 1, 2], [1, 2, 0])
    delta, c, p = 900, 4, 0.35
    C = oracle_mod.count_exact(src, dst, t, *motif, delta)
    assert C > 100
    zs = np.array([oracle_mod.estimate(src, dst, t, *motif, delta, c, p, seed) for seed in range(300)])
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    assert abs(zs.mean() - C) <= 4 * se, (zs.mean(), C, se)
    # b shifts average b single-shift estimates with consecutive k
    z3, parts = oracle_mod.estimate(src, dst, t, *motif, delta, c, p, 77, b=3, return_parts=True)
    assert len(parts) == 3 and abs(z3 - sum(parts) / 3) <= 1e-12 * max(1.0, abs(z3))


def test_estimate_p1_small_c_edge_cases(oracle_mod):
    """p = 1 keeps every window; c = 1 still works (an instance spanning the
    whole window width can never fit, Eq. 2 gives it probability 0 of being
    inside); an empty graph estimates 0."""
    rng = np.random.default_rng(3)
    src, dst, t = synth.random_small_graph(rng, 4, 60, 200)
    motif = ([0, 1], [1, 0])
    for c in (1, 2, 5):
        z = oracle_mod.estimate(src, dst, t, *motif, 7, c, 1.0, seed=1)
        s, recs = oracle_mod.window_records(src, dst, t, *motif, 7, c, seed=1, p=1.0)
        assert all(r["kept"] for r in recs)
        assert z == pytest.approx(sum(r["W"] for r in recs), rel=1e-13)
    e = np.zeros(0, np.int32)
    assert oracle_mod.estimate(e, e, np.zeros(0, np.int64), *motif, 7, 3, 0.5, seed=1) == 0.0


# ---------------------------------------------------------------- P4 through the oracle's own steps
def _seed_for_shift(orng, cd, s, k=0):
    """The first seed whose repetition-k shift is s (shift draws are pinned by the
    SplitMix64 known answers; this only searches them)."""
    seed = 0
    while orng.shift(seed, k, cd) != s:
        seed += 1
    return seed


def test_window_weights_hand_worked(oracle_mod):
    """Windows of Eq. 1 and their weights W_j (Eqs. 2-3) on a hand-worked graph,
    through window_records, z_from_records and estimate: an edge on a window's
    last tick a_j + c delta - 1 belongs to the window, an instance straddling a
    boundary belongs to none, and each instance adds c delta / (c delta - Delta)."""
    from fractions import Fraction
    g = json.load(open(os.path.join(GOLDEN, "window_weights.json")))
    src, dst, t = _arr(g["edges"])
    mu = [e[0] for e in g["motif"]]
    mv = [e[1] for e in g["motif"]]
    delta, c = g["delta"], g["c"]
    cd = c * delta
    cnt, hist, _ = oracle_mod.count_exact_hist(src, dst, t, mu, mv, delta)
    assert cnt == g["count"]
    assert {d: int(x) for d, x in enumerate(hist) if x} == {int(k): v for k, v in g["hist"].items()}
    for sh in g["shifts"]:
        seed = _seed_for_shift(oracle_mod.rng, cd, sh["s"])
        s, recs = oracle_mod.window_records(src, dst, t, mu, mv, delta, c, seed, p=1.0)
        assert s == sh["s"]
        assert len(recs) == len(sh["windows"])
        for r, w in zip(recs, sh["windows"]):
            assert (r["j"], r["a"], r["end"], r["lo"], r["hi"], r["count"]) == \
                (w["j"], w["start"], w["end"], w["lo"], w["hi"], w["count"])
            # each term is rounded once to fp64, then summed: within a few ulp of the fraction
            assert r["W"] == pytest.approx(float(Fraction(*w["W"])), rel=1e-14, abs=0.0)
        want1 = float(sum(Fraction(*w["W"]) for w in sh["windows"]))
        assert oracle_mod.estimate(src, dst, t, mu, mv, delta, c, 1.0, seed) == pytest.approx(want1, rel=1e-14, abs=0.0)
        # p = 1/2: Z = sum over kept windows of W_j / q_j (Algorithm 1's combination step)
        p = 0.5
        kept = [oracle_mod.rng.uniform(seed, 0, w["j"]) < p for w in sh["windows"]]
        want = float(sum(Fraction(*w["W"]) / Fraction(1, 2) for w, k in zip(sh["windows"], kept) if k))
        assert oracle_mod.estimate(src, dst, t, mu, mv, delta, c, p, seed) == pytest.approx(want, rel=1e-14, abs=0.0)
        # Algorithm 1 first normalises times to start at 0: translating every timestamp
        # changes no window, count or weight
        s2, recs2 = oracle_mod.window_records(src, dst, t + 1_000_003, mu, mv, delta, c, seed, p=1.0)
        assert s2 == s
        assert [(r["j"], r["a"], r["lo"], r["hi"], r["count"], r["W"]) for r in recs2] == \
            [(r["j"], r["a"], r["lo"], r["hi"], r["count"], r["W"]) for r in recs]


@pytest.mark.parametrize("motif,delta", [(([0, 1, 2], [1, 2, 0]), 9), (([0, 1, 0], [1, 0, 1]), 7),
                                         (([2, 2, 2], [0, 1, 0]), 8)])
def test_lemma41_through_window_records_and_estimate(oracle_mod, motif, delta):
    """Lemma 4.1 driven through the oracle's own Algorithm 1 steps: with every
    window kept (p = 1), summed over all c delta shifts s, (i) the per-window
    duration histograms of window_records give (c delta - Delta) H[Delta]
    exactly (Eq. 2: an instance of duration Delta lies inside a window for
    c delta - Delta shifts), and (ii) the weights sum_j W_j, and the estimates
    themselves, add up to c delta C_M (to 1e-12), i.e. the mean over shifts of
    ||Y_s||_1 is C_M."""
    rng = np.random.default_rng(4100 + delta)
    src, dst, t = synth.random_small_graph(rng, 4, 200, 300)
    for c in (2, 3):
        cd = c * delta
        C, H, _ = oracle_mod.count_exact_hist(src, dst, t, *motif, delta)
        assert C > 0
        tot = np.zeros(delta + 1, np.int64)
        w_sums, z_sums = [], []
        for s in range(-cd + 1, 1):
            seed = _seed_for_shift(oracle_mod.rng, cd, s)
            s_got, recs = oracle_mod.window_records(src, dst, t, *motif, delta, c, seed, p=1.0)
            assert s_got == s
            for r in recs:
                if r["count"]:
                    tot += r["hist"]
            w_sums.append(math.fsum(r["W"] for r in recs))
            z_sums.append(oracle_mod.estimate(src, dst, t, *motif, delta, c, 1.0, seed))
        assert np.array_equal(tot, np.array([(cd - d) * H[d] for d in range(delta + 1)]))
        assert abs(math.fsum(w_sums) - cd * C) <= 1e-12 * cd * C
        assert abs(math.fsum(z_sums) - cd * C) <= 1e-12 * cd * C
