"""Streaming evaluation (tm_stream_run) against tm_run_batch on the whole graph
and against the oracle: each window and each exact first edge is taken in
exactly one chronological segment, so counts and uniform-q estimates are
bit-identical; q_j = r|T_j|/|T| estimates and var_hat agree to rounding."""
import numpy as np
import pytest

from paper_1810_00980_gb300 import synth

pytestmark = pytest.mark.gpu


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


def _queries(tm, names=("cycle3", "outstar3", "pingpong", "cycle4")):
    qs = []
    for i, n in enumerate(names):
        mo = tm.Motif(*synth.MOTIFS[n])
        for d in (600, 3600, 86400):
            qs.append(tm.exact_query(mo, d))
        qs.append(tm.estimate_query(mo, 3600, 10, 0.3, 11 + i, b=3))
        qs.append(tm.estimate_query(mo, 600, 30, 0.8, 21 + i))
        qs.append(tm.estimate_query(mo, 86400, 2, 0.5, 31 + i, b=2))
        qs.append(tm.estimate_query(mo, 3600, 5, 20.0, 41 + i, q_mode=tm.TM_Q_EDGES))
    return qs


def _same(tm, a, b, q):
    assert a["status"] == b["status"] == 0
    assert a["count"] == b["count"]
    assert a["windows"] == b["windows"] and a["windows_kept"] == b["windows_kept"]
    # (work counters are not compared: in a resident batch, queries that ride along with
    # another query's enumeration report none of their own)
    if q.q_mode == tm.TM_Q_EDGES:
        assert abs(a["estimate"] - b["estimate"]) <= 1e-12 * max(abs(b["estimate"]), 1e-300)
    else:
        assert a["estimate"] == b["estimate"]
    assert abs(a["var_hat"] - b["var_hat"]) <= 1e-12 * max(abs(b["var_hat"]), 1e-300)


def test_stream_matches_whole_graph_batch(tm):
    import torch
    src, dst, t = synth.chung_lu_hawkes(3000, 300_000, 2.1, seed=41, horizon=6_000_000)
    n = int(max(src.max(), dst.max())) + 1
    g = tm.Graph(*(torch.from_numpy(x).cuda() for x in (src, dst, t)))
    qs = _queries(tm)
    want = tm.run_batch(g, qs)
    for seg in (7_919, 40_000, 1_000_000):
        got, st = tm.stream_run(src, dst, t, qs, seg, n)
        for a, b, q in zip(got, want, qs):
            _same(tm, a, b, q)
        if seg < len(t):
            assert st["segments"] > 1 and st["edges_copied"] >= len(t)
        else:
            assert st["segments"] == 1
    # pinned host tensors are copied without staging
    got, _ = tm.stream_run(*(torch.from_numpy(x).pin_memory() for x in (src, dst, t)), qs, 50_000, n)
    for a, b, q in zip(got, want, qs):
        _same(tm, a, b, q)
    g.free()


def test_stream_tiny_graphs_against_oracle(tm, orc):
    """Ties, multi-edges and one-timestamp segments (segment_edges = 1)."""
    rng = np.random.default_rng(91)
    for trial in range(25):
        src, dst, t = synth.random_small_graph(rng, 5, int(rng.integers(1, 60)), int(rng.integers(5, 200)),
                                               self_loops=trial % 4 == 0)
        n = int(max(src.max(), dst.max())) + 1
        for ms, md in (synth.MOTIFS["cycle3"], synth.MOTIFS["pingpong"], ([0, 0, 0], [1, 2, 3])):
            mo = tm.Motif(ms, md)
            qs = [tm.exact_query(mo, 7), tm.exact_query(mo, 40), tm.estimate_query(mo, 9, 3, 0.6, trial, b=2)]
            for seg in (1, 3, 17):
                res, _ = tm.stream_run(src, dst, t, qs, seg, n)
                assert res[0]["count"] == orc.count_exact(src, dst, t, ms, md, 7)
                assert res[1]["count"] == orc.count_exact(src, dst, t, ms, md, 40)
                zo = orc.estimate(src, dst, t, ms, md, 9, 3, 0.6, trial, b=2)
                assert abs(res[2]["estimate"] - zo) <= 1e-12 * max(abs(zo), 1e-300)


def test_stream_rejects_and_empty(tm):
    src, dst, t = synth.random_small_graph(np.random.default_rng(3), 4, 30, 50)
    mo = tm.Motif(*synth.MOTIFS["cycle3"])
    qs = [tm.exact_query(mo, 10), tm.Query(mo, -1)]
    res, _ = tm.stream_run(src, dst, t, qs, 8, 4, check=False)
    assert res[1]["status"] == tm.TM_EINVAL and res[0]["status"] == 0
    e = np.zeros(0, np.int32)
    res, st = tm.stream_run(e, e, np.zeros(0, np.int64), [tm.exact_query(mo, 10),
                                                           tm.estimate_query(mo, 10, 2, 0.5, 1)], 8, 4)
    assert res[0]["count"] == 0 and res[1]["estimate"] == 0.0
