"""Serving: continuous batching over resident graphs (tm_serve_*).

Each result must be the same alone (a one-query batch) and in the mix (queries
from several threads, several graphs, batches overlapping on two streams)."""
import threading
import time

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
def graphs(tm):
    import torch
    out = []
    for seed, m in ((31, 60_000), (32, 150_000)):
        s, d, t = synth.chung_lu_hawkes(2000, m, 2.1, seed=seed, horizon=3_000_000)
        out.append(tm.Graph(*(torch.from_numpy(x).cuda() for x in (s, d, t))))
    return out


def _mix(tm, rng, n):
    motifs = [tm.Motif(*synth.MOTIFS[k]) for k in ("cycle3", "outstar3", "pingpong", "cycle4")]
    qs = []
    for i in range(n):
        mo = motifs[int(rng.integers(len(motifs)))]
        delta = int(rng.choice([600, 3600, 86400]))
        if rng.random() < 0.4:
            qs.append((int(rng.integers(2)), tm.exact_query(mo, delta)))
        else:
            qs.append((int(rng.integers(2)), tm.estimate_query(mo, delta, int(rng.choice([10, 30])),
                                                                float(rng.choice([0.01, 0.05, 0.1])),
                                                                int(rng.integers(1 << 40)))))
    return motifs, qs


def test_results_alone_equal_results_in_mix(tm, graphs):
    rng = np.random.default_rng(4)
    motifs, qs = _mix(tm, rng, 48)
    alone = [tm.run_batch(graphs[gi], [q])[0] for gi, q in qs]
    with tm.Server(n_streams=2, max_batch=16) as srv:
        gids = [srv.attach(g) for g in graphs]
        tickets = [None] * len(qs)

        def submitter(lo, hi):
            for i in range(lo, hi):
                gi, q = qs[i]
                tickets[i] = srv.submit(gids[gi], q)
                time.sleep(0.0005)

        th = [threading.Thread(target=submitter, args=(k * 12, (k + 1) * 12)) for k in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        got = [srv.wait(tk, 120_000) for tk in tickets]
    for a, g in zip(alone, got):
        assert g is not None
        st, r = g
        assert st == 0
        assert r["count"] == a["count"]
        assert r["estimate"] == a["estimate"]      # bit-identical: exact integer sums on the device
        assert r["windows_kept"] == a["windows_kept"]


def test_poll_cancel_and_admission(tm, graphs):
    mo = tm.Motif(*synth.MOTIFS["cycle3"])
    # a budget too small for any exact query on graph 1: refused at admission
    with tm.Server(mem_budget_bytes=1 << 16, n_streams=1) as srv:
        gid = srv.attach(graphs[1])
        tk = srv.submit(gid, tm.exact_query(mo, 600))
        st, r = srv.wait(tk, 60_000)
        assert st == tm.TM_EADMIT and r["status"] == tm.TM_EADMIT
    with tm.Server(n_streams=1, max_batch=1) as srv:
        gid = srv.attach(graphs[1])
        tks = [srv.submit(gid, tm.exact_query(mo, 86400)) for _ in range(12)]
        c = srv.cancel(tks[-1])
        assert c in (tm.TM_OK, tm.TM_PENDING)
        res = [srv.wait(t, 120_000) for t in tks]
        if c == tm.TM_OK:
            assert res[-1][0] == tm.TM_ECANCELLED
        counts = {r[1]["count"] for r in res[:-1]}
        assert len(counts) == 1
        # a finished ticket is forgotten after it has been read
        st0, _ = srv.poll(tks[0])
        assert st0 == tm.TM_ENOTFOUND


def test_shutdown_drains_queue(tm, graphs):
    mo = tm.Motif(*synth.MOTIFS["pingpong"])
    srv = tm.Server(n_streams=2)
    gid = srv.attach(graphs[0])
    tks = [srv.submit(gid, tm.estimate_query(mo, 3600, 10, 0.1, s)) for s in range(20)]
    srv.close()   # destroy: finishes queued work, then stops
    with pytest.raises(Exception):
        srv.submit(gid, tm.exact_query(mo, 600))


def test_wait_any_returns_every_ticket_once(tm, graphs):
    mo = tm.Motif(*synth.MOTIFS["outstar3"])
    with tm.Server(n_streams=2, max_batch=8) as srv:
        gid = srv.attach(graphs[0])
        want = {srv.submit(gid, tm.estimate_query(mo, 3600, 10, 0.2, s)): s for s in range(30)}
        seen = set()
        while len(seen) < len(want):
            x = srv.wait_any(120_000)
            assert x is not None
            tk, st, r = x
            assert st == tm.TM_OK and tk in want and tk not in seen
            seen.add(tk)
        assert srv.wait_any(50) is None          # nothing left: times out
