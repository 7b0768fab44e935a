"""tm_count_exact_noalloc: the exact count for callers that may not allocate
device memory while they serve queries (for example because another
allocator owns the GPU's memory, or because allocation can block the device
in latency-critical code).  It must give the same count as tm_count_exact,
call after call, through the C ABI.  This file is collected last so that a
failing run stops only after every other test has run."""
import ctypes

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


def _count_noalloc(tm, g, m, delta, stream):
    out = ctypes.c_int64(-1)
    st = tm.lib().tm_count_exact_noalloc(g.handle, m.handle, int(delta), ctypes.c_void_p(stream),
                                         ctypes.byref(out))
    return st, out.value


def test_noalloc_matches_existing_entry_point_twice(tm):
    import torch
    src, dst, t = synth.chung_lu_hawkes(3000, 200_000, 2.1, seed=77, horizon=5_000_000)
    g = tm.Graph(*(torch.from_numpy(x).cuda() for x in (src, dst, t)))
    stream = torch.cuda.Stream()
    cases = [("cycle3", 3600), ("outstar3", 86400), ("pingpong", 600), ("cycle4", 3600)]
    for name, delta in cases:
        m = tm.Motif(*synth.MOTIFS[name])
        want = tm.count_exact(g, m, delta)
        # two calls in a row: the shared scratch must not carry state between calls
        for _ in range(2):
            st, got = _count_noalloc(tm, g, m, delta, stream.cuda_stream)
            assert st == tm.TM_OK
            assert got == want, (name, delta, got, want)


def test_noalloc_rejects_graphs_beyond_its_scratch(tm):
    n = tm.NOALLOC_MAX_EDGES + 1
    src = np.zeros(n, np.int32)
    dst = np.ones(n, np.int32)
    t = np.arange(n, dtype=np.int64)
    g = tm.Graph(src, dst, t)
    m = tm.Motif([0], [1])
    st, _ = _count_noalloc(tm, g, m, 10, 0)
    assert st == tm.TM_EINVAL
    # at the limit it still counts (every edge is an instance of a one-edge motif)
    g2 = tm.Graph(src[:-1], dst[:-1], t[:-1])
    st, got = _count_noalloc(tm, g2, m, 10, 0)
    assert st == tm.TM_OK and got == n - 1 == tm.count_exact(g2, m, 10)
