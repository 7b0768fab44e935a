"""tm_count_exact_noalloc: the exact count for callers that may not allocate
device memory while they serve queries (for example because another
allocator owns the GPU's memory, or because allocation can block the device
in latency-critical code).  It must give the same count as tm_count_exact and
as the CPU oracle, call after call, through the C ABI, and it must not touch
the device's stream-ordered memory pool.  This file is collected last so that
a failing run stops only after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1810_00980_gb300 import synth

pytestmark = pytest.mark.gpu

# cudaMemPoolAttr values of the CUDA runtime API
_POOL_USED_CURRENT = 7
_POOL_USED_HIGH = 8


@pytest.fixture(scope="module")
def tm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_1810_00980_gb300 import tm as _tm
    _tm.lib()
    return _tm


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.core.build()
    return oracle


def _count_noalloc(tm, g, m, delta, stream):
    out = ctypes.c_int64(-1)
    st = tm.lib().tm_count_exact_noalloc(g.handle, m.handle, int(delta), ctypes.c_void_p(stream),
                                         ctypes.byref(out))
    return st, out.value


class _DefaultPool:
    """The current device's default stream-ordered memory pool, read through the CUDA
    runtime the library itself loaded (cudaMallocAsync draws from it)."""

    def __init__(self):
        import torch
        self.rt = ctypes.CDLL("libcudart.so.13")   # already loaded: resolved by its soname
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), torch.cuda.current_device()) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        # setting the high watermark (to 0) resets it to the current use
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, _POOL_USED_HIGH, ctypes.byref(v)) == 0


def _check_graph(tm, orc, src, dst, t, cases, stream):
    import torch
    g = tm.Graph(*(torch.from_numpy(x).cuda() for x in (src, dst, t)))
    pool = _DefaultPool()
    for name, delta in cases:
        ms, md = synth.MOTIFS[name]
        m = tm.Motif(ms, md)
        want = orc.count_exact(src, dst, t, ms, md, delta, threads=8)
        assert tm.count_exact(g, m, delta) == want, (name, delta)
        torch.cuda.synchronize()
        used0 = pool.get(_POOL_USED_CURRENT)
        pool.reset_high()
        # two calls in a row: the shared scratch must not carry state between calls
        for _ in range(2):
            st, got = _count_noalloc(tm, g, m, delta, stream.cuda_stream)
            assert st == tm.TM_OK
            assert got == want, (name, delta, got, want)
        # no stream-ordered allocation, not even one freed again inside the call
        assert pool.get(_POOL_USED_HIGH) == used0 == pool.get(_POOL_USED_CURRENT)
    return g


def test_noalloc_matches_oracle_and_existing_entry_point_twice(tm, orc):
    import torch
    src, dst, t = synth.chung_lu_hawkes(3000, 200_000, 2.1, seed=77, horizon=5_000_000)
    stream = torch.cuda.Stream()
    cases = [("cycle3", 3600), ("outstar3", 86400), ("pingpong", 600), ("cycle4", 3600)]
    g = _check_graph(tm, orc, src, dst, t, cases, stream)
    assert g.info().t_max < 2 ** 31   # 32-bit time arrays


def test_noalloc_64_bit_times(tm, orc):
    """A graph whose normalised times need 64 bits (one edge 3e9 s after the rest):
    the 64-bit-time instantiation gives the same counts."""
    import torch
    src, dst, t = synth.chung_lu_hawkes(2000, 100_000, 2.1, seed=78, horizon=3_000_000)
    src = np.append(src, np.int32(0))
    dst = np.append(dst, np.int32(1))
    t = np.append(t, np.int64(t.max() + 3_000_000_000))
    stream = torch.cuda.Stream()
    g = _check_graph(tm, orc, src, dst, t, [("cycle3", 3600), ("outstar3", 600), ("cycle4", 86400)], stream)
    assert g.info().t_max >= 2 ** 31


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
