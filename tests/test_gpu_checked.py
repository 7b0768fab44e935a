"""The bounds-checked build (libtmotif_checked.so, compiled with TM_CHECKED).

Every index its kernels derive from data is checked against the size of the array it
indexes; a failed check sets a bit of a device error word and redirects the access to
element 0 (never outside the array, never a trap).  Here the checked library runs the
batched paths on small graphs -- exact and estimate queries, estimates riding along,
smaller spans, two-node motifs, a four-edge motif, a prepared batch, the no-allocation
count -- against the CPU oracle, and no check may fire; then its self-test sends one
index past a one-element array through the check and the bit must be set.  It runs in a
child process, so that the checked library is the only one loaded there."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import math, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1810_00980_gb300 import synth, tm
assert tm.LIB_PATH.endswith("libtmotif_checked.so"), tm.LIB_PATH
oracle.core.build()
torch.cuda.set_device(0)

def close(a, b):
    return abs(a - b) <= 1e-12 * max(abs(b), 1e-300) or (a == 0 and b == 0)

def dev(src, dst, t):
    return tm.Graph(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (src, dst, t)))

assert tm.check_status(clear=True) == 0
# tiny graphs with ties, duplicates and self-loops
rng = np.random.default_rng(5)
shapes = [([0, 1], [1, 0]), ([0, 1, 2], [1, 2, 0]), ([2, 2, 2], [0, 1, 0]), ([0, 1, 0], [1, 0, 1]),
          ([0, 1, 2, 3], [1, 2, 3, 0]), ([0, 2, 1], [1, 3, 2])]
for trial in range(12):
    src, dst, t = synth.random_small_graph(rng, int(rng.integers(2, 7)), int(rng.integers(1, 60)), 80,
                                           self_loops=trial % 3 == 0)
    g = dev(src, dst, t)
    for ms, md in shapes:
        mo = tm.Motif(ms, md)
        for delta in (0, 5, 40):
            assert tm.count_exact(g, mo, delta) == oracle.count_exact(src, dst, t, ms, md, delta)
        z = tm.estimate(g, mo, 7, 3, 0.5, trial)
        assert close(z, oracle.estimate(src, dst, t, ms, md, 7, 3, 0.5, trial))
    g.free()
# a bursty graph: one batch with spans and riders of each three-edge motif, two-node and
# four-edge queries, then a prepared batch and the no-allocation count
src, dst, t = synth.chung_lu_hawkes(1500, 60_000, 2.1, seed=9, horizon=2_000_000)
g = dev(src, dst, t)
qs, want = [], []
for name in ("cycle3", "outstar3", "pingpong", "cycle4"):
    ms, md = synth.MOTIFS[name]
    mo = tm.Motif(ms, md)
    for d in (600, 3600):
        qs.append(tm.exact_query(mo, d))
        want.append(("exact", oracle.count_exact(src, dst, t, ms, md, d, threads=8)))
    for (d, c, p, s, b) in ((600, 10, 0.3, 11, 1), (3600, 4, 1.0, 12, 1), (3600, 5, 0.5, 13, 2)):
        qs.append(tm.estimate_query(mo, d, c, p, s, b=b))
        want.append(("est", oracle.estimate(src, dst, t, ms, md, d, c, p, s, b=b, threads=8)))
res = tm.run_batch(g, qs)
for r, (kind, w) in zip(res, want):
    assert r["status"] == 0
    assert (r["count"] == w) if kind == "exact" else close(r["estimate"], w), (r, w)
pb = tm.PreparedBatch(g, qs)
st = torch.cuda.Stream()
pb.launch(st.cuda_stream)
for a, b in zip(pb.results(st.cuda_stream), res):
    assert a["count"] == b["count"] and a["estimate"] == b["estimate"]
pb.free()
import ctypes
out = ctypes.c_int64(-1)
mo = tm.Motif(*synth.MOTIFS["cycle3"])
assert tm.lib().tm_count_exact_noalloc(g.handle, mo.handle, 3600, None, ctypes.byref(out)) == 0
assert out.value == want[1][1]   # the cycle at delta = 3600
torch.cuda.synchronize()
word = tm.check_status(clear=True)
assert word == 0, f"bounds checks fired: {word:#x}"
# the mechanism itself: one index past a one-element array sets the self-test bit
tm.check_selftest()
assert tm.check_status(clear=True) == 64
assert tm.check_status(clear=True) == 0
print("checked ok")
"""


def test_checked_build_runs_clean_and_reports():
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, TMOTIF_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])


def test_ordinary_build_has_no_checks():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_1810_00980_gb300 import tm
    if tm.LIB_PATH.endswith("libtmotif_checked.so"):
        pytest.skip("this process loaded the checked build")
    with pytest.raises(tm.TmError) as e:
        tm.check_status()
    assert e.value.status == tm.TM_EINVAL
