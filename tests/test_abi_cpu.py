"""CPU checks of the C ABI: the CUDA library builds for sm_103a, loads without
a GPU, exports every function include/tm.h declares, and the binding's
structs have the C layout.  No compute calls."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tm.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_00980_gb300 import tm
    return tm


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tm_graph_load", "tm_motif_compile", "tm_count_exact", "tm_estimate",
                     "tm_estimate_windows", "tm_run_batch", "tm_serve_submit", "tm_serve_poll"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    L = built.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # and the binding covers them all
    assert set(_declared_functions()) <= set(built._SIGS)


def test_nm_shows_exports(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (tm_\w+)", out))
    assert set(_declared_functions()) <= exported


def test_struct_layouts_match_c(built, tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tm.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    'sizeof(tm_graph_info), sizeof(tm_window_rec), sizeof(tm_query), sizeof(tm_result),'
                    'sizeof(tm_tuning), sizeof(tm_serve_cfg), offsetof(tm_result, var_hat),'
                    'offsetof(tm_profile, launches), sizeof(tm_profile),'
                    'offsetof(tm_query, q_mode), sizeof(tm_stream_stats),'
                    'offsetof(tm_stream_stats, copy_wait_ms));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    import ctypes
    tm = built
    assert vals == [ctypes.sizeof(tm.GraphInfo), ctypes.sizeof(tm.WindowRec), ctypes.sizeof(tm.QueryC),
                    ctypes.sizeof(tm.ResultC), ctypes.sizeof(tm.TuningC), ctypes.sizeof(tm.ServeCfg),
                    tm.ResultC.var_hat.offset, tm.ProfileC.launches.offset, ctypes.sizeof(tm.ProfileC),
                    tm.QueryC.q_mode.offset,
                    ctypes.sizeof(tm.StreamStatsC), tm.StreamStatsC.copy_wait_ms.offset]


def test_stream_run_validates_on_the_host(built):
    """tm_stream_run's argument checks run before any device call."""
    import numpy as np
    tm = built
    mo = tm.Motif([0, 1, 2], [1, 2, 0])
    s = np.array([0, 1, 2], np.int32)
    d = np.array([1, 2, 0], np.int32)
    with pytest.raises(tm.TmError) as e:
        tm.stream_run(s, d, np.array([5, 3, 9], np.int64), [tm.exact_query(mo, 10)], 2, 3)
    assert e.value.status == tm.TM_EUNSORTED
    for seg, n in ((0, 3), (2, 0)):
        with pytest.raises(tm.TmError) as e:
            tm.stream_run(s, d, np.array([1, 2, 3], np.int64), [tm.exact_query(mo, 10)], seg, n)
        assert e.value.status == tm.TM_EINVAL
    res, st = tm.stream_run(s, d, np.array([1, 2, 3], np.int64), [], 2, 3)
    assert res == [] and st["segments"] == 0


def test_strerror_without_gpu(built):
    L = built.lib()
    assert L.tm_strerror(0) == b"ok"
    assert L.tm_strerror(built.TM_EUNSORTED) == b"timestamps not sorted"
    assert L.tm_version().startswith(b"libtmotif")


def test_motif_compile_rejects_bad_motifs(built):
    """Host-only validation (Def. 2.1: motif edges join two distinct nodes)."""
    tm = built
    with pytest.raises(tm.TmError) as e:
        tm.Motif([0, 1], [1, 1])
    assert e.value.status == tm.TM_EINVAL
    with pytest.raises(tm.TmError):
        tm.Motif([], [])
    with pytest.raises(tm.TmError):
        tm.Motif(list(range(9)), list(range(1, 10)))   # l > TM_L_MAX
    m = tm.Motif([5, 7, 9], [7, 9, 5])
    assert m.l == 3


def test_product_has_no_oracle_dependency():
    """The library package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_1810_00980_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower() or f == "synth.py", f


def test_ride_capacity_is_checked_on_the_host(built):
    """tm_set_ride_capacity takes 1 .. 2^36 records and rejects the rest (no device call)."""
    tm = built
    for bad in (0, -5, (1 << 36) + 1):
        with pytest.raises(tm.TmError) as e:
            tm.set_ride_capacity(bad)
        assert e.value.status == tm.TM_EINVAL
    tm.set_ride_capacity(1 << 23)   # the default
