"""bench.py's algorithmic-byte accounting of the matcher kernels (no GPU): k_match is charged
its candidates, range-counted closings and the entries estimates read one by one; k_ride the
entries read for the riders (counted on the exact query they ride on); k_level2 16 bytes per
first edge, with the implementation's 52 bytes per first edge beside it."""
from types import SimpleNamespace

import bench


def _r(first=0, cand=0, last=0, inst=0):
    return {"first_edges": first, "cand_edges": cand, "last_ranges": last, "inst_read": inst}


def test_bytes_split_between_matcher_and_rider_pass():
    qs = [SimpleNamespace(mode=0), SimpleNamespace(mode=1), SimpleNamespace(mode=0)]
    res = [_r(first=100, cand=40, last=30, inst=7), _r(first=50, cand=5, last=0, inst=3), _r()]
    b = bench.kernel_bytes(qs, res)
    assert b["k_match"] == 12 * 45 + 16 * 30 + 8 * 3
    assert b["k_ride"] == 8 * 7
    assert b["k_level2"] == 16 * 150
    assert b["k_level2_impl"] == 52 * 150


def test_bytes_without_riders_are_all_the_matchers():
    qs = [SimpleNamespace(mode=1)] * 2
    res = [_r(first=10, cand=4, last=2, inst=5), _r(first=10, cand=1, last=1, inst=1)]
    b = bench.kernel_bytes(qs, res)
    assert b["k_ride"] == 0
    assert b["k_match"] == 12 * 5 + 16 * 3 + 8 * 6
