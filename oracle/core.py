"""Oracle implementation -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Citations refer to Liu, Benson & Charikar, "A sampling framework for counting
temporal motifs" (WSDM 2019).
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
from collections import Counter, defaultdict
from fractions import Fraction

import numpy as np

from . import rng

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile enum.c with gcc into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "enum.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_count.restype = ctypes.c_int64
        P = ctypes.c_void_p
        lib.oracle_count.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, P, P, ctypes.c_int32,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, P, P, ctypes.c_int32]
        _lib = lib
    return _lib


def relabel_motif(msrc, mdst):
    """Motif edges (u_i, v_i) with arbitrary integer labels -> labels 0..k-1 in
    order of first appearance (Def. 2.1: the motif is a multigraph plus an edge
    order; node names carry no meaning).  Raises on a self-loop."""
    lab = {}
    out_s, out_d = [], []
    for a, b in zip(list(msrc), list(mdst)):
        a, b = int(a), int(b)
        if a == b:
            raise ValueError("motif self-loop")
        for x in (a, b):
            if x not in lab:
                lab[x] = len(lab)
        out_s.append(lab[a])
        out_d.append(lab[b])
    return np.array(out_s, np.int32), np.array(out_d, np.int32), len(lab)


def _n_nodes(src, dst):
    if len(src) == 0:
        return 0
    return int(max(int(np.max(src)), int(np.max(dst)))) + 1


# --------------------------------------------------------------------------
# Def. 2.2 / 2.3 written out
# --------------------------------------------------------------------------
def count_bruteforce(src, dst, t, msrc, mdst, delta, w_lo=None, w_hi=None):
    """Every l-subset of edges (restricted to times in [w_lo, w_hi]), ordered by
    time; an instance when the times strictly increase, t_l - t_1 <= delta
    (Def. 2.2 item 2) and one node map, injective both ways, sends motif edge i
    onto edge i (Def. 2.2 item 1).  Returns (count, Counter{duration: count})
    -- the count-duration pairs of Def. 2.3.  Exponential: tiny graphs only."""
    mu, mv, _ = relabel_motif(msrc, mdst)
    l = len(mu)
    edges = [(int(s), int(d), int(tt)) for s, d, tt in zip(src, dst, t)
             if (w_lo is None or tt >= w_lo) and (w_hi is None or tt <= w_hi)]
    hist = Counter()
    for combo in itertools.combinations(range(len(edges)), l):
        seq = sorted(combo, key=lambda i: edges[i][2])
        times = [edges[i][2] for i in seq]
        if any(times[x] >= times[x + 1] for x in range(l - 1)):
            continue
        if times[-1] - times[0] > delta:
            continue
        fwd, bwd, ok = {}, {}, True
        for pos, ei in enumerate(seq):
            for mnode, gnode in ((int(mu[pos]), edges[ei][0]), (int(mv[pos]), edges[ei][1])):
                if fwd.setdefault(mnode, gnode) != gnode or bwd.setdefault(gnode, mnode) != mnode:
                    ok = False
        if ok:
            hist[times[-1] - times[0]] += 1
    return sum(hist.values()), hist


# --------------------------------------------------------------------------
# The exact counter A(T', M, delta) (Section 4 intro, Section 5.1), in C
# --------------------------------------------------------------------------
def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def count_exact_hist(src, dst, t, msrc, mdst, delta, w_lo=None, w_hi=None,
                     first=None, threads=1, want_hist=True, n_nodes=None):
    """Exact count of delta-instances among edges with time in [w_lo, w_hi],
    first edge restricted to the index range `first` = (lo, hi).
    Returns (count, hist ndarray of length delta+1 or None, visited)."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    t = np.ascontiguousarray(t, np.int64)
    mu, mv, _ = relabel_motif(msrc, mdst)
    m = len(t)
    n = _n_nodes(src, dst) if n_nodes is None else int(n_nodes)
    lo = -(1 << 62) if w_lo is None else int(w_lo)
    hi = (1 << 62) if w_hi is None else int(w_hi)
    f_lo, f_hi = (0, m) if first is None else (int(first[0]), int(first[1]))
    hist = np.zeros(int(delta) + 1, np.int64) if want_hist else None
    visited = ctypes.c_int64(0)
    c = _load().oracle_count(_ptr(src), _ptr(dst), _ptr(t), m, n, _ptr(mu), _ptr(mv), len(mu),
                             int(delta), lo, hi, f_lo, f_hi, _ptr(hist),
                             ctypes.addressof(visited), int(threads))
    if c < 0:
        raise ValueError(f"oracle_count failed ({c})")
    return int(c), hist, int(visited.value)


def count_exact(src, dst, t, msrc, mdst, delta, threads=1, **kw):
    return count_exact_hist(src, dst, t, msrc, mdst, delta, threads=threads,
                            want_hist=False, **kw)[0]


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
def windows_of_shift(t_max: int, cdelta: int, s: int):
    """Windows of Eq. 1 for shift s: I_j = [s + (j-1) c delta, s + j c delta - 1]
    for j = 1 .. 1 + ceil(t_max / (c delta)) (the loop bound of Algorithm 1,
    timestamps normalised to start at 0).  Returns [(j, start, end)]."""
    J = 1 + (t_max + cdelta - 1) // cdelta
    return [(j, s + (j - 1) * cdelta, s + j * cdelta - 1) for j in range(1, J + 1)]


def _weight_terms(hist, cdelta, q):
    """Terms count_i / ((1 - Delta_i/(c delta)) * q_j) of Algorithm 1, each
    correctly rounded to fp64.  1/(1 - Delta/(c delta)) is evaluated as the same
    rational number c delta / (c delta - Delta), exactly, to avoid the
    cancellation of forming 1 - Delta/(c delta) in floating point."""
    qn, qd = Fraction(q).as_integer_ratio()
    out = []
    nz = np.nonzero(hist)[0]
    for d in nz:
        cnt = int(hist[d])
        out.append((cnt * cdelta * qd) / ((cdelta - int(d)) * qn))
    return out


def window_records(src, dst, t, msrc, mdst, delta, c, seed, k=0, p=None, q=None,
                   threads=1, only_kept=True):
    """Per-window view of one repetition k of Algorithm 1.

    Returns (s, records) where each record is a dict with the window index j,
    start a_j, end, the first and one-past-last edge index of T_j, kept flag,
    exact count, and W_j = w(I_j) = sum over instances in I_j of 1/p_{M'}
    (Eqs. 2-4) as a correctly rounded fp64 sum of correctly rounded terms.
    Timestamps are normalised t' = t - min t first."""
    t = np.asarray(t, np.int64)
    m = len(t)
    cdelta = int(c) * int(delta)
    if m == 0:
        return 0, []
    tn = t - t.min()
    s = rng.shift(seed, k, cdelta)
    recs = []
    for (j, a, e) in windows_of_shift(int(tn.max()), cdelta, s):
        qj = p if q is None else q(j, a, e)
        kept = rng.uniform(seed, k, j) < qj
        if only_kept and not kept:
            continue
        lo = int(np.searchsorted(tn, a, side="left"))
        hi = int(np.searchsorted(tn, e, side="right"))
        rec = dict(j=j, a=a, end=e, lo=lo, hi=hi, kept=bool(kept), q=qj, count=0, W=0.0)
        if kept and hi > lo:
            # T_j = edges with t' in I_j: a contiguous slice of the sorted edge list
            cnt, hist, _ = count_exact_hist(src[lo:hi], dst[lo:hi], tn[lo:hi], msrc, mdst, delta,
                                            threads=threads, n_nodes=_n_nodes(src, dst))
            rec["count"] = cnt
            rec["W"] = math.fsum(_weight_terms(hist, cdelta, 1.0))
            rec["hist"] = hist
        recs.append(rec)
    return s, recs


def z_from_records(recs, cdelta):
    """Combination step of Algorithm 1 for one shift: the sum over kept windows
    of count_i / ((1 - Delta_i/(c delta)) q_j), i.e. Z = sum_j Q_j Y_{s,j} / q_j
    (Eq. 5)."""
    terms = []
    for r in recs:
        if r["kept"] and r["count"]:
            terms += _weight_terms(r["hist"], cdelta, r["q"])
    return math.fsum(terms)


def estimate(src, dst, t, msrc, mdst, delta, c, p, seed, b=1, q=None, threads=1,
             return_parts=False):
    """Algorithm 1 with uniform q_j = p (or q(j, a_j, end_j) if given).

    For k = 1..b: draw the shift s, then for every window j keep it when
    Uniform(0,1) < q_j, count the instances inside T_j exactly with their
    durations, and add count_i / ((1 - Delta_i/(c delta)) q_j) to Z_k.
    Returns the mean of Z_1..Z_b.  Every term is an exactly rounded rational;
    Z_k is their correctly rounded sum (math.fsum)."""
    if int(c) < 1 or int(delta) < 1:
        raise ValueError("need c >= 1 and delta >= 1")
    cdelta = int(c) * int(delta)
    zs = []
    for k in range(int(b)):
        _, recs = window_records(src, dst, t, msrc, mdst, delta, c, seed, k=k, p=p, q=q,
                                 threads=threads)
        zs.append(z_from_records(recs, cdelta))
    z = math.fsum(zs) / len(zs)
    return (z, zs) if return_parts else z


# --------------------------------------------------------------------------
# Algorithm 2 (EX23)
# --------------------------------------------------------------------------
def ex23(src, dst, t, delta):
    """Algorithm 2 for the motif (u,v),(v,u),(u,v), run for both orientations
    of every node pair that exchanges edges.  For each first edge e_i = (u,v),
    walk later edges e_j of the pair while t_j - t_i <= delta: a (v,u) edge
    raises the number N_b of possible middle edges; a (u,v) edge closes N_b
    instances of duration t_j - t_i.  The inner loop starts at j = i + 1 (the
    printed i + 2 would skip a middle edge right after e_i).  Assumes distinct
    timestamps, as the algorithm's input specification does.
    Returns (count, Counter{duration: count})."""
    pairs = defaultdict(list)
    for idx, (s, d, tt) in enumerate(zip(src, dst, t)):
        s, d = int(s), int(d)
        if s == d:
            continue
        key = (min(s, d), max(s, d))
        pairs[key].append((int(tt), idx, (s, d)))
    C = Counter()
    for (a, b), lst in pairs.items():
        lst.sort()
        for (u, v) in ((a, b), (b, a)):
            L = len(lst)
            for i in range(L):
                ti, _, ei = lst[i]
                if ei != (u, v):
                    continue
                nb = 0
                for j in range(i + 1, L):
                    tj, _, ej = lst[j]
                    if tj - ti > delta:
                        break
                    if ej == (v, u):
                        nb += 1
                    else:
                        C[tj - ti] += nb
    C = Counter({d: c for d, c in C.items() if c})
    return sum(C.values()), C
