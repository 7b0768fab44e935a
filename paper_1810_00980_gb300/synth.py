"""Seeded synthetic temporal graphs.

This module only draws inputs.  It holds none of the motif-counting or
estimator arithmetic, so both the CUDA path and the CPU oracle can be fed
from it without sharing any of the method's code.

The paper measures on ten real temporal networks (Section 5, Table 1: 10^4 to
10^8 nodes, 6*10^4 to 6.4*10^8 edges, one-second resolution, spans of one hour
to ten years).  Those datasets are not available here; the generators below
stand in for them with the same kind of structure:

* ``uniform_graph``      -- uniform endpoints, uniform integer times (a smoke case).
* ``chung_lu_hawkes``    -- directed Chung-Lu endpoints with power-law out/in
  weights and self-exciting (Hawkes) timestamps: Poisson immigrants plus
  Poisson(n) children per event at Exp(mean) delays, where a child either
  repeats its parent's source to a fresh destination or replies along the
  reversed edge.  An optional hub-burst stage makes the heaviest sources emit
  short bursts of edges.
* ``clique_reduction``   -- the temporal graph and star motif of the
  k-Clique reduction in Theorem 3.1, whose instance count is the number of
  k-cliques of the static input graph.

Every array is returned time-sorted (stable by draw order), as the library
expects: ``src`` and ``dst`` int32, ``t`` int64.
"""
from __future__ import annotations

import numpy as np

TWO_YEARS_S = 63_072_000


def _sorted(src, dst, t):
    order = np.argsort(t, kind="stable")
    return (np.ascontiguousarray(src[order], dtype=np.int32),
            np.ascontiguousarray(dst[order], dtype=np.int32),
            np.ascontiguousarray(t[order], dtype=np.int64))


def uniform_graph(n_nodes: int, m_edges: int, t_span: int, seed: int):
    """src, dst ~ U[0, n) with src != dst (dst redrawn), t ~ U{0..t_span-1}."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n_nodes, m_edges, dtype=np.int64)
    dst = rng.integers(0, n_nodes, m_edges, dtype=np.int64)
    bad = src == dst
    while bad.any():
        dst[bad] = rng.integers(0, n_nodes, int(bad.sum()), dtype=np.int64)
        bad = src == dst
    t = rng.integers(0, t_span, m_edges, dtype=np.int64)
    return _sorted(src, dst, t)


def random_small_graph(rng: np.random.Generator, n_nodes: int, m_edges: int,
                       t_span: int, self_loops: bool = False):
    """Tiny graphs for exhaustive checks: repeated pairs, equal timestamps and
    (optionally) self-loops all occur often."""
    src = rng.integers(0, n_nodes, m_edges, dtype=np.int64)
    dst = rng.integers(0, n_nodes, m_edges, dtype=np.int64)
    if not self_loops:
        bad = src == dst
        dst[bad] = (dst[bad] + 1 + rng.integers(0, max(n_nodes - 1, 1), int(bad.sum()))) % n_nodes
    t = rng.integers(0, t_span, m_edges, dtype=np.int64)
    return _sorted(src, dst, t)


def _power_weights(n: int, gamma: float, i0: float, cap_frac: float | None):
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))
    w /= w.sum()
    if cap_frac is not None:
        # Cap the heaviest weights (to bound the maximum expected degree) and
        # renormalise; iterate because renormalising raises the others.
        for _ in range(50):
            over = w > cap_frac
            if not over.any():
                break
            w[over] = cap_frac
            w /= w.sum()
    return w


def _draw(rng, cdf, k):
    u = rng.random(k)
    idx = np.searchsorted(cdf, u, side="right")
    return np.minimum(idx, len(cdf) - 1).astype(np.int64)


def chung_lu_hawkes(n_nodes: int, m_edges: int, gamma: float, seed: int,
                    horizon: int = TWO_YEARS_S, branching: float = 0.5,
                    kernel_mean_s: float = 60.0, i0: float = 1.0,
                    max_degree: int | None = None,
                    hub_bursts: int = 0, burst_max: int = 10_000,
                    burst_window_s: float = 60.0):
    """Directed Chung-Lu endpoints with Hawkes-process timestamps.

    Out- and in-weights are ``(i + i0)^(-1/(gamma-1))`` over independent random
    node permutations.  Immigrant events form a Poisson process of rate
    ``(1 - branching) * m / horizon`` (so the expected total is about m);
    every event has Poisson(branching) children at Exp(kernel_mean_s) delays.
    A child repeats the parent's source with a fresh destination (prob. 1/2)
    or replies along the reversed edge (prob. 1/2).  Events past the horizon
    are dropped; the earliest ``m_edges`` events are kept.  ``hub_bursts``
    extra bursts (each up to ``burst_max`` edges within ``burst_window_s``)
    are emitted by the heaviest sources and replace the latest events so that
    exactly ``m_edges`` remain.
    """
    rng = np.random.default_rng(seed)
    cap = None if max_degree is None else max_degree / float(m_edges)
    w_out = _power_weights(n_nodes, gamma, i0, cap)
    w_in = _power_weights(n_nodes, gamma, i0, cap)
    perm_out = rng.permutation(n_nodes)
    perm_in = rng.permutation(n_nodes)
    cdf_out = np.cumsum(w_out)
    cdf_in = np.cumsum(w_in)
    cdf_out /= cdf_out[-1]
    cdf_in /= cdf_in[-1]

    def draw_src(k):
        return perm_out[_draw(rng, cdf_out, k)]

    def draw_dst(k):
        return perm_in[_draw(rng, cdf_in, k)]

    def fix_loops(s, d):
        bad = s == d
        while bad.any():
            d[bad] = draw_dst(int(bad.sum()))
            bad = s == d
        return d

    srcs, dsts, ts = [], [], []
    total = 0
    target = int(m_edges * 1.03) + 64
    while total < m_edges:
        n_imm = rng.poisson((1.0 - branching) * target)
        t_par = rng.random(n_imm) * horizon
        s_par = draw_src(n_imm)
        d_par = fix_loops(s_par, draw_dst(n_imm))
        gen_s, gen_d, gen_t = [s_par], [d_par], [t_par]
        while len(t_par):
            kids = rng.poisson(branching, len(t_par))
            n_k = int(kids.sum())
            if n_k == 0:
                break
            rep = np.repeat(np.arange(len(t_par)), kids)
            t_c = t_par[rep] + rng.exponential(kernel_mean_s, n_k)
            reply = rng.random(n_k) < 0.5
            s_c = np.where(reply, d_par[rep], s_par[rep])
            d_c = np.where(reply, s_par[rep], draw_dst(n_k))
            d_c = fix_loops(s_c, d_c)
            keep = t_c < horizon
            t_par, s_par, d_par = t_c[keep], s_c[keep], d_c[keep]
            gen_s.append(s_par)
            gen_d.append(d_par)
            gen_t.append(t_par)
        s_all = np.concatenate(gen_s)
        d_all = np.concatenate(gen_d)
        t_all = np.concatenate(gen_t)
        srcs.append(s_all)
        dsts.append(d_all)
        ts.append(t_all)
        total += len(t_all)
        target = max(m_edges - total, 0) + 64
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    t = np.floor(np.concatenate(ts)).astype(np.int64)

    if hub_bursts > 0:
        hubs = perm_out[np.argsort(-w_out)[: max(1, min(hub_bursts, 64))]]
        bs, bd, bt = [], [], []
        for b in range(hub_bursts):
            size = int(rng.integers(burst_max // 2, burst_max + 1))
            h = hubs[b % len(hubs)]
            start = rng.random() * (horizon - burst_window_s)
            bt.append(np.floor(start + rng.random(size) * burst_window_s).astype(np.int64))
            bs.append(np.full(size, h, dtype=np.int64))
            bd.append(fix_loops(np.full(size, h, dtype=np.int64), draw_dst(size)))
        n_b = sum(len(x) for x in bt)
        keep_first = max(m_edges - n_b, 0)
        order = np.argsort(t, kind="stable")[:keep_first]
        src = np.concatenate([src[order], *bs])[:m_edges]
        dst = np.concatenate([dst[order], *bd])[:m_edges]
        t = np.concatenate([t[order], *bt])[:m_edges]
        return _sorted(src, dst, t)

    order = np.argsort(t, kind="stable")[:m_edges]
    return _sorted(src[order], dst[order], t[order])


def clique_reduction(n: int, edges, k: int):
    """Temporal graph T and star motif S of the k-Clique reduction (Theorem 3.1).

    Static graph nodes are 1..n and the centre is node 0.  For each undirected
    edge {u, v}: forward edges (0, u) at time (v-1)(n+2)+u+1 and (0, v) at
    time (u-1)(n+2)+v+1.  For each node u: backward edges (u, 0) at the first
    and last time of block u, (u-1)(n+2)+1 and u(n+2).  The motif's leaves
    1..k come in order; leaf i contributes (i->0), then (0->j) for every other
    leaf j in increasing order, then (i->0) again.  With an unbounded time
    span the number of instances equals the number of k-cliques.

    Returns (src, dst, t, motif_src, motif_dst, delta).
    """
    s, d, t = [], [], []
    for (u, v) in edges:
        s += [0, 0]
        d += [u, v]
        t += [(v - 1) * (n + 2) + u + 1, (u - 1) * (n + 2) + v + 1]
    for u in range(1, n + 1):
        s += [u, u]
        d += [0, 0]
        t += [(u - 1) * (n + 2) + 1, u * (n + 2)]
    ms, md = [], []
    for i in range(1, k + 1):
        ms.append(i); md.append(0)
        for j in range(1, k + 1):
            if j != i:
                ms.append(0); md.append(j)
        ms.append(i); md.append(0)
    src, dst, tt = _sorted(np.array(s, np.int64), np.array(d, np.int64), np.array(t, np.int64))
    delta = int(n * n + 2 * n)
    return src, dst, tt, np.array(ms, np.int32), np.array(md, np.int32), delta


# Workloads with the sizes of the configurations this library is measured on.
def uniform_1k_graph(seed: int = 1):
    """N=1,000, M=20,000, uniform endpoints, t ~ U{0..999,999}."""
    return uniform_graph(1_000, 20_000, 1_000_000, seed)


def bursty_100k_10m_graph(seed: int = 2, m_edges: int = 10_000_000, n_nodes: int = 100_000):
    """Chung-Lu (exponent 2.1) + Hawkes times over two years; N=1e5, M=1e7."""
    return chung_lu_hawkes(n_nodes, m_edges, 2.1, seed)


def bursty_1m_100m_graph(seed: int = 3, m_edges: int = 100_000_000, n_nodes: int = 1_000_000):
    """As bursty_100k_10m_graph with exponent 2.0; N=1e6, M=1e8."""
    return chung_lu_hawkes(n_nodes, m_edges, 2.0, seed)


# Motifs used by the workloads, as ordered (src, dst) label lists.
MOTIFS = {
    "cycle3": ([0, 1, 2], [1, 2, 0]),          # a->b, b->c, c->a
    "outstar3": ([2, 2, 2], [0, 1, 0]),        # c->a, c->b, c->a
    "pingpong": ([0, 1, 0], [1, 0, 1]),        # a->b, b->a, a->b
    "cycle4": ([0, 1, 2, 3], [1, 2, 3, 0]),    # a->b, b->c, c->d, d->a
}


def chung_lu_hawkes_gpu(n_nodes: int, m_edges: int, gamma: float, seed: int,
                        horizon: int = TWO_YEARS_S, branching: float = 0.5,
                        kernel_mean_s: float = 60.0, i0: float = 1.0,
                        max_degree: int | None = None, hub_bursts: int = 0,
                        burst_max: int = 10_000, burst_window_s: float = 60.0,
                        device: str = "cuda"):
    """The same recipe as chung_lu_hawkes, drawn with torch on a CUDA device
    (seeded torch generator) for graphs too large to draw in numpy: returns
    time-sorted (src int32, dst int32, t int64) device tensors.  Its random
    stream differs from the numpy generator's."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    cap = None if max_degree is None else max_degree / float(m_edges)
    w = _power_weights(n_nodes, gamma, i0, cap)
    cdf = torch.from_numpy(np.cumsum(w) / np.sum(w)).to(device)
    perm_out = torch.randperm(n_nodes, generator=gen, device=device).to(torch.int32)
    perm_in = torch.randperm(n_nodes, generator=gen, device=device).to(torch.int32)

    def draw(perm, k):
        u = torch.rand(k, generator=gen, device=device, dtype=torch.float64)
        idx = torch.searchsorted(cdf, u, right=True).clamp_(max=n_nodes - 1)
        return perm[idx]

    def fix_loops(s, d):
        bad = s == d
        nb = int(bad.sum())
        while nb:
            d[bad] = draw(perm_in, nb)
            bad = s == d
            nb = int(bad.sum())
        return d

    n_b_total = 0
    bursts = []
    if hub_bursts > 0:
        hubs = perm_out[torch.from_numpy(np.argsort(-w)[: max(1, min(hub_bursts, 64))].copy()).to(device)]
        rs = np.random.default_rng(seed)
        for b in range(hub_bursts):
            size = int(rs.integers(burst_max // 2, burst_max + 1))
            start = rs.random() * (horizon - burst_window_s)
            bt = torch.floor(start + torch.rand(size, generator=gen, device=device, dtype=torch.float64)
                             * burst_window_s)
            bs = torch.full((size,), int(hubs[b % len(hubs)]), dtype=torch.int32, device=device)
            bd = fix_loops(bs, draw(perm_in, size))
            bursts.append((bs, bd, bt))
            n_b_total += size
    m_base = max(m_edges - n_b_total, 0)

    srcs, dsts, ts = [], [], []
    total = 0
    target = int(m_base * 1.03) + 64
    rs = np.random.default_rng(seed + 1)
    while total < m_base:
        n_imm = int(rs.poisson((1.0 - branching) * target))
        t_par = torch.rand(n_imm, generator=gen, device=device, dtype=torch.float64) * horizon
        s_par = draw(perm_out, n_imm)
        d_par = fix_loops(s_par, draw(perm_in, n_imm))
        gs_, gd_, gt_ = [s_par], [d_par], [t_par]
        while t_par.numel():
            rate = torch.full((t_par.numel(),), branching, device=device, dtype=torch.float64)
            kids = torch.poisson(rate, generator=gen).to(torch.int64)
            n_k = int(kids.sum())
            if n_k == 0:
                break
            rep = torch.repeat_interleave(torch.arange(t_par.numel(), device=device), kids)
            delay = torch.empty(n_k, device=device, dtype=torch.float64).exponential_(1.0 / kernel_mean_s,
                                                                                    generator=gen)
            t_c = t_par[rep] + delay
            reply = torch.rand(n_k, generator=gen, device=device) < 0.5
            s_c = torch.where(reply, d_par[rep], s_par[rep])
            d_c = torch.where(reply, s_par[rep], draw(perm_in, n_k))
            d_c = fix_loops(s_c, d_c)
            keep = t_c < horizon
            t_par, s_par, d_par = t_c[keep], s_c[keep], d_c[keep]
            gs_.append(s_par)
            gd_.append(d_par)
            gt_.append(t_par)
        s_all, d_all, t_all = torch.cat(gs_), torch.cat(gd_), torch.cat(gt_)
        del gs_, gd_, gt_
        srcs.append(s_all)
        dsts.append(d_all)
        ts.append(t_all)
        total += t_all.numel()
        target = max(m_base - total, 0) + 64
    t = torch.floor(torch.cat(ts)).to(torch.int64)
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts, ts
    # earliest m_base background events, then the bursts, all sorted by time (stable)
    order = torch.sort(t, stable=True).indices[:m_base]
    src, dst, t = src[order], dst[order], t[order]
    del order
    if bursts:
        src = torch.cat([src] + [b[0] for b in bursts])
        dst = torch.cat([dst] + [b[1] for b in bursts])
        t = torch.cat([t] + [b[2].to(torch.int64) for b in bursts])
        order = torch.sort(t, stable=True).indices
        src, dst, t = src[order], dst[order], t[order]
        del order
    src, dst, t = src.contiguous(), dst.contiguous(), t.contiguous()
    torch.cuda.empty_cache()   # hand the generator's scratch back before the graph is built
    return src, dst, t


def hub_bursty_10m_1b_graph_gpu(seed: int = 5, m_edges: int = 1_000_000_000, n_nodes: int = 10_000_000,
                      device: str = "cuda"):
    """N=1e7, M=1e9, Chung-Lu exponent 1.8 with the maximum expected degree
    capped at 5e6, Hawkes times over two years, and 1,000 hub bursts of up to
    1e4 edges within 60 s; drawn on the GPU."""
    return chung_lu_hawkes_gpu(n_nodes, m_edges, 1.8, seed, max_degree=5_000_000, hub_bursts=1000,
                               burst_max=10_000, device=device)
