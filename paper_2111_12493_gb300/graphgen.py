"""Seeded synthetic graph generators for the k-bisimulation workloads.

This module only draws random graphs. It holds none of the refinement
arithmetic, so both the CPU oracle and the CUDA path can consume its output
without sharing any code of the method itself.

Every generator returns plain numpy arrays:

    n        number of vertices (int)
    src, dst int32 [m]  directed edges src -> dst (multi-edges and self-loops allowed)
    elabel   int32 [m]  edge label
    vlabel   int32 [n]  vertex label; UNTYPED (-1) is an ordinary label of its own

The paper evaluates on LUBM, BSBM and DyLDO crawls (Section 4.1, Section 7
"Experiment 4"). Those datasets are not available here; the generators below
are stand-ins with the size, degree skew and label distributions of the five
workloads the library is measured on:

  uniform_graph        10k vertices / 50k uniform edges, 8 edge labels, 4 vertex labels
  powerlaw_graph       out-degree power law (exponent 2.1), targets preferential by
                       in-degree (copy model), Zipf edge labels, Zipf vertex labels,
                       10% untyped (10M / 100M at full size)
  chain_graph          directed paths plus uniform extra edges (long k-chaining)
  batched_graphs       thousands of independent small graphs (disjoint union)
  update_stream        batches of edge/vertex operations for incremental serving
"""

from __future__ import annotations

import math

import numpy as np

UNTYPED = -1

OP_EDGE_ADD = 0
OP_EDGE_DEL = 1
OP_VERTEX_ADD = 2
OP_VERTEX_DEL = 3


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def zipf_labels(rng: np.random.Generator, count: int, n_values: int, s: float) -> np.ndarray:
    """Draw `count` labels in [0, n_values) with P(r) proportional to (r+1)^-s."""
    w = np.arange(1, n_values + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(count)
    out = np.searchsorted(cdf, u, side="right")
    np.minimum(out, n_values - 1, out=out)
    return out.astype(np.int32)


def _powerlaw_degrees(rng, n: int, m: int, exponent: float, dmax: int, dmin: int = 1) -> np.ndarray:
    """Out-degrees from a floored continuous Pareto on [dmin, dmax], rescaled to sum m.

    Scaling uses stochastic rounding; the residual is fixed by +-1 at random
    vertices, keeping every degree in [dmin, dmax] where possible.
    """
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    m = min(m, n * dmax)                  # no degree sequence can exceed n * dmax
    a = exponent - 1.0
    u = rng.random(n)
    tail = (dmax / dmin) ** (-a)
    x = dmin * (1.0 - u * (1.0 - tail)) ** (-1.0 / a)
    d = np.floor(x)
    d = np.clip(d, dmin, dmax)
    scale = m / d.sum()
    ds = d * scale
    fl = np.floor(ds)
    d = fl + (rng.random(n) < (ds - fl))
    d = np.clip(d, 0, dmax).astype(np.int64)
    resid = int(m - d.sum())
    # fix the residual one unit at a time at random vertices (vectorised in blocks)
    while resid != 0:
        k = min(abs(resid), n)
        idx = rng.choice(n, size=k, replace=False)
        if resid > 0:
            ok = idx[d[idx] < dmax]
            if len(ok) == 0:
                ok = np.flatnonzero(d < dmax)[:k]
            ok = ok[:resid]
            d[ok] += 1
            resid -= len(ok)
        else:
            ok = idx[d[idx] > dmin]
            if len(ok) == 0:
                ok = np.flatnonzero(d > 0)[:k]
            ok = ok[:-resid]
            d[ok] -= 1
            resid += len(ok)
    return d


def _copy_model_targets(rng, n: int, m: int, p_copy: float) -> np.ndarray:
    """Targets for m edges in order: with prob p_copy copy the target of a uniformly
    chosen earlier edge, else pick a uniform vertex (preferential by in-degree)."""
    j = np.arange(m, dtype=np.int64)
    copy = rng.random(m) < p_copy
    copy[0] = False if m > 0 else copy[:0]
    parent = np.where(copy, np.floor(rng.random(m) * j).astype(np.int64), j)
    fresh = rng.integers(0, n, size=m, dtype=np.int64)
    # resolve each edge to the root edge whose target was drawn fresh (pointer jumping)
    while True:
        pp = parent[parent]
        if np.array_equal(pp, parent):
            break
        parent = pp
    return fresh[parent].astype(np.int32)


def uniform_graph(n: int = 10_000, m: int = 50_000, n_elabels: int = 8, n_vlabels: int = 4,
                  seed: int = 1) -> dict:
    """Endpoints uniform at random; labels uniform."""
    rng = _rng(seed)
    src = rng.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    dst = rng.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    elabel = rng.integers(0, n_elabels, size=m, dtype=np.int64).astype(np.int32)
    vlabel = rng.integers(0, n_vlabels, size=n, dtype=np.int64).astype(np.int32)
    return dict(n=n, src=src, dst=dst, elabel=elabel, vlabel=vlabel)


def powerlaw_graph(n: int = 10_000_000, m: int = 100_000_000, exponent: float = 2.1,
                   dmax: int = 1_000_000, n_elabels: int = 1000, elabel_s: float = 1.1,
                   n_vlabels: int = 200, vlabel_s: float = 1.0, untyped_frac: float = 0.1,
                   p_copy: float = 0.8, seed: int = 2) -> dict:
    """Out-degree power law, copy-model targets, Zipf labels, a fraction untyped."""
    rng = _rng(seed)
    dmax = min(dmax, max(1, m))
    deg = _powerlaw_degrees(rng, n, m, exponent, dmax)
    src = np.repeat(np.arange(n, dtype=np.int32), deg)
    order = rng.permutation(m)            # edges take targets in random order
    tgt = _copy_model_targets(rng, n, m, p_copy)
    dst = np.empty(m, dtype=np.int32)
    dst[order] = tgt
    elabel = zipf_labels(rng, m, n_elabels, elabel_s)
    vlabel = zipf_labels(rng, n, n_vlabels, vlabel_s)
    vlabel[rng.random(n) < untyped_frac] = UNTYPED
    return dict(n=n, src=src, dst=dst, elabel=elabel, vlabel=vlabel)


def chain_graph(n_paths: int = 1000, path_len: int = 1000, extra: int = 2_000_000,
                n_elabels: int = 16, n_vlabels: int = 2, seed: int = 3) -> dict:
    """Directed paths (vertex ids path-major) plus uniform random extra edges."""
    rng = _rng(seed)
    n = n_paths * path_len
    base = (np.arange(n_paths, dtype=np.int64) * path_len)[:, None]
    step = np.arange(path_len - 1, dtype=np.int64)[None, :]
    psrc = (base + step).reshape(-1)
    pdst = psrc + 1
    esrc = rng.integers(0, n, size=extra, dtype=np.int64)
    edst = rng.integers(0, n, size=extra, dtype=np.int64)
    src = np.concatenate([psrc, esrc]).astype(np.int32)
    dst = np.concatenate([pdst, edst]).astype(np.int32)
    m = len(src)
    elabel = rng.integers(0, n_elabels, size=m, dtype=np.int64).astype(np.int32)
    vlabel = rng.integers(0, n_vlabels, size=n, dtype=np.int64).astype(np.int32)
    return dict(n=n, src=src, dst=dst, elabel=elabel, vlabel=vlabel)


def batched_graphs(n_graphs: int = 4096, nmin: int = 100, nmax: int = 100_000,
                   mean_deg: float = 5.0, exponent: float = 2.3, n_elabels: int = 64,
                   elabel_s: float = 1.1, n_vlabels: int = 16, seed: int = 4) -> dict:
    """Independent graphs with log-uniform vertex counts; local ids per graph.

    Returns vertex_offsets / edge_offsets (int64 [n_graphs+1]) and local
    src/dst (int32) alongside elabel / vlabel over the union.
    """
    rng = _rng(seed)
    ng = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n_graphs))).astype(np.int64)
    ng = np.maximum(ng, 2)
    srcs, dsts = [], []
    ecount = np.zeros(n_graphs, dtype=np.int64)
    for g in range(n_graphs):
        n = int(ng[g])
        m = int(round(mean_deg * n))
        deg = _powerlaw_degrees(rng, n, m, exponent, dmax=n - 1)
        s = np.repeat(np.arange(n, dtype=np.int32), deg)
        d = rng.integers(0, n, size=len(s), dtype=np.int64).astype(np.int32)
        srcs.append(s)
        dsts.append(d)
        ecount[g] = len(s)
    vo = np.zeros(n_graphs + 1, dtype=np.int64)
    vo[1:] = np.cumsum(ng)
    eo = np.zeros(n_graphs + 1, dtype=np.int64)
    eo[1:] = np.cumsum(ecount)
    src = np.concatenate(srcs) if srcs else np.zeros(0, np.int32)
    dst = np.concatenate(dsts) if dsts else np.zeros(0, np.int32)
    elabel = zipf_labels(rng, len(src), n_elabels, elabel_s)
    vlabel = rng.integers(0, n_vlabels, size=int(vo[-1]), dtype=np.int64).astype(np.int32)
    return dict(n_graphs=n_graphs, vertex_offsets=vo, edge_offsets=eo, src_local=src,
                dst_local=dst, elabel=elabel, vlabel=vlabel)


def batched_union(b: dict) -> dict:
    """Disjoint union of a batched set as one graph with global ids, plus graph ids."""
    vo, eo = b["vertex_offsets"], b["edge_offsets"]
    gid_e = np.repeat(np.arange(b["n_graphs"], dtype=np.int64), np.diff(eo))
    off = vo[:-1][gid_e]
    src = (b["src_local"].astype(np.int64) + off).astype(np.int32)
    dst = (b["dst_local"].astype(np.int64) + off).astype(np.int32)
    gid_v = np.repeat(np.arange(b["n_graphs"], dtype=np.int32), np.diff(vo))
    return dict(n=int(vo[-1]), src=src, dst=dst, elabel=b["elabel"], vlabel=b["vlabel"], graph=gid_v)


def update_stream(base: dict, n_batches: int, min_ops: int = 1000, max_ops: int = 1_000_000,
                  p_add: float = 0.70, p_edel: float = 0.25, n_elabels: int = 1000,
                  elabel_s: float = 1.1, p_copy: float = 0.8, fixed_size: int | None = None,
                  rate_hz: float = 200.0, seed: int = 50) -> list:
    """Batches of operations against `base`, drawn so that they stay valid.

    Each op is a row (kind, src, dst, label) of an int32 [n_ops, 4] array.
    EDGE_ADD draws src uniform among alive vertices and dst by the copy model
    over the current edge targets; EDGE_DEL picks a uniform existing edge;
    VERTEX_DEL a uniform alive vertex. Returns a list of dicts with `ops` and
    the Poisson `arrival_s` time of each batch.
    """
    rng = _rng(seed)
    n = base["n"]
    alive = np.ones(n, dtype=bool)
    # current edge multiset as parallel arrays with a tombstone mask
    src = np.asarray(base["src"]).copy()
    dst = np.asarray(base["dst"]).copy()
    lab = np.asarray(base["elabel"]).copy()
    live = np.ones(len(src), dtype=bool)
    out = []
    t = 0.0
    for _ in range(n_batches):
        if fixed_size is not None:
            size = fixed_size
        else:
            size = int(math.floor(math.exp(rng.uniform(math.log(min_ops), math.log(max_ops)))))
        t += rng.exponential(1.0 / rate_hz)
        kinds = rng.random(size)
        ops = np.zeros((size, 4), dtype=np.int32)
        new_src, new_dst, new_lab = [], [], []
        alive_idx = np.flatnonzero(alive)
        for i in range(size):
            r = kinds[i]
            if r < p_add or len(np.flatnonzero(live)) == 0:
                s = int(alive_idx[rng.integers(0, len(alive_idx))])
                live_idx = np.flatnonzero(live)
                if len(live_idx) > 0 and rng.random() < p_copy:
                    d = int(dst[live_idx[rng.integers(0, len(live_idx))]])
                    if not alive[d]:
                        d = int(alive_idx[rng.integers(0, len(alive_idx))])
                else:
                    d = int(alive_idx[rng.integers(0, len(alive_idx))])
                lb = int(zipf_labels(rng, 1, n_elabels, elabel_s)[0])
                ops[i] = (OP_EDGE_ADD, s, d, lb)
                src = np.append(src, s)
                dst = np.append(dst, d)
                lab = np.append(lab, lb)
                live = np.append(live, True)
            elif r < p_add + p_edel:
                live_idx = np.flatnonzero(live)
                e = int(live_idx[rng.integers(0, len(live_idx))])
                ops[i] = (OP_EDGE_DEL, int(src[e]), int(dst[e]), int(lab[e]))
                live[e] = False
            else:
                v = int(alive_idx[rng.integers(0, len(alive_idx))])
                ops[i] = (OP_VERTEX_DEL, v, 0, 0)
                alive[v] = False
                live &= ~((src == v) | (dst == v))
                alive_idx = np.flatnonzero(alive)
        out.append(dict(ops=ops, arrival_s=t))
    return out


def update_batches(base: dict, n_batches: int, min_ops: int = 1000, max_ops: int = 1_000_000,
                   fixed_size: int | None = None, p_add: float = 0.70, p_edel: float = 0.25,
                   n_elabels: int = 1000, elabel_s: float = 1.1, p_copy: float = 0.8,
                   rate_hz: float = 200.0, seed: int = 50) -> list:
    """Update batches for a large base graph, drawn in bulk so that every batch is valid.

    Per batch: 70% EDGE_ADD (src uniform among live vertices, dst copied from
    the target of a uniform base edge with probability p_copy else uniform live,
    label Zipf(elabel_s)), 25% EDGE_DEL of a uniform base edge (a no-op if it is
    already gone), 5% VERTEX_DEL of distinct live vertices, placed last in the
    batch so that no EDGE_ADD of the batch names a vertex deleted before it.
    Sizes are log-uniform in [min_ops, max_ops] unless fixed_size is given;
    arrival times are Poisson at rate_hz. Returns dicts with `ops` (int32
    [n_ops, 4] rows kind, src, dst, label) and `arrival_s`.
    """
    rng = _rng(seed)
    n = base["n"]
    bsrc, bdst, blab = base["src"], base["dst"], base["elabel"]
    m = len(bsrc)
    alive = np.ones(n, dtype=bool)
    out = []
    t = 0.0
    for _ in range(n_batches):
        size = fixed_size if fixed_size is not None else \
            int(math.floor(math.exp(rng.uniform(math.log(min_ops), math.log(max_ops)))))
        na, nd, nv = rng.multinomial(size, [p_add, p_edel, 1.0 - p_add - p_edel])
        live = np.flatnonzero(alive)
        src = live[rng.integers(0, len(live), na)]
        if m > 0:
            cand = bdst[rng.integers(0, m, na)]
        else:
            cand = live[rng.integers(0, len(live), na)]
        uni = live[rng.integers(0, len(live), na)]
        dst = np.where((rng.random(na) < p_copy) & alive[cand], cand, uni)
        lab = zipf_labels(rng, na, n_elabels, elabel_s)
        adds = np.stack([np.zeros(na, np.int64), src, dst, lab], axis=1)
        if m > 0 and nd > 0:
            e = rng.integers(0, m, nd)
            dels = np.stack([np.ones(nd, np.int64), bsrc[e], bdst[e], blab[e]], axis=1)
        else:
            dels = np.zeros((0, 4), np.int64)
        nv = min(nv, max(0, len(live) - 1))
        vd = rng.choice(live, size=nv, replace=False) if nv > 0 else np.zeros(0, np.int64)
        vdel = np.stack([np.full(nv, OP_VERTEX_DEL, np.int64), vd, np.zeros(nv, np.int64),
                         np.zeros(nv, np.int64)], axis=1)
        body = np.concatenate([adds, dels])
        body = body[rng.permutation(len(body))]
        ops = np.concatenate([body, vdel]).astype(np.int32)
        alive[vd] = False
        t += rng.exponential(1.0 / rate_hz)
        out.append(dict(ops=ops, arrival_s=t))
    return out
