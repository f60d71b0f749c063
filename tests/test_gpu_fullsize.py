"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

- power-law 10M / 100M to the fixpoint: every round is checked element by
  element. The oracle recomputes P_0 and, from the device's P_i, the exact
  P_{i+1} (one oracle round each, independent of one another, so they run in
  parallel processes); by induction the device's fixpoint partition is exact.
  The summary graph and block sizes of that partition are checked against a
  numpy sort and count of its edge images.
- chains (1000 paths of 1000 + 2M random edges) to the fixpoint: the whole
  oracle run.
- 4096 batched graphs at k = 3: a seeded sample of the graphs (plus the
  smallest and the largest) against solo oracle runs.
- the resident 5M / 50M graph under update batches at k = 2: the oracle
  applies the same batches and refines the edited graph.
"""

import multiprocessing as mp
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_12493_gb300 import bisim
    return bisim


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ----------------------------------------------------------------------------- oracle workers (spawned)

def _oracle_task(task):
    """Runs in a spawned process: one oracle call on arrays stored as .npy files."""
    import numpy as np

    import oracle as orc
    d, what, pin = task
    load = lambda k: np.load(os.path.join(d, k + ".npy"))
    n = int(load("n")[0])
    src, dst, lab, vl = load("src"), load("dst"), load("elabel"), load("vlabel")
    alive = load("alive") if os.path.exists(os.path.join(d, "alive.npy")) else None
    if what == "label":
        return orc.label_partition(n, vl, alive=alive)
    if what == "round":
        return orc.refine_round(n, src, dst, lab, vl, np.load(pin), alive=alive)
    k = int(what.split(":")[1])
    return orc.refine(n, src, dst, lab, vl, k, alive=alive)[0]


def _save_graph(d, g, alive=None):
    np.save(os.path.join(d, "n.npy"), np.array([g["n"]], np.int64))
    for k in ("src", "dst", "elabel", "vlabel"):
        np.save(os.path.join(d, k + ".npy"), np.ascontiguousarray(g[k], dtype=np.int32))
    if alive is not None:
        np.save(os.path.join(d, "alive.npy"), np.ascontiguousarray(alive, dtype=np.uint8))


def _pool(n):
    return mp.get_context("spawn").Pool(processes=max(1, min(n, os.cpu_count() or 1)))


def _same(got, want, what):
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{what}: {bad.size} vertices differ, first {bad[:5]} got {got[bad[:5]]} want {want[bad[:5]]}"


# ----------------------------------------------------------------------------- workloads

def test_powerlaw_10M_100M_every_round(B):
    g = graphgen.powerlaw_graph(n=10_000_000, m=100_000_000, exponent=2.1, dmax=1_000_000, n_elabels=1000,
                                n_vlabels=200, untyped_frac=0.1, seed=2)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    r, blocks = B.bisim_iterate(ctx, B.FIXPOINT, 10)
    final = B.get_partition(ctx).cpu().numpy()
    # the summary graph and count payload of the fixpoint partition (which the
    # rounds below check against the oracle); numpy's sort stands in for the
    # oracle's set at this size
    es, el, et = (x.cpu().numpy() for x in B.get_summary_edges(ctx))
    sizes = B.get_block_sizes(ctx).cpu().numpy()
    assert np.array_equal(sizes, np.bincount(final, minlength=g["n"]).astype(np.int32))
    sb, tb = final[g["src"]].astype(np.int64), final[g["dst"]].astype(np.int64)
    key = (sb << 32) | (g["elabel"].astype(np.int64) + 2 ** 31)
    order = np.lexsort((tb, key))
    ks, ts = key[order], tb[order]
    head = np.ones(len(ks), bool)
    head[1:] = (ks[1:] != ks[:-1]) | (ts[1:] != ts[:-1])
    assert np.array_equal(es, (ks[head] >> 32).astype(np.int32))
    assert np.array_equal(el, ((ks[head] & 0xffffffff) - 2 ** 31).astype(np.int32))
    assert np.array_equal(et, ts[head].astype(np.int32))
    del sb, tb, key, order, ks, ts, head
    P = []
    for k in range(r + 2):
        B.bisim_iterate(ctx, k, 0)
        P.append(B.get_partition(ctx).cpu().numpy())
    B.summarize_destroy(ctx)
    _same(final, P[r], "fixpoint result vs k = r")
    assert np.array_equal(P[r + 1], P[r]) and len(np.unique(final)) == blocks
    with tempfile.TemporaryDirectory() as d:
        _save_graph(d, g)
        tasks = [(d, "label", None)]
        for i in range(r + 1):
            path = os.path.join(d, f"P{i}.npy")
            np.save(path, P[i])
            tasks.append((d, "round", path))
        with _pool(len(tasks)) as pool:
            want = pool.map(_oracle_task, tasks)
    _same(P[0], want[0], "P_0")
    for i in range(r + 1):
        _same(P[i + 1], want[i + 1], f"round {i} -> {i + 1}")


def test_chain_full_fixpoint(B):
    g = graphgen.chain_graph(seed=3)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    r, _ = B.bisim_iterate(ctx, B.FIXPOINT, 10_000)
    got = B.get_partition(ctx).cpu().numpy()
    B.summarize_destroy(ctx)
    want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], oracle.FIXPOINT, 10_000)
    assert r == wr
    _same(got, want, "chain fixpoint")


def test_batched_4096_sampled_graphs(B):
    """The 4096-graph workload through the union's round kernels (the default),
    a split between them and the persistent kernel, and the persistent kernel
    alone: identical partitions, sampled graphs equal to their oracle runs."""
    b = graphgen.batched_graphs(seed=4)
    vo, eo = b["vertex_offsets"], b["edge_offsets"]
    d = [_dev(vo), _dev(eo), _dev(b["src_local"]), _dev(b["dst_local"]), _dev(b["elabel"]), _dev(b["vlabel"])]
    runs = {}
    for split in (0, 16384, 2**31 - 1):
        ctx = B.summarize_init_batched(*d, options=B.default_options(batch_split=split))
        runs[split] = B.bisim_iterate(ctx, 3, 0), B.get_partition(ctx).cpu().numpy()
        B.summarize_destroy(ctx)
    got = runs[0][1]
    for split, (rb, P) in runs.items():
        assert rb == runs[0][0], split
        _same(P, got, f"batch_split={split}")
    sizes = np.diff(vo)
    rng = np.random.default_rng(44)
    pick = sorted(set(rng.choice(b["n_graphs"], 48, replace=False).tolist()) |
                  {int(np.argmin(sizes)), int(np.argmax(sizes))})
    for gi in pick:
        a, z = int(vo[gi]), int(vo[gi + 1])
        ea, ez = int(eo[gi]), int(eo[gi + 1])
        want, _, _ = oracle.refine(z - a, b["src_local"][ea:ez], b["dst_local"][ea:ez], b["elabel"][ea:ez],
                                   b["vlabel"][a:z], 3)
        _same(got[a:z], want, f"graph {gi} ({z - a} vertices)")


def test_resident_5M_50M_under_update_batches(B):
    g = graphgen.powerlaw_graph(n=5_000_000, m=50_000_000, exponent=2.1, dmax=1_000_000, n_elabels=1000,
                                n_vlabels=200, untyped_frac=0.1, seed=5)
    batches = [b["ops"] for b in graphgen.update_batches(g, 4, seed=50)]
    results = {}
    for mode, flags in (("incremental", 0), ("full", B.FLAG_FULL_RECOMPUTE)):
        ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                                   options=B.default_options(k_incremental=2, flags=flags))
        B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
        for ops in batches:
            B.apply_updates(ctx, _dev(ops))
        results[mode] = B.get_partition(ctx).cpu().numpy()
        B.summarize_destroy(ctx)
    base = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"], src=g["src"], dst=g["dst"],
                elabel=g["elabel"])
    edited, rejected = oracle.apply_batches(base, batches)
    assert rejected == []
    with tempfile.TemporaryDirectory() as d:
        _save_graph(d, edited, alive=edited["alive"])
        with _pool(1) as pool:
            want = pool.map(_oracle_task, [(d, "refine:2", None)])[0]
    _same(results["incremental"], want, "incremental")
    _same(results["full"], want, "full recompute")
