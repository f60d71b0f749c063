"""The summary graph and its count payload (get_summary_edges, get_block_sizes)
against the oracle.

Section 2.6 defines the summary graph (one vertex per block, an l-labelled
edge between the blocks of the endpoints of every l-edge, parallel edges of
one label collapsed); Section 3.1 the count payload (vertices per block).
Both sides compute them from the same partition, which is itself checked
against the oracle, so the triples and counts must match exactly.
"""

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen
from refcheck import edges_to_arrays, parse_golden

pytestmark = pytest.mark.gpu


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


def _gpu_summary(B, ctx):
    s, l, t = (x.cpu().numpy() for x in B.get_summary_edges(ctx))
    return list(zip(s.tolist(), l.tolist(), t.tolist()))


def _check(B, ctx, src, dst, elabel, P):
    got_P = B.get_partition(ctx).cpu().numpy()
    assert np.array_equal(got_P, P)
    assert _gpu_summary(B, ctx) == oracle.summary_edges(src, dst, elabel, P)
    assert B.get_block_sizes(ctx).cpu().numpy().tolist() == oracle.block_sizes(P).tolist()


def test_summary_of_the_worked_example(B):
    gf = parse_golden("fig3_worked_example.txt")
    s, d, l = edges_to_arrays(gf["edges"])
    vl = np.array(gf["vlabel"]["L"], np.int32)
    ctx = B.summarize_init_coo(gf["n"], _dev(s), _dev(d), _dev(l), _dev(vl))
    B.bisim_iterate(ctx, 2, 0)
    assert _gpu_summary(B, ctx) == gf["summary"][2]
    assert B.get_block_sizes(ctx).cpu().numpy().tolist() == gf["sizes"][2].tolist()
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("k", [0, 1, 2, -1])
def test_uniform_graph_every_k(B, k):
    g = graphgen.uniform_graph(seed=1)
    # signed labels exercise the label order of the output
    lab = (g["elabel"] - 4).astype(np.int32)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(lab), _dev(g["vlabel"]))
    B.bisim_iterate(ctx, k, 10)
    P, _, _ = oracle.refine(g["n"], g["src"], g["dst"], lab, g["vlabel"], k, 10)
    _check(B, ctx, g["src"], g["dst"], lab, P)
    B.summarize_destroy(ctx)


def test_powerlaw_graph_with_hubs_and_dead_vertices(B):
    g = graphgen.powerlaw_graph(n=100_000, m=1_000_000, dmax=50_000, n_elabels=40, n_vlabels=6, seed=31)
    alive = (np.random.default_rng(5).random(g["n"]) > 0.05).astype(np.uint8)
    keep = alive[g["src"]].astype(bool) & alive[g["dst"]].astype(bool)
    src, dst, lab = g["src"][keep], g["dst"][keep], g["elabel"][keep]
    ctx = B.summarize_init_coo(g["n"], _dev(src), _dev(dst), _dev(lab), _dev(g["vlabel"]), alive=_dev(alive))
    for k in (1, -1):
        B.bisim_iterate(ctx, k, 10)
        P, _, _ = oracle.refine(g["n"], src, dst, lab, g["vlabel"], k, 10, alive=alive)
        _check(B, ctx, src, dst, lab, P)
    B.summarize_destroy(ctx)


def test_batched_graphs_report_union_ids(B):
    b = graphgen.batched_graphs(n_graphs=40, nmin=20, nmax=3000, seed=12)
    ctx = B.summarize_init_batched(*(_dev(b[x]) for x in ("vertex_offsets", "edge_offsets", "src_local",
                                                           "dst_local", "elabel", "vlabel")))
    B.bisim_iterate(ctx, 3, 0)
    u = graphgen.batched_union(b)
    P, _, _ = oracle.refine(u["n"], u["src"], u["dst"], u["elabel"], u["vlabel"], 3, graph=u["graph"])
    assert _gpu_summary(B, ctx) == oracle.summary_edges(u["src"], u["dst"], u["elabel"], P)
    assert B.get_block_sizes(ctx).cpu().numpy().tolist() == oracle.block_sizes(P).tolist()
    B.summarize_destroy(ctx)


def test_summary_follows_update_batches(B):
    from test_gpu_updates import random_batch
    rng = np.random.default_rng(9)
    g = graphgen.uniform_graph(n=400, m=1600, n_elabels=3, n_vlabels=3, seed=41)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=2))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    for _ in range(6):
        ops = random_batch(rng, state, int(rng.integers(5, 80)))
        try:
            new_state = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = new_state
        P, _, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"], 2,
                                alive=state["alive"])
        _check(B, ctx, state["src"], state["dst"], state["elabel"], P)
    B.summarize_destroy(ctx)


def test_host_outputs_and_capacity(B):
    import ctypes
    import torch
    g = graphgen.uniform_graph(n=2000, m=9000, n_elabels=3, n_vlabels=2, seed=13)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    B.bisim_iterate(ctx, 1, 0)
    P, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], 1)
    want = oracle.summary_edges(g["src"], g["dst"], g["elabel"], P)
    sizes = torch.empty(g["n"], dtype=torch.int32).pin_memory()
    B.get_block_sizes(ctx, out=sizes)
    assert sizes.numpy().tolist() == oracle.block_sizes(P).tolist()
    # capacity 0 sizes the output; a short capacity writes a prefix; host arrays work
    count = ctypes.c_int64()
    assert B._lib.get_summary_edges(ctx.ptr, None, None, None, 0, ctypes.byref(count), None) == 0
    assert count.value == len(want)
    cap = len(want) // 2
    outs = [torch.empty(cap, dtype=torch.int32).pin_memory() for _ in range(3)]
    assert B._lib.get_summary_edges(ctx.ptr, *[ctypes.c_void_p(o.data_ptr()) for o in outs], cap,
                                    ctypes.byref(count), None) == 0
    assert count.value == len(want)
    assert list(zip(*(o.numpy().tolist() for o in outs))) == want[:cap]
    B.summarize_destroy(ctx)
