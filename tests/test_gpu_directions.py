"""Backward and forward-backward bisimulation and label-filtered edges on the
GPU, against the oracle's direction modes (Section 2.5: forward bisimulation
compares outgoing edges, backward bisimulation incoming ones; Section 2.4.2:
label-parameterized edge relations).

Each mode is checked for the three ways of creating a context (edge list,
CSR, batched graphs), under update batches, and for the summary graph, which
reports the caller's edges and labels whatever the mode.
"""

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen

pytestmark = pytest.mark.gpu

MODES = [("backward", 1), ("both", 2)]


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


def _csr(g):
    order = np.argsort(g["src"], kind="stable")
    rp = np.zeros(g["n"] + 1, np.int64)
    rp[1:] = np.cumsum(np.bincount(g["src"], minlength=g["n"]))
    return rp, g["dst"][order].astype(np.int32), g["elabel"][order].astype(np.int32)


def _same(got, want):
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{bad.size} differ; first {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}"


@pytest.mark.parametrize("mode,code", MODES)
@pytest.mark.parametrize("k", [1, 2, -1])
def test_directions_on_an_edge_list(B, mode, code, k):
    g = graphgen.powerlaw_graph(n=30_000, m=200_000, dmax=20_000, n_elabels=30, n_vlabels=5, seed=61)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(direction=code))
    rounds, blocks = B.bisim_iterate(ctx, k, 10)
    want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, 10, direction=mode)
    _same(B.get_partition(ctx).cpu().numpy(), want)
    assert rounds == wr and blocks == len(np.unique(want))
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("mode,code", MODES + [("forward", 0)])
def test_directions_from_a_csr_with_a_label_filter(B, mode, code):
    g = graphgen.uniform_graph(n=5_000, m=30_000, n_elabels=6, n_vlabels=3, seed=62)
    keep = [0, 2, 3]
    rp, col, lab = _csr(g)
    ctx = B.summarize_init(g["n"], _dev(rp), _dev(col), _dev(lab), _dev(g["vlabel"]),
                           options=B.default_options(direction=code, label_filter=keep))
    for k in (1, 3, -1):
        rounds, _ = B.bisim_iterate(ctx, k, 20)
        want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, 20, direction=mode,
                                    label_filter=keep)
        _same(B.get_partition(ctx).cpu().numpy(), want)
        assert rounds == wr
    # the summary graph: the caller's direction and labels, filtered edges left out
    es, el, et = (x.cpu().numpy() for x in B.get_summary_edges(ctx))
    P = B.get_partition(ctx).cpu().numpy()
    assert list(zip(es.tolist(), el.tolist(), et.tolist())) == \
        oracle.summary_edges(g["src"], g["dst"], g["elabel"], P, label_filter=keep)
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("mode,code", MODES)
def test_directions_on_batched_graphs(B, mode, code):
    b = graphgen.batched_graphs(n_graphs=30, nmin=20, nmax=2000, seed=63)
    keep = list(range(0, 64, 2))
    ctx = B.summarize_init_batched(*(_dev(b[x]) for x in ("vertex_offsets", "edge_offsets", "src_local",
                                                           "dst_local", "elabel", "vlabel")),
                                   options=B.default_options(direction=code, label_filter=keep))
    B.bisim_iterate(ctx, 3, 0)
    got = B.get_partition(ctx).cpu().numpy()
    vo, eo = b["vertex_offsets"], b["edge_offsets"]
    for gi in range(b["n_graphs"]):
        a, z, ea, ez = int(vo[gi]), int(vo[gi + 1]), int(eo[gi]), int(eo[gi + 1])
        want, _, _ = oracle.refine(z - a, b["src_local"][ea:ez], b["dst_local"][ea:ez], b["elabel"][ea:ez],
                                   b["vlabel"][a:z], 3, direction=mode, label_filter=keep)
        _same(got[a:z], want)
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("mode,code", MODES)
@pytest.mark.parametrize("full", [False, True])
def test_directions_under_update_batches(B, mode, code, full):
    from test_gpu_updates import random_batch
    rng = np.random.default_rng(64 + code)
    g = graphgen.uniform_graph(n=300, m=900, n_elabels=4, n_vlabels=3, seed=65)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    keep = [0, 1, 3]
    opt = B.default_options(k_incremental=2, direction=code, label_filter=keep,
                            flags=B.FLAG_FULL_RECOMPUTE if full else 0)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=opt)
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    for _ in range(10):
        ops = random_batch(rng, state, int(rng.integers(1, 60)))
        try:
            new_state = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = new_state
        want, _, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"], 2,
                                   alive=state["alive"], direction=mode, label_filter=keep)
        _same(B.get_partition(ctx).cpu().numpy(), want)
    B.summarize_destroy(ctx)


def test_forward_backward_rejects_labels_outside_its_range(B):
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    vl = np.zeros(3, np.int32)
    for bad in (1 << 30, -(1 << 30) - 1):
        with pytest.raises(B.BisimError) as ei:
            B.summarize_init_coo(3, _dev(src), _dev(dst), _dev(np.array([0, bad], np.int32)), _dev(vl),
                                 options=B.default_options(direction=B.DIR_BOTH))
        assert ei.value.status == 1
    ctx = B.summarize_init_coo(3, _dev(src), _dev(dst), _dev(np.array([-(1 << 30), (1 << 30) - 1], np.int32)),
                               _dev(vl), options=B.default_options(direction=B.DIR_BOTH, k_incremental=1))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    with pytest.raises(B.BisimError) as ei:
        B.apply_updates(ctx, _dev(np.array([[0, 2, 0, 1 << 30]], np.int32)))
    assert ei.value.status == 1
    with pytest.raises(B.BisimError):
        B.summarize_init_coo(3, _dev(src), _dev(dst), _dev(np.zeros(2, np.int32)), _dev(vl),
                             options=B.default_options(direction=7))
    B.summarize_destroy(ctx)
