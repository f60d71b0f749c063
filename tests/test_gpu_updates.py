"""apply_updates against the oracle: after every batch the maintained
partition must equal a batch refinement of the edited graph (Theorem 2 and
its corollary, Section 3.2.2), and invalid batches must change nothing."""

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


def random_batch(rng, state, size, n_elabels=4, n_vlabels=3, p_bad=0.0):
    """Ops drawn against the evolving state so that most are meaningful."""
    n = state["n"]
    alive = state["alive"].astype(bool).copy()
    edges = list(zip(state["src"].tolist(), state["dst"].tolist(), state["elabel"].tolist()))
    ops = []
    for _ in range(size):
        r = rng.random()
        live = np.flatnonzero(alive)
        if r < 0.45 and len(live):
            u, w = rng.choice(live), rng.choice(live)
            ops.append((0, u, w, rng.integers(n_elabels)))
            edges.append((u, w, ops[-1][3]))
        elif r < 0.70 and edges:
            e = edges[rng.integers(len(edges))]
            ops.append((1, *e))                           # may already be gone: a no-op then
        elif r < 0.78:
            ops.append((1, rng.integers(n), rng.integers(n), rng.integers(n_elabels)))   # mostly absent
        elif r < 0.86:
            v = rng.integers(n)
            ops.append((3, v, 0, 0))
            alive[v] = False
            edges = [e for e in edges if e[0] != v and e[1] != v]
        else:
            v = rng.integers(n)
            ops.append((2, v, 0, rng.integers(n_vlabels)))
            alive[v] = True
    return np.array(ops, dtype=np.int32).reshape(-1, 4)


def check_partition(B, ctx, state, k):
    got = B.get_partition(ctx).cpu().numpy()
    want, _, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"], k,
                               alive=state["alive"])
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{bad.size} differ; first {bad[:5]}: got {got[bad[:5]]} want {want[bad[:5]]}"


@pytest.mark.parametrize("seed,k", [(0, 2), (1, 1), (2, 3), (3, 0)])
def test_random_batches_match_batch_refinement(B, seed, k):
    rng = np.random.default_rng(seed)
    g = graphgen.uniform_graph(n=300, m=900, n_elabels=4, n_vlabels=3, seed=40 + seed)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    opt = B.default_options(k_incremental=k)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=opt)
    for step in range(12):
        ops = random_batch(rng, state, int(rng.integers(1, 60)))
        try:
            new_state = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            with pytest.raises(B.BisimError):
                B.apply_updates(ctx, _dev(ops))
            continue
        B.apply_updates(ctx, _dev(ops))
        state = new_state
        check_partition(B, ctx, state, k)
    B.summarize_destroy(ctx)


def test_powerlaw_batches_with_hubs(B):
    rng = np.random.default_rng(7)
    g = graphgen.powerlaw_graph(n=5000, m=60_000, dmax=12_000, n_elabels=6, n_vlabels=4, seed=77)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=2, mid_max_degree=1024))
    for step in range(4):
        ops = random_batch(rng, state, 300, n_elabels=6, n_vlabels=4)
        try:
            state2 = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = state2
        check_partition(B, ctx, state, 2)
    B.summarize_destroy(ctx)


def test_sequential_semantics_edge_cases(B):
    # add then delete, delete absent, delete+re-add of a vertex with edges around it
    n = 6
    src = np.array([0, 0, 1, 2], np.int32)
    dst = np.array([1, 1, 2, 3], np.int32)
    lab = np.array([5, 5, 6, 7], np.int32)
    vl = np.zeros(n, np.int32)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=vl.copy(), src=src, dst=dst, elabel=lab)
    ctx = B.summarize_init_coo(n, _dev(src), _dev(dst), _dev(lab), _dev(vl), options=B.default_options(k_incremental=2))
    batches = [
        [[0, 4, 5, 1], [1, 4, 5, 1]],                          # add then delete: nothing
        [[1, 0, 1, 5]],                                        # one of two parallel copies
        [[1, 3, 0, 9]],                                        # absent: no-op
        [[3, 2, 0, 0], [2, 2, 0, 4], [0, 1, 2, 6], [0, 2, 3, 1]],   # kill 2, re-add, new edges
        [[0, 5, 5, 2], [0, 5, 5, 2], [1, 5, 5, 2]],            # self-loop copies
        [[2, 0, 0, 9]],                                        # relabel a live vertex
    ]
    for ops in batches:
        ops = np.array(ops, np.int32)
        state = oracle.apply_ops(state, ops)
        B.apply_updates(ctx, _dev(ops))
        check_partition(B, ctx, state, 2)
    B.summarize_destroy(ctx)


def test_rejected_batch_changes_nothing(B):
    g = graphgen.uniform_graph(n=200, m=700, seed=5)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    B.apply_updates(ctx, _dev(np.array([[3, 7, 0, 0]], np.int32)))         # delete vertex 7
    state = oracle.apply_ops(state, np.array([[3, 7, 0, 0]], np.int32))
    before = B.get_partition(ctx).cpu().numpy()
    for bad in ([[0, 1, 7, 0]],                                          # edge to a dead vertex
                [[0, 1, 2, 0], [9, 0, 0, 0]],                            # unknown kind
                [[0, 1, 200, 0]],                                        # out of range
                [[2, 7, 0, 1], [3, 7, 0, 0], [0, 7, 1, 0]]):             # dead again at its position
        with pytest.raises(B.BisimError) as ei:
            B.apply_updates(ctx, _dev(np.array(bad, np.int32)))
        assert ei.value.status == 1
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), before)
    # still consistent after the rejections
    ops = np.array([[0, 1, 2, 0], [2, 7, 0, 2], [0, 7, 1, 3]], np.int32)
    state = oracle.apply_ops(state, ops)
    B.apply_updates(ctx, _dev(ops))
    check_partition(B, ctx, state, 2)
    B.summarize_destroy(ctx)


def test_fig1_relabel_as_update(B):
    gf = parse_golden("fig1_schemex_reconstructed.txt")
    s, d, l = edges_to_arrays(gf["edges"])
    vl = np.array(gf["vlabel"]["t"], np.int32)
    ctx = B.summarize_init_coo(gf["n"], _dev(s), _dev(d), _dev(l), _dev(vl), options=B.default_options(k_incremental=1))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    assert B.get_partition(ctx).cpu().tolist() == gf["expect"][("t", 1)].tolist()
    B.apply_updates(ctx, _dev(np.array(gf["ops"]["t1"], np.int32)))
    assert B.get_partition(ctx).cpu().tolist() == gf["expect"][("t1", 1)].tolist()
    B.summarize_destroy(ctx)


def test_iterate_after_updates_uses_the_edited_graph(B):
    rng = np.random.default_rng(11)
    g = graphgen.uniform_graph(n=400, m=1600, seed=12)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    ops = random_batch(rng, state, 80)
    state = oracle.apply_ops(state, ops)
    B.apply_updates(ctx, _dev(ops))
    r, _ = B.bisim_iterate(ctx, oracle.FIXPOINT, 50)
    want, wr, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"],
                                oracle.FIXPOINT, 50, alive=state["alive"])
    assert r == wr and np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("opts", [dict(hash_bits=6), dict(small_max_degree=0, mid_max_degree=64, hub_chunk=256),
                                  dict(flags=2)])
def test_update_paths_and_forced_collisions(B, opts):
    """Incremental maintenance with forced hash collisions, with every vertex on
    the shared-memory / hub paths, and the full-recompute flag: all exact."""
    rng = np.random.default_rng(99)
    g = graphgen.powerlaw_graph(n=2000, m=16_000, dmax=1500, n_elabels=5, n_vlabels=3, seed=98)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=2, **opts))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    check_partition(B, ctx, state, 2)
    for step in range(5):
        ops = random_batch(rng, state, int(rng.integers(5, 120)), n_elabels=5, n_vlabels=3)
        try:
            state2 = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = state2
        check_partition(B, ctx, state, 2)
    B.summarize_destroy(ctx)


def test_many_small_batches_long_run(B):
    """A longer stream of small batches (the serving pattern), every result checked."""
    rng = np.random.default_rng(5150)
    g = graphgen.powerlaw_graph(n=3000, m=24_000, dmax=2000, n_elabels=4, n_vlabels=3, seed=51)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=2))
    for step in range(40):
        ops = random_batch(rng, state, int(rng.integers(1, 12)), n_elabels=4, n_vlabels=3)
        try:
            state2 = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = state2
        check_partition(B, ctx, state, 2)
    assert B.bisim_get_stats(ctx)["last_frontier"] < state["n"]
    B.summarize_destroy(ctx)


def _apply_big(state, ops):
    new, rejected = oracle.apply_batches(state, [ops])
    assert rejected == []
    return new


def test_batch_that_outgrows_the_row_store(B):
    """One batch adds more copies to a single row than the row store keeps free,
    so the store is rebuilt half-way through the batch; the following batches
    (deleting that vertex, bringing it back with new edges, deleting many of
    the copies) must still give the exact partition."""
    rng = np.random.default_rng(61)
    n = 2000
    g = graphgen.uniform_graph(n=n, m=6000, n_elabels=3, n_vlabels=2, seed=61)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=g["vlabel"].copy(), src=g["src"], dst=g["dst"],
                 elabel=g["elabel"])
    ctx = B.summarize_init_coo(n, _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=2))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    na = 1_300_000
    big = np.stack([np.zeros(na), np.full(na, 7), rng.integers(0, n, na), rng.integers(0, 3, na)],
                   axis=1).astype(np.int32)
    state = _apply_big(state, big)
    B.apply_updates(ctx, _dev(big))
    check_partition(B, ctx, state, 2)
    follow = [
        np.array([[1, 7, int(big[i, 2]), int(big[i, 3])] for i in range(0, 5000, 7)], np.int32),   # delete copies
        np.array([[3, 7, 0, 0], [3, 11, 0, 0]], np.int32),                                       # delete vertices
        np.array([[2, 7, 0, 1], [2, 11, 0, 0], [0, 7, 11, 2], [0, 11, 7, 2], [0, 3, 11, 1]], np.int32),  # revive
    ]
    for ops in follow:
        state = _apply_big(state, ops)
        B.apply_updates(ctx, _dev(ops))
        check_partition(B, ctx, state, 2)
    # the full recompute of the edited graph agrees (the CSR is rebuilt from the store)
    B.bisim_iterate(ctx, 2, 0)
    check_partition(B, ctx, state, 2)
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("k", [1, 2])
def test_vertex_deleted_and_added_again_with_its_label(B, k):
    """A vertex deleted and added again in one batch with the label it had is
    live before and after and keeps its label, yet its out-edges are gone:
    its signatures above level 0 must be recomputed."""
    n = 7
    src = np.array([0, 0, 2, 5], np.int32)
    dst = np.array([1, 3, 3, 6], np.int32)
    lab = np.array([1, 2, 1, 1], np.int32)
    vl = np.zeros(n, np.int32)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=vl.copy(), src=src, dst=dst, elabel=lab)
    ctx = B.summarize_init_coo(n, _dev(src), _dev(dst), _dev(lab), _dev(vl), options=B.default_options(k_incremental=k))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    for ops in ([[3, 0, 0, 0], [2, 0, 0, 0]], [[0, 0, 1, 1]], [[3, 2, 0, 0], [2, 2, 0, 0], [0, 4, 2, 1]],
                [[0, 0, 3, 2], [3, 0, 0, 0], [2, 0, 0, 0]]):
        ops = np.array(ops, np.int32)
        state = oracle.apply_ops(state, ops)
        B.apply_updates(ctx, _dev(ops))
        check_partition(B, ctx, state, k)
    B.summarize_destroy(ctx)


def test_revived_vertices_do_not_keep_old_in_edges(B):
    """A vertex deleted in one batch and added again in a later one comes back
    without the edges it had (edges into it stayed in their source rows while
    it was dead and must be purged then)."""
    n = 8
    src = np.array([0, 1, 2, 3, 0, 4], np.int32)
    dst = np.array([5, 5, 5, 5, 1, 5], np.int32)
    lab = np.array([1, 1, 2, 2, 3, 1], np.int32)
    vl = np.array([0, 0, 0, 0, 0, 1, 0, 0], np.int32)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=vl.copy(), src=src, dst=dst, elabel=lab)
    ctx = B.summarize_init_coo(n, _dev(src), _dev(dst), _dev(lab), _dev(vl), options=B.default_options(k_incremental=3))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    for ops in ([[3, 5, 0, 0]], [[0, 6, 7, 1]], [[2, 5, 0, 1]], [[0, 1, 5, 1]], [[3, 5, 0, 0], [2, 5, 0, 1]],
                [[0, 2, 5, 2], [1, 2, 5, 2], [0, 2, 5, 2]]):
        ops = np.array(ops, np.int32)
        state = oracle.apply_ops(state, ops)
        B.apply_updates(ctx, _dev(ops))
        check_partition(B, ctx, state, 3)
    B.summarize_destroy(ctx)


def test_vertex_joining_a_singleton_block_one_level_down(B):
    """Vertices alone in their block one level down are not re-hashed; when another
    vertex later joins that block, the singleton must be compared again (here u is
    the only vertex with label 7 until x is relabelled to 7, and both point to w
    with the same edge label, so they become bisimilar at every level)."""
    n = 8
    u, x, w = 0, 1, 2
    src = np.array([u, x, w, 3, 4, 5], np.int32)
    dst = np.array([w, w, 3, 4, 5, 6], np.int32)
    lab = np.array([1, 1, 2, 2, 2, 2], np.int32)
    vl = np.array([7, 0, 0, 0, 0, 0, 0, 0], np.int32)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=vl.copy(), src=src, dst=dst, elabel=lab)
    for k in (1, 2, 3):
        ctx = B.summarize_init_coo(n, _dev(src), _dev(dst), _dev(lab), _dev(vl),
                                   options=B.default_options(k_incremental=k))
        B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
        st = state
        for ops in ([[2, x, 0, 7]],                    # x joins u's label block
                    [[2, x, 0, 0]],                    # and leaves it again
                    [[2, 7, 0, 7], [0, 7, w, 1]],      # a third vertex with u's label and row
                    [[1, u, w, 1], [0, u, 3, 1]]):     # u's row changes
            ops = np.array(ops, np.int32)
            st = oracle.apply_ops(st, ops)
            B.apply_updates(ctx, _dev(ops))
            check_partition(B, ctx, st, k)
        B.summarize_destroy(ctx)


@pytest.mark.parametrize("n", [1, 2, 17])
def test_updates_from_an_empty_edge_set(B, n):
    """Graphs that start without edges (rows of capacity two), grow by batches
    that fill and move rows, and lose vertices again: every result exact."""
    rng = np.random.default_rng(300 + n)
    vl = (np.arange(n) % 2).astype(np.int32)
    empty = np.zeros(0, np.int32)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=vl.copy(), src=empty, dst=empty, elabel=empty)
    ctx = B.summarize_init_coo(n, _dev(empty), _dev(empty), _dev(empty), _dev(vl),
                               options=B.default_options(k_incremental=2))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    check_partition(B, ctx, state, 2)
    for step in range(6):
        size = int(rng.integers(1, 40))
        ops = np.stack([np.zeros(size), rng.integers(0, n, size), rng.integers(0, n, size),
                        rng.integers(0, 3, size)], axis=1).astype(np.int32)
        if step == 4 and n > 1:
            ops = np.concatenate([ops, np.array([[3, n - 1, 0, 0]], np.int32)])
        if step == 5 and n > 1:
            ops = np.array([[2, n - 1, 0, 1], [0, n - 1, 0, 2], [0, 0, n - 1, 2]], np.int32)
        state = oracle.apply_ops(state, ops)
        B.apply_updates(ctx, _dev(ops))
        check_partition(B, ctx, state, 2)
    B.summarize_destroy(ctx)


def _churn_batch(rng, n, last_added, size, label_base):
    """Removes the previous batch's edges and adds `size` new ones, each with a
    label of its own: every source leaves its (large) block for a block of its
    own at every level above 0, and returns to the large block a batch later,
    leaving that block without members."""
    ops = [(1, u, w, l) for u, w, l in last_added]
    srcs = rng.choice(n, size=size, replace=False)
    added = [(int(u), int(rng.integers(n)), label_base + i) for i, u in enumerate(srcs)]
    ops += [(0, u, w, l) for u, w, l in added]
    return np.array(ops, dtype=np.int32).reshape(-1, 4), added


def test_block_ids_are_reused_and_the_state_is_built_once(B):
    """A long stream whose batches keep making and emptying blocks. Block ids
    are never renamed, so a level would run out of them after about
    bcap - n = n + 1024 new blocks if the ids of emptied blocks were not
    reused; here every batch makes about 1.5k new blocks per level (about 18k
    per level over the run, for n = 4000) and the state must still be built
    only once, with every partition equal to the oracle's. The index's
    tombstones are cleared in place along the way. A copy exported half way
    and imported (its free lists rebuilt from the block sizes) continues in
    step, without a build of its own."""
    rng = np.random.default_rng(2024)
    n = 4000
    src = np.arange(n, dtype=np.int32)
    dst = rng.integers(0, n, n).astype(np.int32)
    elabel = np.zeros(n, np.int32)
    vlabel = rng.integers(0, 2, n).astype(np.int32)
    state = dict(n=n, alive=np.ones(n, np.uint8), vlabel=vlabel, src=src, dst=dst, elabel=elabel)
    ctx = B.summarize_init_coo(n, _dev(src), _dev(dst), _dev(elabel), _dev(vlabel),
                               options=B.default_options(k_incremental=2))
    B.apply_updates(ctx, _dev(np.zeros((0, 4), np.int32)))
    B.bisim_profile_reset()
    B.bisim_profile_enable(True)
    try:
        added, copy = [], None
        for step in range(12):
            ops, added = _churn_batch(rng, n, added, 1500, 1000 + 10_000 * step)
            state = _apply_big(state, ops)
            B.apply_updates(ctx, _dev(ops))
            if copy is not None:
                B.apply_updates(copy, _dev(ops))
                assert np.array_equal(B.get_partition(copy).cpu().numpy(), B.get_partition(ctx).cpu().numpy())
            check_partition(B, ctx, state, 2)
            if step == 5:
                copy = B.bisim_import_state(B.bisim_export_state(ctx))
        refills = sum(p["launches"] for p in B.bisim_profile_read() if p["name"] == "inc_index_refill")
    finally:
        B.bisim_profile_enable(False)
    assert B.bisim_get_stats(ctx)["state_builds"] == 1
    assert B.bisim_get_stats(copy)["state_builds"] == 0
    assert refills >= 1
    B.summarize_destroy(ctx)
    B.summarize_destroy(copy)


def test_long_mixed_stream_reuses_block_ids(B):
    """150 batches of edge adds and deletes, vertex deletions, revivals and
    relabels on a 600-vertex graph at k = 3. The level-3 partitions alone
    show about 3.4k new member sets over the run, against 2n + 1024 = 2224
    ids per level of which about 1.6k are spare after the build, so without
    reuse the state would be rebuilt on the way; every partition must equal
    the oracle's and the state be built once."""
    rng = np.random.default_rng(606)
    g = graphgen.uniform_graph(n=600, m=1800, n_elabels=3, n_vlabels=4, seed=66)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=3))
    applied = 0
    for step in range(150):
        ops = random_batch(rng, state, int(rng.integers(100, 400)), n_elabels=3, n_vlabels=4)
        try:
            state2 = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = state2
        applied += 1
        check_partition(B, ctx, state, 3)
    assert applied >= 100
    assert B.bisim_get_stats(ctx)["state_builds"] == 1
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("seed", [11, 12])
def test_long_mixed_streams_on_power_law_graphs(B, seed):
    """Eighty batches of mixed operations on a power-law graph with hubs
    (out-degrees up to 600, so hub rows take the long-row and hub paths),
    k = 2, every partition equal to the oracle's."""
    rng = np.random.default_rng(seed)
    g = graphgen.powerlaw_graph(n=1500, m=9000, dmax=600, n_elabels=4, n_vlabels=3, seed=700 + seed)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=2, mid_max_degree=256))
    applied = 0
    for step in range(80):
        ops = random_batch(rng, state, int(rng.integers(20, 300)), n_elabels=4, n_vlabels=3)
        try:
            state2 = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = state2
        applied += 1
        check_partition(B, ctx, state, 2)
    assert applied >= 50
    assert B.bisim_get_stats(ctx)["state_builds"] == 1
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("direction,mode,keep", [(1, "backward", None), (2, "both", [1, 3])])
def test_long_streams_in_other_directions_and_with_a_label_filter(B, direction, mode, keep):
    """Forty batches of mixed operations with backward or forward-backward
    signatures, with and without a label filter, k = 3: every partition equal
    to the oracle's under the same parameterization (Section 2.4.2)."""
    rng = np.random.default_rng(44 + direction)
    g = graphgen.uniform_graph(n=500, m=1500, n_elabels=4, n_vlabels=3, seed=45)
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"],
                 dst=g["dst"], elabel=g["elabel"])
    opts = dict(direction=direction)
    if keep is not None:
        opts["label_filter"] = keep
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(k_incremental=3, **opts))
    for step in range(40):
        ops = random_batch(rng, state, int(rng.integers(1, 250)), n_elabels=4, n_vlabels=3)
        try:
            state2 = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        B.apply_updates(ctx, _dev(ops))
        state = state2
        got = B.get_partition(ctx).cpu().numpy()
        want, _, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"], 3,
                                   alive=state["alive"], direction=mode, label_filter=keep)
        assert np.array_equal(got, want), step
    B.summarize_destroy(ctx)
