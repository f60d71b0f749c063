"""Batched contexts: the persistent per-graph kernel, the union's round
kernels and splits between the two, against the oracle.

With batch_split = INT32_MAX bisim_iterate on a batched context is one launch
of a persistent kernel whose CTAs take whole graphs from a queue; with 0 (the
default) the union's single-graph round kernels refine every graph; in
between the two run side by side. Every graph's partition must equal its solo
run in the oracle (graph-local canonical ids), and the round count and block
count must be those of the disjoint union refined together: the largest
fixpoint round over the graphs, and the sum of their block counts.
"""

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen

pytestmark = pytest.mark.gpu

INT32_MAX = 2**31 - 1


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


def run_batched(B, b, k, cap=10_000, options=None):
    ctx = B.summarize_init_batched(*(_dev(b[key]) for key in
                                     ("vertex_offsets", "edge_offsets", "src_local", "dst_local", "elabel", "vlabel")),
                                   options=options)
    rounds, blocks = B.bisim_iterate(ctx, k, cap)
    P = B.get_partition(ctx).cpu().numpy()
    stats = B.bisim_get_stats(ctx)
    B.summarize_destroy(ctx)
    return P, rounds, blocks, stats


def oracle_batched(b, k, cap=10_000):
    """Per-graph oracle runs: (partition, union round count, union block count)."""
    vo, eo = b["vertex_offsets"], b["edge_offsets"]
    out = np.empty(int(vo[-1]), dtype=np.int32)
    rounds, blocks = 0, 0
    for g in range(b["n_graphs"]):
        v0, v1, e0, e1 = int(vo[g]), int(vo[g + 1]), int(eo[g]), int(eo[g + 1])
        P, r, _ = oracle.refine(v1 - v0, b["src_local"][e0:e1], b["dst_local"][e0:e1], b["elabel"][e0:e1],
                                b["vlabel"][v0:v1], k, cap)
        out[v0:v1] = P
        rounds = max(rounds, r)
        blocks += len(np.unique(P))
    if k != oracle.FIXPOINT:
        rounds = k
    return out, rounds, blocks


def _same(got, want, what):
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{what}: {bad.size} vertices differ, first {bad[:5]} got {got[bad[:5]]} want {want[bad[:5]]}"


def _concat(graphs):
    """Batched arrays from a list of (n, src, dst, elabel, vlabel) graphs with local ids."""
    vo = np.zeros(len(graphs) + 1, np.int64)
    eo = np.zeros(len(graphs) + 1, np.int64)
    vo[1:] = np.cumsum([g[0] for g in graphs])
    eo[1:] = np.cumsum([len(g[1]) for g in graphs])
    cat = lambda i: (np.concatenate([np.asarray(g[i], np.int32) for g in graphs]) if graphs else
                     np.zeros(0, np.int32))
    return dict(n_graphs=len(graphs), vertex_offsets=vo, edge_offsets=eo, src_local=cat(1), dst_local=cat(2),
                elabel=cat(3), vlabel=cat(4))


@pytest.mark.parametrize("k", [0, 1, 3, oracle.FIXPOINT])
def test_persistent_kernel_matches_solo_runs(B, k):
    b = graphgen.batched_graphs(n_graphs=64, nmin=2, nmax=6000, seed=14)
    want, wr, wb = oracle_batched(b, k, cap=12)
    for name, opt in (("persistent", B.default_options(batch_split=INT32_MAX)),
                      ("union", B.default_options(flags=B.FLAG_UNION_ROUNDS))):
        P, rounds, blocks, _ = run_batched(B, b, k, cap=12, options=opt)
        _same(P, want, f"{name} k={k}")
        assert rounds == wr, (name, rounds, wr)
        assert blocks == wb, (name, blocks, wb)


@pytest.mark.parametrize("bits", [1, 8])
def test_persistent_kernel_resolves_hash_collisions(B, bits):
    b = graphgen.batched_graphs(n_graphs=12, nmin=20, nmax=600 if bits == 1 else 3000, seed=15 + bits)
    want, wr, wb = oracle_batched(b, oracle.FIXPOINT, cap=8)
    P, rounds, blocks, stats = run_batched(B, b, oracle.FIXPOINT, cap=8,
                                           options=B.default_options(hash_bits=bits, batch_split=INT32_MAX))
    _same(P, want, f"hash_bits={bits}")
    assert (rounds, blocks) == (wr, wb)
    assert stats["collision_levels"] > 0


def test_persistent_kernel_long_rows_and_row_copies(B):
    """Rows for every tier of the kernel, and equal rows that need each comparison.

    Graph 1 holds two vertices with the same 20,000-entry row (the CTA set in
    several sub-range passes, and the CTA comparison of a pair), copies of a
    300-entry row (CTA set, one pass), of a 100-entry row (warp set, CTA
    comparison), of a 20-entry row (warp set and warp comparison) and of a
    5-entry row (inline comparison). Empty graphs and an edgeless one sit
    between the others.
    """
    rng = np.random.default_rng(77)
    n1 = 30_000
    src, dst, lab = [], [], []

    def row_copies(sources, length, nlab):
        tg = rng.choice(np.arange(100, n1), size=length, replace=False)
        lb = rng.integers(0, nlab, size=length)
        for s in sources:
            perm = rng.permutation(length)
            src.append(np.full(length, s))
            dst.append(tg[perm])
            lab.append(lb[perm])

    row_copies([0, 1], 20_000, 9)
    row_copies([2, 3, 4], 300, 5)
    row_copies(list(range(5, 12)), 100, 4)
    row_copies(list(range(12, 30)), 20, 3)
    row_copies(list(range(30, 60)), 5, 2)
    # a duplicated-edge row equal as a set to a plain one
    src.append(np.array([60, 60, 60, 61, 61])); dst.append(np.array([200, 200, 201, 201, 200]))
    lab.append(np.array([1, 1, 0, 0, 1]))
    rest = rng.integers(100, n1, size=60_000)
    src.append(rest); dst.append(rng.integers(0, n1, size=rest.size)); lab.append(rng.integers(0, 6, size=rest.size))
    g1 = (n1, np.concatenate(src), np.concatenate(dst), np.concatenate(lab), np.zeros(n1, np.int32))
    g2 = graphgen.powerlaw_graph(n=3000, m=15_000, dmax=2999, n_elabels=8, n_vlabels=3, seed=78)
    graphs = [(0, [], [], [], []), g1, (0, [], [], [], []),
              (g2["n"], g2["src"], g2["dst"], g2["elabel"], g2["vlabel"]),
              (5, [], [], [], [0, 1, 0, 1, 2]), (1, [0], [0], [3], [4])]
    b = _concat(graphs)
    persistent = B.default_options(batch_split=INT32_MAX)
    for k in (1, 2, oracle.FIXPOINT):
        want, wr, wb = oracle_batched(b, k, cap=10)
        P, rounds, blocks, _ = run_batched(B, b, k, cap=10, options=persistent)
        _same(P, want, f"k={k}")
        assert (rounds, blocks) == (wr, wb)
    # the two long rows, and every group of copies, share a block after one round
    P, _, _, _ = run_batched(B, b, 1, options=persistent)
    v0 = int(b["vertex_offsets"][1])
    for lo, hi in ((0, 2), (2, 5), (5, 12), (12, 30), (30, 60), (60, 62)):
        assert len(set(P[v0 + lo:v0 + hi].tolist())) == 1, (lo, hi)


def test_batched_iterate_is_one_launch(B):
    """With every graph in the persistent kernel, bisim_iterate is a single kernel launch."""
    b = graphgen.batched_graphs(n_graphs=20, nmin=10, nmax=2000, seed=17)
    counts = {}
    for name, opt in (("persistent", B.default_options(batch_split=INT32_MAX)),
                      ("union", B.default_options(flags=B.FLAG_UNION_ROUNDS))):
        ctx = B.summarize_init_batched(*(_dev(b[key]) for key in ("vertex_offsets", "edge_offsets", "src_local",
                                                                  "dst_local", "elabel", "vlabel")), options=opt)
        B.bisim_iterate(ctx, 3, 0)
        c0 = B.bisim_launch_count()
        B.bisim_iterate(ctx, 3, 0)
        counts[name] = B.bisim_launch_count() - c0
        B.summarize_destroy(ctx)
    assert counts["persistent"] == 1 and counts["union"] > 1, counts


def test_persistent_kernel_repeated_calls(B):
    """A context iterated again (the queue and the table regions are reused)."""
    b = graphgen.batched_graphs(n_graphs=40, nmin=10, nmax=4000, seed=16)
    ctx = B.summarize_init_batched(*(_dev(b[key]) for key in
                                     ("vertex_offsets", "edge_offsets", "src_local", "dst_local", "elabel", "vlabel")),
                                   options=B.default_options(batch_split=INT32_MAX))
    try:
        for k in (3, 1, oracle.FIXPOINT, 3):
            rounds, blocks = B.bisim_iterate(ctx, k, 12)
            want, wr, wb = oracle_batched(b, k, cap=12)
            _same(B.get_partition(ctx).cpu().numpy(), want, f"k={k}")
            assert (rounds, blocks) == (wr, wb)
    finally:
        B.summarize_destroy(ctx)



@pytest.mark.parametrize("split", [0, 500, 2500, INT32_MAX])
@pytest.mark.parametrize("k", [1, 3, oracle.FIXPOINT])
def test_split_between_the_two_kernels_matches_solo_runs(B, split, k):
    """Graphs above batch_split go through the union's round kernels while the
    persistent kernel takes the others on a second stream; every split gives
    each graph its solo result and the union's round and block counts."""
    b = graphgen.batched_graphs(n_graphs=48, nmin=2, nmax=6000, seed=19)
    want, wr, wb = oracle_batched(b, k, cap=12)
    P, rounds, blocks, _ = run_batched(B, b, k, cap=12, options=B.default_options(batch_split=split))
    _same(P, want, f"split={split} k={k}")
    assert (rounds, blocks) == (wr, wb)


def test_split_with_hash_collisions(B):
    b = graphgen.batched_graphs(n_graphs=16, nmin=20, nmax=3000, seed=20)
    want, wr, wb = oracle_batched(b, oracle.FIXPOINT, cap=8)
    P, rounds, blocks, stats = run_batched(B, b, oracle.FIXPOINT, cap=8,
                                           options=B.default_options(hash_bits=8, batch_split=1000))
    _same(P, want, "hash_bits=8 split=1000")
    assert (rounds, blocks) == (wr, wb)
    assert stats["collision_levels"] > 0


@pytest.mark.parametrize("which_still", ["small", "large", "none"])
def test_split_round_counts_when_one_side_is_at_its_fixpoint(B, which_still):
    """The fixpoint round of the batch is the larger of the two sides', also
    when one side's graphs are already stable at P_0 (edgeless graphs)."""
    chain = lambda n: (n, np.arange(n - 1), np.arange(1, n), np.zeros(n - 1, np.int32), np.zeros(n, np.int32))
    edgeless = lambda n: (n, [], [], [], np.arange(n) % 3)
    small = chain(40) if which_still == "small" else edgeless(40)
    large = chain(3000) if which_still == "large" else edgeless(3000)
    b = _concat([small, large, edgeless(7)])
    for k in (oracle.FIXPOINT, 2):
        want, wr, wb = oracle_batched(b, k, cap=5000)
        P, rounds, blocks, _ = run_batched(B, b, k, cap=5000, options=B.default_options(batch_split=1000))
        _same(P, want, f"{which_still} k={k}")
        assert (rounds, blocks) == (wr, wb), (which_still, k, rounds, wr, blocks, wb)


def test_split_context_iterated_again(B):
    b = graphgen.batched_graphs(n_graphs=30, nmin=10, nmax=5000, seed=21)
    ctx = B.summarize_init_batched(*(_dev(b[key]) for key in
                                     ("vertex_offsets", "edge_offsets", "src_local", "dst_local", "elabel", "vlabel")),
                                   options=B.default_options(batch_split=1500))
    try:
        for k in (3, oracle.FIXPOINT, 1, 3):
            rounds, blocks = B.bisim_iterate(ctx, k, 12)
            want, wr, wb = oracle_batched(b, k, cap=12)
            _same(B.get_partition(ctx).cpu().numpy(), want, f"k={k}")
            assert (rounds, blocks) == (wr, wb)
    finally:
        B.summarize_destroy(ctx)


def test_autotune_picks_a_listed_split_and_keeps_results(B):
    b = graphgen.batched_graphs(n_graphs=40, nmin=10, nmax=20_000, seed=22)
    want, wr, wb = oracle_batched(b, 3)
    ctx = B.summarize_init_batched(*(_dev(b[key]) for key in
                                     ("vertex_offsets", "edge_offsets", "src_local", "dst_local", "elabel", "vlabel")))
    try:
        tuned = B.bisim_autotune(ctx, rounds=2)
        assert tuned["batch_split"] in (0, 2048, 8192, 32768, INT32_MAX)
        rounds, blocks = B.bisim_iterate(ctx, 3, 0)
        _same(B.get_partition(ctx).cpu().numpy(), want, f"tuned split {tuned['batch_split']}")
        assert (rounds, blocks) == (wr, wb)
    finally:
        B.summarize_destroy(ctx)
