"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Partitions are compared element by element: both sides name a block by its
smallest vertex id, so the result must be bit-identical.
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


def gpu_partition(B, g, k, cap=10_000, options=None, alive=None):
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               alive=None if alive is None else _dev(alive), options=options)
    rounds, blocks = B.bisim_iterate(ctx, k, cap)
    P = B.get_partition(ctx).cpu().numpy()
    stats = B.bisim_get_stats(ctx)
    B.summarize_destroy(ctx)
    return P, rounds, blocks, stats


def check(B, g, ks, cap=10_000, options=None, alive=None):
    for k in ks:
        P, rounds, blocks, stats = gpu_partition(B, g, k, cap, options, alive)
        want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, cap, alive=alive)
        assert P.dtype == np.int32
        bad = np.flatnonzero(P != want)
        assert bad.size == 0, f"k={k}: {bad.size} vertices differ, first {bad[:5]} got {P[bad[:5]]} want {want[bad[:5]]}"
        assert rounds == wr, (k, rounds, wr)
        assert blocks == len(np.unique(want[want >= 0]))
    return stats


# --------------------------------------------------------------------------- paper examples

@pytest.mark.parametrize("mode", ["T", "L"])
def test_fig3_worked_example(B, mode):
    gf = parse_golden("fig3_worked_example.txt")
    s, d, l = edges_to_arrays(gf["edges"])
    g = dict(n=gf["n"], src=s, dst=d, elabel=l, vlabel=np.array(gf["vlabel"][mode], np.int32))
    P, _, _, _ = gpu_partition(B, g, 2)
    assert P.tolist() == gf["expect"][(mode, 2)].tolist()


# --------------------------------------------------------------------------- workloads (scaled where needed)

def test_uniform_10k_50k_full_size(B):
    g = graphgen.uniform_graph()                          # 10k vertices, 50k edges, k = 2
    check(B, g, [0, 1, 2, 3, oracle.FIXPOINT])


def test_powerlaw_scaled_spans_every_bucket(B):
    g = graphgen.powerlaw_graph(n=200_000, m=2_000_000, dmax=200_000, seed=2)
    deg = np.bincount(g["src"], minlength=g["n"])
    assert deg.max() > 8192 and ((deg > 32) & (deg <= 8192)).any()   # hubs and mid vertices present
    stats = check(B, g, [1, 2, oracle.FIXPOINT], cap=10)
    assert stats["n_hub"] > 0 and stats["n_mid"] > 0 and stats["n_small"] > 0


@pytest.mark.parametrize("order", ["sorted", "shuffled", "descending", "one_swap"])
def test_edge_list_order_does_not_matter(B, order):
    # a list sorted by source takes the run-based placement, any other the
    # cursor-based one; both give the oracle's partition
    g = graphgen.powerlaw_graph(n=100_000, m=1_000_000, dmax=100_000, seed=12)
    assert np.all(g["src"][1:] >= g["src"][:-1])
    m = g["src"].size
    if order == "shuffled":
        perm = np.random.default_rng(13).permutation(m)
    elif order == "descending":
        perm = np.argsort(-g["src"].astype(np.int64), kind="stable")
    elif order == "one_swap":
        perm = np.arange(m)
        perm[[m // 2, m // 2 + 1000]] = perm[[m // 2 + 1000, m // 2]]
    else:
        perm = np.arange(m)
    h = dict(g, src=g["src"][perm], dst=g["dst"][perm], elabel=g["elabel"][perm])
    check(B, h, [1, oracle.FIXPOINT], cap=10)


def test_big_hubs_with_few_and_many_distinct_values(B):
    """Hub rows of 100k entries with a few distinct pairs and of 250k with
    about 200k distinct pairs (the hub path's per-hub tables near their
    design load), and a pair of equal 40k-entry rows in different orders,
    against the oracle."""
    rng = np.random.default_rng(91)
    n = 60_000
    src, dst, lab = [], [], []
    # a 100k-entry hub with few distinct pairs (labels 0..3, targets of 3 vertex labels)
    src.append(np.zeros(100_000, np.int64)); dst.append(rng.integers(1000, n, 100_000))
    lab.append(rng.integers(0, 4, 100_000))
    # a 250k-entry hub with about 200k distinct pairs: the set overflows
    src.append(np.ones(250_000, np.int64)); dst.append(rng.integers(1000, n, 250_000))
    lab.append(rng.integers(0, 4000, 250_000))
    # two equal 40k-entry rows (sources 2 and 3), in different orders
    t = rng.integers(1000, n, 40_000); l = rng.integers(0, 50, 40_000)
    for u in (2, 3):
        p = rng.permutation(t.size)
        src.append(np.full(t.size, u)); dst.append(t[p]); lab.append(l[p])
    rest = rng.integers(4, n, 200_000)
    src.append(rest); dst.append(rng.integers(0, n, rest.size)); lab.append(rng.integers(0, 8, rest.size))
    vlabel = rng.integers(0, 3, n).astype(np.int32)
    vlabel[1000:] = rng.integers(0, 60, n - 1000)
    vlabel[3] = vlabel[2]
    g = dict(n=n, src=np.concatenate(src).astype(np.int32), dst=np.concatenate(dst).astype(np.int32),
             elabel=np.concatenate(lab).astype(np.int32), vlabel=vlabel)
    stats = check(B, g, [1, 2, oracle.FIXPOINT], cap=6)
    assert stats["n_hub"] >= 4
    P, _, _, _ = gpu_partition(B, g, 1)
    assert P[2] == P[3] == 2


def test_chain_scaled_fixpoint(B):
    g = graphgen.chain_graph(n_paths=100, path_len=200, extra=4_000, seed=3)
    check(B, g, [5, oracle.FIXPOINT])


def test_batched_scaled_matches_solo_runs(B):
    import torch
    b = graphgen.batched_graphs(n_graphs=48, nmin=20, nmax=4000, seed=4)
    ctx = B.summarize_init_batched(*(torch.from_numpy(b[k]).cuda() for k in
                                     ("vertex_offsets", "edge_offsets", "src_local", "dst_local", "elabel", "vlabel")))
    B.bisim_iterate(ctx, 3, 10)
    P = B.get_partition(ctx).cpu().numpy()
    B.summarize_destroy(ctx)
    want = oracle.refine_batched(b, 3)
    assert np.array_equal(P, want)


# --------------------------------------------------------------------------- every path forced

@pytest.mark.parametrize("small_max,mid_max", [(0, 8192), (0, 0), (32, 32), (4, 64), (16, 0)])
def test_forced_bucket_paths(B, small_max, mid_max):
    g = graphgen.powerlaw_graph(n=20_000, m=200_000, dmax=20_000, n_elabels=30, n_vlabels=6, seed=21)
    opt = B.default_options(small_max_degree=small_max, mid_max_degree=mid_max, hub_chunk=512)
    check(B, g, [1, 3, oracle.FIXPOINT], cap=12, options=opt)


@pytest.mark.parametrize("bits", [1, 8, 16])
def test_forced_hash_collisions_stay_exact(B, bits):
    g = graphgen.powerlaw_graph(n=5_000, m=40_000, dmax=6_000, n_elabels=20, n_vlabels=4, seed=5)
    opt = B.default_options(hash_bits=bits, mid_max_degree=512)
    stats = check(B, g, [0, 2, oracle.FIXPOINT], cap=8, options=opt)
    assert stats["collision_levels"] > 0


# --------------------------------------------------------------------------- edge cases

def test_empty_graph(B):
    g = dict(n=0, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), elabel=np.zeros(0, np.int32),
             vlabel=np.zeros(0, np.int32))
    P, rounds, blocks, _ = gpu_partition(B, g, 3)
    assert P.size == 0 and rounds == 3 and blocks == 0


def test_no_edges_and_single_vertex(B):
    g = dict(n=1, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), elabel=np.zeros(0, np.int32),
             vlabel=np.array([7], np.int32))
    check(B, g, [0, 1, oracle.FIXPOINT])
    g = dict(n=50, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), elabel=np.zeros(0, np.int32),
             vlabel=(np.arange(50) % 3 - 1).astype(np.int32))
    check(B, g, [0, 4, oracle.FIXPOINT])


def test_self_loops_duplicates_and_a_duplicate_heavy_hub(B):
    rng = np.random.default_rng(0)
    n = 3000
    src = np.concatenate([np.zeros(60_000, np.int32), rng.integers(0, n, 20_000).astype(np.int32),
                          np.arange(n, dtype=np.int32)])
    dst = np.concatenate([np.full(60_000, 5, np.int32), rng.integers(0, n, 20_000).astype(np.int32),
                          np.arange(n, dtype=np.int32)])
    lab = np.concatenate([np.zeros(60_000, np.int32), rng.integers(0, 3, 20_000).astype(np.int32),
                          np.ones(n, np.int32)])
    g = dict(n=n, src=src, dst=dst, elabel=lab, vlabel=rng.integers(0, 2, n).astype(np.int32))
    check(B, g, [1, 2, oracle.FIXPOINT])


def test_equal_hubs_are_compared_exactly(B):
    # hubs 0 and 1 have identical rows of 30k distinct pairs (their sets are
    # compared in sub-ranges); hub 2 differs from them in one edge label; hub 3
    # repeats hub 0's row twice (a different degree, the same set)
    n = 40_000
    targets = np.arange(4, 30_004, dtype=np.int32)
    labels = np.arange(len(targets), dtype=np.int32)          # 30k distinct pairs per row
    lab2 = labels.copy()
    lab2[12_345] = 1_000_000
    src = np.concatenate([np.zeros_like(targets), np.ones_like(targets), np.full_like(targets, 2),
                          np.full(2 * len(targets), 3, np.int32)])
    dst = np.concatenate([targets, targets, targets, targets, targets])
    lab = np.concatenate([labels, labels, lab2, labels, labels])
    rng = np.random.default_rng(3)
    extra_s = rng.integers(4, n, 50_000).astype(np.int32)
    extra_d = rng.integers(0, n, 50_000).astype(np.int32)
    g = dict(n=n, src=np.concatenate([src, extra_s]), dst=np.concatenate([dst, extra_d]),
             elabel=np.concatenate([lab, rng.integers(0, 3, 50_000).astype(np.int32)]),
             vlabel=np.zeros(n, np.int32))
    for opts in (None, B.default_options(mid_max_degree=256, hub_chunk=256)):
        check(B, g, [1, 2, oracle.FIXPOINT], options=opts)
    P, _, _, _ = gpu_partition(B, g, 2)
    assert P[1] == 0 and P[3] == 0 and P[2] == 2


def test_dead_vertices(B):
    g = graphgen.uniform_graph(n=2000, m=8000, seed=8)
    alive = np.ones(g["n"], np.uint8)
    dead = np.random.default_rng(1).choice(g["n"], 300, replace=False)
    alive[dead] = 0
    keep = alive[g["src"]].astype(bool) & alive[g["dst"]].astype(bool)
    g = dict(g, src=g["src"][keep], dst=g["dst"][keep], elabel=g["elabel"][keep])
    check(B, g, [0, 2, oracle.FIXPOINT], alive=alive)


def test_negative_and_extreme_labels(B):
    rng = np.random.default_rng(3)
    n, m = 4000, 30_000
    g = dict(n=n, src=rng.integers(0, n, m).astype(np.int32), dst=rng.integers(0, n, m).astype(np.int32),
             elabel=rng.choice(np.array([-2**31, -1, 0, 2**31 - 1], np.int64), m).astype(np.int32),
             vlabel=rng.choice(np.array([-2**31, -1, 2**31 - 1], np.int64), n).astype(np.int32))
    check(B, g, [1, 3, oracle.FIXPOINT])


def test_invalid_input_is_rejected(B):
    g = graphgen.uniform_graph(n=100, m=500, seed=9)
    bad = g["dst"].copy()
    bad[17] = 100
    with pytest.raises(B.BisimError) as ei:
        B.summarize_init_coo(100, _dev(g["src"]), _dev(bad), _dev(g["elabel"]), _dev(g["vlabel"]))
    assert ei.value.status == 1
    rp = np.array([0, 3, 2, 5], np.int64)               # not monotone
    with pytest.raises(B.BisimError):
        B.summarize_init(3, _dev(rp), _dev(np.zeros(5, np.int32)), _dev(np.zeros(5, np.int32)),
                         _dev(np.zeros(3, np.int32)))


def test_csr_entry_point_and_repeat_iterate(B):
    g = graphgen.powerlaw_graph(n=30_000, m=250_000, dmax=30_000, seed=12)
    order = np.argsort(g["src"], kind="stable")
    rp = np.zeros(g["n"] + 1, np.int64)
    rp[1:] = np.cumsum(np.bincount(g["src"], minlength=g["n"]))
    ctx = B.summarize_init(g["n"], _dev(rp), _dev(g["dst"][order]), _dev(g["elabel"][order]), _dev(g["vlabel"]))
    for k in (3, 1, 3, oracle.FIXPOINT):
        rounds, _ = B.bisim_iterate(ctx, k, 10)
        P = B.get_partition(ctx).cpu().numpy()
        want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, 10)
        assert np.array_equal(P, want) and rounds == wr
    B.summarize_destroy(ctx)


def test_host_memory_inputs_and_outputs(B):
    import torch
    g = graphgen.uniform_graph(n=3000, m=12_000, seed=13)
    pinned = {k: torch.from_numpy(g[k]).pin_memory() for k in ("src", "dst", "elabel", "vlabel")}
    ctx = B.summarize_init_coo(g["n"], pinned["src"], pinned["dst"], pinned["elabel"], pinned["vlabel"])
    B.bisim_iterate(ctx, 2)
    out = torch.empty(g["n"], dtype=torch.int32).pin_memory()
    B.get_partition(ctx, out=out)
    torch.cuda.synchronize()
    want, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], 2)
    assert np.array_equal(out.numpy(), want)
    B.summarize_destroy(ctx)
    pageable = {k: torch.from_numpy(g[k].copy()) for k in ("src", "dst", "elabel", "vlabel")}
    ctx = B.summarize_init_coo(g["n"], pageable["src"], pageable["dst"], pageable["elabel"], pageable["vlabel"])
    B.bisim_iterate(ctx, 2)
    assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
    B.summarize_destroy(ctx)


def test_host_lists_are_checked_while_they_arrive(B):
    """A host COO list is copied in beside the build (sources first): a bad
    source is caught before the layout, a bad target after it, and both give
    BISIM_EINVAL; an unsorted and a sorted power-law list, pinned, refine to
    the oracle's partition."""
    import torch
    g = graphgen.powerlaw_graph(n=50_000, m=500_000, dmax=40_000, seed=14)
    want, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], 3)
    perm = np.random.default_rng(15).permutation(g["src"].size)
    for order in (np.arange(g["src"].size), perm):
        h = {k: torch.from_numpy(np.ascontiguousarray(g[k][order] if k != "vlabel" else g[k])).pin_memory()
             for k in ("src", "dst", "elabel", "vlabel")}
        ctx = B.summarize_init_coo(g["n"], h["src"], h["dst"], h["elabel"], h["vlabel"])
        B.bisim_iterate(ctx, 3)
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
        B.summarize_destroy(ctx)
    for which in ("src", "dst"):
        bad = {k: torch.from_numpy(g[k].copy()).pin_memory() for k in ("src", "dst", "elabel", "vlabel")}
        bad[which][g["src"].size // 2] = g["n"] + 5
        with pytest.raises(B.BisimError) as ei:
            B.summarize_init_coo(g["n"], bad["src"], bad["dst"], bad["elabel"], bad["vlabel"])
        assert ei.value.status == 1, which
    # the library is still usable afterwards
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    B.bisim_iterate(ctx, 3)
    assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("bits", [64, 8])
def test_device_round_loop_matches_eager_rounds(B, bits):
    # default: the round loop runs as one captured graph (while node on the
    # device); FLAG_EAGER and profiling run it round by round from the host
    g = graphgen.powerlaw_graph(n=30_000, m=300_000, dmax=30_000, n_elabels=20, n_vlabels=5, seed=21)
    want = {k: oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, 10) for k in (1, 3, -1)}
    for flags in (0, B.FLAG_EAGER):
        opt = B.default_options(hash_bits=bits, flags=flags, mid_max_degree=1024)
        ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                                   options=opt)
        for k in (3, 1, -1, 3, -1):         # repeated calls replay the captured loop
            rounds, blocks = B.bisim_iterate(ctx, k, 10)
            P = B.get_partition(ctx).cpu().numpy()
            wP, wr, _ = want[k]
            assert np.array_equal(P, wP), (flags, k)
            assert rounds == wr and blocks == len(np.unique(wP))
        B.bisim_profile_enable(True)
        rounds, _ = B.bisim_iterate(ctx, -1, 10)
        B.bisim_profile_enable(False)
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want[-1][0]) and rounds == want[-1][1]
        B.summarize_destroy(ctx)


def test_autotune_keeps_results_and_picks_listed_settings(B):
    g = graphgen.powerlaw_graph(n=40_000, m=400_000, dmax=40_000, n_elabels=30, n_vlabels=6, seed=31)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    tuned = B.bisim_autotune(ctx, rounds=2)
    assert tuned["mid_max_degree"] in (2048, 4096, 8192)
    assert tuned["small_max_degree"] in (8, 16, 32)
    assert tuned["hub_chunk"] in (1024, 2048, 4096)
    for k in (2, -1):
        rounds, _ = B.bisim_iterate(ctx, k, 10)
        want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, 10)
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want) and rounds == wr
    B.summarize_destroy(ctx)
