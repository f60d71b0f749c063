"""Pins for the CPU oracle: it is checked against things other than itself.

* the paper's worked examples (tests/golden/, each with its citation);
* closed forms that follow from the definition (Section 2.5);
* brute force of the pairwise definition on tiny graphs (exhaustive and random);
* the Paige-Tarjan coarsest stable partition for the fixpoint;
* invariants: refinement, stability, permutation / edge-order / duplicate-edge
  invariance, and the own-label form of the self term;
* planted mistakes: every wrong variant of the oracle fails at least one pin.
"""

import itertools
import random

import numpy as np
import pytest

import oracle
from refcheck import (brute_force, canonical, coarsest_stable, edges_to_arrays,
                      parse_golden)


def run(n, edges, vlabel, k, variant=0, cap=10_000, alive=None):
    s, d, l = edges_to_arrays(edges)
    P, rounds, _ = oracle.refine(n, s, d, l, np.array(vlabel, dtype=np.int32), k, cap,
                                 alive=alive, variant=variant)
    return P, rounds


# --------------------------------------------------------------------------- worked examples

@pytest.mark.parametrize("mode", ["T", "L"])
def test_fig3_worked_example(mode):
    g = parse_golden("fig3_worked_example.txt")
    for (m, k), want in g["expect"].items():
        if m != mode:
            continue
        P, _ = run(g["n"], g["edges"], g["vlabel"][mode], k)
        assert P.tolist() == want.tolist()


def test_fig1_schemex_reconstructed():
    g = parse_golden("fig1_schemex_reconstructed.txt")
    P, _ = run(g["n"], g["edges"], g["vlabel"]["t"], 1)
    assert P.tolist() == g["expect"][("t", 1)].tolist()
    assert P[0] == P[3]                       # v1 ~ v7 at time t
    s, d, l = edges_to_arrays(g["edges"])
    state = dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=np.array(g["vlabel"]["t"], np.int32),
                 src=s, dst=d, elabel=l)
    st = oracle.apply_ops(state, np.array(g["ops"]["t1"], dtype=np.int32))
    P1, _, _ = oracle.refine(st["n"], st["src"], st["dst"], st["elabel"], st["vlabel"], 1,
                             alive=st["alive"])
    assert P1.tolist() == g["expect"][("t1", 1)].tolist()
    assert P1[0] != P1[3]                     # v1 and v7 separate after v8 becomes an Agent


# --------------------------------------------------------------------------- closed forms

def test_no_edges_keeps_label_partition():
    vl = [3, 1, 3, 0, 1, 1, 7]
    P0, _ = run(7, [], vl, 0)
    assert P0.tolist() == [0, 1, 0, 3, 1, 1, 6]
    for k in range(1, 5):
        Pk, _ = run(7, [], vl, k)
        assert Pk.tolist() == P0.tolist()
    Pf, r = run(7, [], vl, oracle.FIXPOINT)
    assert r == 0 and Pf.tolist() == P0.tolist()


@pytest.mark.parametrize("m", [1, 2, 5, 13])
def test_directed_path(m):
    # v_0 -> v_1 -> ... -> v_m, one label everywhere. Vertex j lies m-j hops from
    # the sink; after round i the vertices >= i hops away share block 0 and the
    # others are singletons, so round i has min(i+1, m+1) blocks, fixpoint r = m.
    edges = [(j, j + 1, 0) for j in range(m)]
    vl = [0] * (m + 1)
    for i in range(m + 3):
        P, _ = run(m + 1, edges, vl, i)
        want = [0 if (m - j) >= i else j for j in range(m + 1)]
        assert P.tolist() == want
        assert len(set(P.tolist())) == min(i + 1, m + 1)
    P, r = run(m + 1, edges, vl, oracle.FIXPOINT)
    assert r == m and P.tolist() == list(range(m + 1))


@pytest.mark.parametrize("n", [1, 2, 7])
def test_directed_cycle_is_one_block(n):
    edges = [(j, (j + 1) % n, 4) for j in range(n)]
    for k in range(4):
        P, _ = run(n, edges, [2] * n, k)
        assert P.tolist() == [0] * n


def test_complete_digraph_is_one_block():
    n = 6
    edges = [(u, v, 1) for u in range(n) for v in range(n) if u != v]
    P, r = run(n, edges, [5] * n, oracle.FIXPOINT)
    assert P.tolist() == [0] * n and r == 0


def test_out_star():
    # hub 0 (label 0) -> leaves with labels 0/1; leaves are sinks, grouped by label;
    # from k = 1 on the hub is a block of its own.
    leaves = [0, 1, 1, 0, 1, 0, 0]
    vl = [0] + leaves
    edges = [(0, j + 1, 9) for j in range(len(leaves))]
    P0, _ = run(len(vl), edges, vl, 0)
    assert P0[0] == 0 and P0[1] == 0
    first = {0: 1, 1: 2}
    for k in (1, 2, 3):
        P, _ = run(len(vl), edges, vl, k)
        assert P[0] == 0
        assert P[1:].tolist() == [first[x] for x in leaves]


def test_label_to_neighbour_pairing_is_kept():
    # v -a-> X, v -b-> Y, v' -a-> Y, v' -b-> X, X -c-> sink, Y -d-> sink.
    # At k = 1 v ~ v' (X and Y share the label block); at k = 2 the definition
    # separates them because (a, [X]) != (a, [Y]). Hashing only the neighbour
    # ids without their edge labels would merge them.
    v, vp, X, Y, z = 0, 1, 2, 3, 4
    a, b, c, d = 0, 1, 2, 3
    edges = [(v, X, a), (v, Y, b), (vp, Y, a), (vp, X, b), (X, z, c), (Y, z, d)]
    vl = [0, 0, 0, 0, 0]
    P1, _ = run(5, edges, vl, 1)
    assert P1[v] == P1[vp]
    P2, _ = run(5, edges, vl, 2)
    assert P2[v] != P2[vp]


# --------------------------------------------------------------------------- brute force

def _check_against_brute(n, edges, vl, kmax, alive=None):
    bf = brute_force(n, edges, vl, kmax, alive=alive)
    for k in range(kmax + 1):
        P, _ = run(n, edges, vl, k, alive=alive)
        assert P.tolist() == bf[k].tolist(), (n, edges, vl, k)


def test_brute_force_exhaustive_n3_one_label():
    pairs = [(u, v) for u in range(3) for v in range(3)]
    for mask in range(1 << len(pairs)):
        edges = [(u, v, 0) for i, (u, v) in enumerate(pairs) if mask >> i & 1]
        for vl in ([0, 0, 0], [0, 0, 1], [0, 1, 0], [1, 0, 0]):
            _check_against_brute(3, edges, vl, 3)


def test_brute_force_exhaustive_n2_two_labels():
    cand = [(u, v, l) for u in range(2) for v in range(2) for l in range(2)]
    for mask in range(1 << len(cand)):
        edges = [e for i, e in enumerate(cand) if mask >> i & 1]
        for vl in ([0, 0], [0, 1]):
            _check_against_brute(2, edges, vl, 3)


def test_brute_force_random_multigraphs():
    rnd = random.Random(12493)
    for _ in range(250):
        n = rnd.randint(1, 11)
        m = rnd.randint(0, 3 * n)
        L = rnd.randint(1, 3)
        edges = [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(L)) for _ in range(m)]
        edges += edges[: rnd.randint(0, len(edges))]          # duplicate some edges
        vl = [rnd.choice([-1, 0, 1]) for _ in range(n)]
        alive = [rnd.random() > 0.15 for _ in range(n)]
        _check_against_brute(n, edges, vl, rnd.randint(0, 5), alive=np.array(alive, np.uint8))


# --------------------------------------------------------------------------- backward and forward-backward

def _run_dir(n, edges, vl, k, direction, alive=None):
    s, d, l = edges_to_arrays(edges) if edges else (np.zeros(0, np.int32),) * 3
    P, r, _ = oracle.refine(n, s, d, l, np.array(vl, np.int32), k, alive=alive, direction=direction)
    return P, r


@pytest.mark.parametrize("direction", ["backward", "both"])
def test_directions_exhaustive_n3_one_label(direction):
    pairs = [(u, v) for u in range(3) for v in range(3)]
    for mask in range(1 << len(pairs)):
        edges = [(u, v, 0) for i, (u, v) in enumerate(pairs) if mask >> i & 1]
        for vl in ([0, 0, 0], [0, 0, 1]):
            bf = brute_force(3, edges, vl, 3, direction=direction)
            for k in range(4):
                assert _run_dir(3, edges, vl, k, direction)[0].tolist() == bf[k].tolist(), (edges, vl, k)


@pytest.mark.parametrize("direction", ["backward", "both"])
def test_directions_random_multigraphs(direction):
    rnd = random.Random(2111 + len(direction))
    for _ in range(150):
        n = rnd.randint(1, 10)
        edges = [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(2)) for _ in range(rnd.randint(0, 3 * n))]
        vl = [rnd.choice([-1, 0, 1]) for _ in range(n)]
        alive = np.array([rnd.random() > 0.15 for _ in range(n)], np.uint8)
        kmax = rnd.randint(0, 5)
        bf = brute_force(n, edges, vl, kmax, alive=alive, direction=direction)
        for k in range(kmax + 1):
            assert _run_dir(n, edges, vl, k, direction, alive)[0].tolist() == bf[k].tolist()


@pytest.mark.parametrize("m", [1, 4, 7])
def test_directed_path_backward_and_both(m):
    # backward: a vertex sees only its predecessors, so after k rounds the
    # vertices at distance >= k from the source form one block (the mirror of
    # the forward form); both: a vertex is told apart by min(distance to the
    # source, k) and min(distance to the sink, k)
    edges = [(i, i + 1, 0) for i in range(m)]
    vl = [0] * (m + 1)
    for k in range(m + 2):
        P, _ = _run_dir(m + 1, edges, vl, k, "backward")
        assert P.tolist() == [i if i < k else k for i in range(m + 1)]
        P, _ = _run_dir(m + 1, edges, vl, k, "both")
        key = [(min(i, k), min(m - i, k)) for i in range(m + 1)]
        first = {}
        assert P.tolist() == [first.setdefault(x, i) for i, x in enumerate(key)]
    assert _run_dir(m + 1, edges, vl, oracle.FIXPOINT, "backward")[1] == m


def test_backward_fixpoint_is_the_coarsest_stable_partition_of_the_reversed_graph():
    rnd = random.Random(8)
    for _ in range(80):
        n = rnd.randint(1, 14)
        edges = [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(3)) for _ in range(rnd.randint(0, 3 * n))]
        vl = [rnd.randrange(2) for _ in range(n)]
        P, _ = _run_dir(n, edges, vl, oracle.FIXPOINT, "backward")
        assert P.tolist() == coarsest_stable(n, [(d, s, l) for s, d, l in edges], vl).tolist()


def test_label_filter_keeps_only_listed_labels():
    # an out-star with leaf labels: filtering the only edge label that tells
    # two hubs apart merges them
    edges = [(0, 2, 5), (1, 3, 6)]
    s, d, l = edges_to_arrays(edges)
    vl = np.zeros(4, np.int32)
    P, _, _ = oracle.refine(4, s, d, l, vl, 1)
    assert P.tolist() == [0, 1, 2, 2]
    P, _, _ = oracle.refine(4, s, d, l, vl, 1, label_filter=[5])
    assert P.tolist() == [0, 1, 1, 1]               # vertex 1 lost its only edge: like a sink
    P, _, _ = oracle.refine(4, s, d, l, vl, 1, label_filter=[])
    assert P.tolist() == [0, 0, 0, 0]
    P, _, _ = oracle.refine(4, s, d, l, vl, 1, label_filter=[5, 6, 7])
    assert P.tolist() == [0, 1, 2, 2]


# --------------------------------------------------------------------------- fixpoint

def test_fixpoint_equals_coarsest_stable_partition():
    rnd = random.Random(7)
    for _ in range(120):
        n = rnd.randint(1, 16)
        m = rnd.randint(0, 3 * n)
        L = rnd.randint(1, 3)
        edges = [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(L)) for _ in range(m)]
        vl = [rnd.randrange(2) for _ in range(n)]
        P, r = run(n, edges, vl, oracle.FIXPOINT)
        assert P.tolist() == coarsest_stable(n, edges, vl).tolist()
        # r is the first round after which nothing changes
        Pr, _ = run(n, edges, vl, r)
        assert Pr.tolist() == P.tolist()
        if r > 0:
            Prm, _ = run(n, edges, vl, r - 1)
            assert Prm.tolist() != P.tolist()


# --------------------------------------------------------------------------- invariants

def _rand_graph(seed, n=60, m=200, L=4, V=3):
    rnd = np.random.default_rng(seed)
    return (n, rnd.integers(0, n, m).astype(np.int32), rnd.integers(0, n, m).astype(np.int32),
            rnd.integers(0, L, m).astype(np.int32), rnd.integers(0, V, n).astype(np.int32))


def _refines(fine, coarse):
    seen = {}
    for f, c in zip(fine.tolist(), coarse.tolist()):
        if seen.setdefault(f, c) != c:
            return False
    return True


@pytest.mark.parametrize("seed", range(6))
def test_refinement_and_stability(seed):
    n, s, d, l, vl = _rand_graph(seed)
    P, r, ex, hist = oracle.refine(n, s, d, l, vl, oracle.FIXPOINT, history=True)
    for i in range(1, len(hist)):
        assert _refines(hist[i], hist[i - 1])
        assert len(set(hist[i].tolist())) >= len(set(hist[i - 1].tolist()))
    again = oracle.refine_round(n, s, d, l, vl, P)
    assert again.tolist() == P.tolist()


@pytest.mark.parametrize("seed", range(6))
def test_permutation_invariance(seed):
    n, s, d, l, vl = _rand_graph(seed)
    pi = np.random.default_rng(100 + seed).permutation(n).astype(np.int32)
    for k in (0, 1, 2, 4):
        P, _, _ = oracle.refine(n, s, d, l, vl, k)
        vl2 = np.empty_like(vl)
        vl2[pi] = vl
        Q, _, _ = oracle.refine(n, pi[s], pi[d], l, vl2, k)
        # the partition maps under pi: u ~ v  <=>  pi(u) ~ pi(v)
        assert canonical(Q[pi]).tolist() == P.tolist()


@pytest.mark.parametrize("seed", range(4))
def test_edge_order_and_duplicate_invariance(seed):
    n, s, d, l, vl = _rand_graph(seed)
    P, _, _ = oracle.refine(n, s, d, l, vl, 3)
    order = np.random.default_rng(seed).permutation(len(s))
    dup = np.random.default_rng(seed + 1).integers(0, len(s), 80)
    s2 = np.concatenate([s[order], s[dup]])
    d2 = np.concatenate([d[order], d[dup]])
    l2 = np.concatenate([l[order], l[dup]])
    Q, _, _ = oracle.refine(n, s2, d2, l2, vl, 3)
    assert Q.tolist() == P.tolist()


@pytest.mark.parametrize("seed", range(6))
def test_own_label_self_term_gives_same_partition(seed):
    n, s, d, l, vl = _rand_graph(seed)
    for k in (1, 2, 5, oracle.FIXPOINT):
        P, r1, _ = oracle.refine(n, s, d, l, vl, k)
        Q, r2, _ = oracle.refine(n, s, d, l, vl, k, variant=oracle.VARIANT_OWN_LABEL)
        assert P.tolist() == Q.tolist() and r1 == r2


def test_batched_graph_ids_keep_graphs_apart():
    from paper_2111_12493_gb300 import graphgen
    b = graphgen.batched_graphs(n_graphs=12, nmin=5, nmax=60, seed=9)
    u = graphgen.batched_union(b)
    P, _, _ = oracle.refine(u["n"], u["src"], u["dst"], u["elabel"], u["vlabel"], 3, graph=u["graph"])
    local = oracle.refine_batched(b, 3)
    off = np.repeat(b["vertex_offsets"][:-1], np.diff(b["vertex_offsets"]))
    assert (P - off).tolist() == local.tolist()


# --------------------------------------------------------------------------- summary graph and payload

def test_summary_of_the_worked_example():
    gf = parse_golden("fig3_worked_example.txt")
    s, d, l = edges_to_arrays(gf["edges"])
    for mode in ("T", "L"):
        P, _, _ = oracle.refine(gf["n"], s, d, l, np.array(gf["vlabel"][mode], np.int32), 2)
        assert oracle.summary_edges(s, d, l, P) == gf["summary"][2]
        assert oracle.block_sizes(P).tolist() == gf["sizes"][2].tolist()


@pytest.mark.parametrize("m", [1, 4, 9])
def test_summary_of_a_directed_path(m):
    # after k rounds: vertices 0..m-k form block 0, the rest are alone; the
    # summary keeps the path's direction and label
    s = np.arange(m, dtype=np.int32)
    d = s + 1
    l = np.full(m, 3, np.int32)
    for k in range(0, m + 2):
        P, _, _ = oracle.refine(m + 1, s, d, l, np.zeros(m + 1, np.int32), k)
        head = max(0, m - k)                        # last vertex of block 0
        want = set()
        for u in range(m):
            a = 0 if u <= head else u
            b = 0 if u + 1 <= head else u + 1
            want.add((a, 3, b))
        assert oracle.summary_edges(s, d, l, P) == sorted(want), k
        sizes = [0] * (m + 1)
        sizes[0] = head + 1
        for v in range(head + 1, m + 1):
            sizes[v] = 1
        assert oracle.block_sizes(P).tolist() == sizes


def test_summary_collapses_parallel_edges_of_one_label():
    # a directed cycle with uniform labels is one block: its n edges collapse
    # into one self-loop per label
    n = 6
    s = np.arange(n, dtype=np.int32)
    d = ((s + 1) % n).astype(np.int32)
    for labels, want in ((np.zeros(n, np.int32), [(0, 0, 0)]),):
        P, _, _ = oracle.refine(n, s, d, labels, np.zeros(n, np.int32), oracle.FIXPOINT)
        assert oracle.summary_edges(s, d, labels, P) == want
        assert oracle.block_sizes(P).tolist() == [n] + [0] * (n - 1)
    # an out-star whose leaves share one class but are reached by three labels:
    # one summary edge per label
    s = np.zeros(5, np.int32)
    d = np.arange(1, 6, dtype=np.int32)
    l = np.array([7, 8, 7, 9, 8], np.int32)
    P, _, _ = oracle.refine(6, s, d, l, np.zeros(6, np.int32), 2)
    assert P.tolist() == [0, 1, 1, 1, 1, 1]
    assert oracle.summary_edges(s, d, l, P) == [(0, 7, 1), (0, 8, 1), (0, 9, 1)]


def test_summary_skips_dead_vertices_and_every_edge_has_a_witness():
    n, s, d, l, vl = _rand_graph(11, n=80, m=300, L=3, V=2)
    alive = (np.random.default_rng(3).random(n) > 0.2).astype(np.uint8)
    P, _, _ = oracle.refine(n, s, d, l, vl, 2, alive=alive)
    E = oracle.summary_edges(s, d, l, P)
    images = {(int(P[u]), int(x), int(P[w])) for u, w, x in zip(s, d, l) if alive[u] and alive[w]}
    assert set(E) == images and len(E) == len(images)
    sizes = oracle.block_sizes(P)
    assert sizes.sum() == int(alive.sum())
    assert sorted(np.flatnonzero(sizes).tolist()) == sorted(set(int(b) for b in P if b >= 0))


# --------------------------------------------------------------------------- Algorithm 4 taken literally

def test_literal_alg4_reproduces_the_worked_example():
    # the worked example of Section 3.3.1 runs Algorithm 4 itself on the
    # Figure 3 graph at k = 2 (tautology start): classes {v1}, {v2}, {v3, v4}
    gf = parse_golden("fig3_worked_example.txt")
    s, d, l = edges_to_arrays(gf["edges"])
    for mode in ("T", "L"):
        P = oracle.literal_alg4(gf["n"], s, d, l, np.array(gf["vlabel"][mode], np.int32), 2)
        assert P.tolist() == gf["expect"][(mode, 2)].tolist()


def test_literal_alg4_merges_what_the_definition_separates():
    # v -a-> X, v -b-> Y and v' -a-> Y, v' -b-> X, where X and Y differ by
    # their own out-label: the last round of Algorithm 4 drops the edge label,
    # so it merges v and v' at k = 2; the definition keeps the pairing apart
    edges = [(0, 2, 0), (0, 3, 1), (1, 3, 0), (1, 2, 1), (2, 4, 2), (3, 5, 3)]
    s, d, l = edges_to_arrays(edges)
    vl = np.zeros(6, np.int32)
    lit = oracle.literal_alg4(6, s, d, l, vl, 2)
    P, _, _ = oracle.refine(6, s, d, l, vl, 2)
    assert lit[0] == lit[1] and P[0] != P[1]


def test_literal_alg4_keeps_sinks_apart_by_their_identifier():
    # two sinks with different labels reached over the same edge label: the
    # sinks keep their id_o (no messages), so their predecessors stay apart
    edges = [(0, 2, 0), (1, 3, 0)]
    s, d, l = edges_to_arrays(edges)
    vl = np.array([0, 0, 1, 2], np.int32)
    lit = oracle.literal_alg4(4, s, d, l, vl, 2)
    assert lit.tolist() == [0, 1, 2, 3]


def test_literal_alg4_is_refined_by_the_definition():
    rnd = random.Random(4)
    for _ in range(200):
        n = rnd.randint(1, 12)
        edges = [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(2)) for _ in range(rnd.randint(0, 3 * n))]
        s, d, l = edges_to_arrays(edges) if edges else (np.zeros(0, np.int32),) * 3
        vl = np.array([rnd.randrange(2) for _ in range(n)], np.int32)
        alive = np.array([rnd.random() > 0.1 for _ in range(n)], np.uint8)
        for k in range(0, 5):
            lit = oracle.literal_alg4(n, s, d, l, vl, k, alive=alive)
            P, _, _ = oracle.refine(n, s, d, l, vl, k, alive=alive)
            if k <= 1:
                assert lit.tolist() == P.tolist()      # one round: the same signature
            assert _refines(P, lit)


# --------------------------------------------------------------------------- CPU baselines

@pytest.mark.parametrize("seed", range(4))
def test_round_over_a_vertex_range_numbers_by_the_range_minimum(seed):
    # within a range, v's id is the smallest vertex of the range in v's block
    # of the full round (computed here from the full round by numpy)
    n, s, d, l, vl = _rand_graph(seed, n=300, m=900, L=2, V=2)
    P0 = oracle.label_partition(n, vl)
    full = oracle.refine_round(n, s, d, l, vl, P0)
    assert oracle.refine_round_range(n, s, d, l, vl, P0, 0, n).tolist() == full.tolist()
    cuts = [0, 37, 150, 151, 299, 300]
    out = np.full(n, -7, np.int32)
    for v0, v1 in zip(cuts[:-1], cuts[1:]):
        oracle.refine_round_range(n, s, d, l, vl, P0, v0, v1, out=out)
        blk = full[v0:v1]
        first = {}
        for i, b in enumerate(blk.tolist()):
            first.setdefault(b, v0 + i)
        assert out[v0:v1].tolist() == [first[b] for b in blk.tolist()]
    with pytest.raises(ValueError):
        oracle.refine_round_range(n, s, d, l, vl, P0, 10, 5)


@pytest.mark.parametrize("threads", [1, 2, 3, 7])
def test_threaded_round_equals_the_oracle_round(threads):
    for seed in range(5):
        n, s, d, l, vl = _rand_graph(seed, n=400, m=1500, L=3, V=3)
        alive = (np.random.default_rng(seed).random(n) > 0.1).astype(np.uint8)
        P, _, _ = oracle.refine(n, s, d, l, vl, 2, alive=alive)
        want = oracle.refine_round(n, s, d, l, vl, P, alive=alive)
        got = oracle.refine_round_threads(n, s, d, l, P, threads=threads, alive=alive)
        assert got.tolist() == want.tolist()
    from paper_2111_12493_gb300 import graphgen
    b = graphgen.batched_graphs(n_graphs=10, nmin=5, nmax=80, seed=5)
    u = graphgen.batched_union(b)
    P, _, _ = oracle.refine(u["n"], u["src"], u["dst"], u["elabel"], u["vlabel"], 1, graph=u["graph"])
    want = oracle.refine_round(u["n"], u["src"], u["dst"], u["elabel"], u["vlabel"], P, graph=u["graph"])
    got = oracle.refine_round_threads(u["n"], u["src"], u["dst"], u["elabel"], P, threads=threads, graph=u["graph"])
    assert got.tolist() == want.tolist()


# --------------------------------------------------------------------------- planted mistakes

PINS = []


def _pin(f):
    PINS.append(f)
    return f


@_pin
def _pin_fig3(variant):
    g = parse_golden("fig3_worked_example.txt")
    for (mode, k), want in g["expect"].items():
        P, _ = run(g["n"], g["edges"], g["vlabel"][mode], k, variant=variant)
        if P.tolist() != want.tolist():
            return False
    return True


@_pin
def _pin_no_edges(variant):
    vl = [3, 1, 3, 0, 1]
    P, _ = run(5, [], vl, 2, variant=variant)
    return P.tolist() == [0, 1, 0, 3, 1]


@_pin
def _pin_path(variant):
    m = 6
    edges = [(j, j + 1, 0) for j in range(m)]
    for i in range(m + 1):
        P, _ = run(m + 1, edges, [0] * (m + 1), i, variant=variant)
        if P.tolist() != [0 if (m - j) >= i else j for j in range(m + 1)]:
            return False
    return True


@_pin
def _pin_pairing(variant):
    edges = [(0, 2, 0), (0, 3, 1), (1, 3, 0), (1, 2, 1), (2, 4, 2), (3, 4, 3)]
    P, _ = run(5, edges, [0] * 5, 2, variant=variant)
    return P[0] != P[1]


@_pin
def _pin_brute(variant):
    rnd = random.Random(5)
    for _ in range(60):
        n = rnd.randint(2, 8)
        edges = [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(2)) for _ in range(rnd.randint(1, 2 * n))]
        edges += edges[:2]
        vl = [rnd.randrange(2) for _ in range(n)]
        bf = brute_force(n, edges, vl, 3)
        for k in range(4):
            P, _ = run(n, edges, vl, k, variant=variant)
            if P.tolist() != bf[k].tolist():
                return False
    return True


def test_definition_passes_every_pin():
    for pin in PINS:
        assert pin(oracle.VARIANT_DEFINITION), pin.__name__
        assert pin(oracle.VARIANT_OWN_LABEL), pin.__name__


@pytest.mark.parametrize("variant", [oracle.VARIANT_DROP_EDGE_LABEL, oracle.VARIANT_DROP_SELF,
                                     oracle.VARIANT_REVERSE, oracle.VARIANT_MULTISET])
def test_planted_mistake_is_caught(variant):
    failed = [pin.__name__ for pin in PINS if not pin(variant)]
    assert failed, f"variant {variant} passed every pin"


# --------------------------------------------------------------------------- update semantics

def test_apply_ops_sequential_semantics():
    st = dict(n=4, alive=np.ones(4, np.uint8), vlabel=np.zeros(4, np.int32),
              src=np.array([0, 0, 1], np.int32), dst=np.array([1, 1, 2], np.int32),
              elabel=np.array([5, 5, 6], np.int32))
    ops = np.array([[oracle.OP_EDGE_DEL, 0, 1, 5],     # removes one of the two parallel edges
                    [oracle.OP_EDGE_DEL, 3, 2, 1],     # absent: no-op
                    [oracle.OP_EDGE_ADD, 2, 3, 7],
                    [oracle.OP_VERTEX_DEL, 1, 0, 0],   # drops 0->1 and 1->2
                    [oracle.OP_VERTEX_ADD, 1, 0, 9]],  # back, with no edges and label 9
                   dtype=np.int32)
    out = oracle.apply_ops(st, ops)
    assert out["alive"].tolist() == [1, 1, 1, 1]
    assert out["vlabel"].tolist() == [0, 9, 0, 0]
    assert sorted(zip(out["src"].tolist(), out["dst"].tolist(), out["elabel"].tolist())) == [(2, 3, 7)]


def test_vertex_deleted_and_added_with_its_label_has_no_edges_left():
    # a vertex deleted and added again in one batch with the label it had
    # comes back without its edges: with every label equal and no edge left,
    # every vertex is in one block at k = 1 (before the batch, vertex 0's
    # out-edge set it apart)
    st = dict(n=4, alive=np.ones(4, np.uint8), vlabel=np.zeros(4, np.int32),
              src=np.array([0], np.int32), dst=np.array([1], np.int32), elabel=np.array([1], np.int32))
    before, _, _ = oracle.refine(4, st["src"], st["dst"], st["elabel"], st["vlabel"], 1)
    assert before.tolist() == [0, 1, 1, 1]
    out = oracle.apply_ops(st, np.array([[oracle.OP_VERTEX_DEL, 0, 0, 0], [oracle.OP_VERTEX_ADD, 0, 0, 0]], np.int32))
    assert len(out["src"]) == 0 and out["alive"].tolist() == [1, 1, 1, 1] and out["vlabel"].tolist() == [0, 0, 0, 0]
    after, _, _ = oracle.refine(4, out["src"], out["dst"], out["elabel"], out["vlabel"], 1, alive=out["alive"])
    assert after.tolist() == [0, 0, 0, 0]


def test_apply_ops_rejects_whole_batch():
    st = dict(n=3, alive=np.array([1, 1, 0], np.uint8), vlabel=np.zeros(3, np.int32),
              src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), elabel=np.zeros(0, np.int32))
    with pytest.raises(oracle.UpdateRejected):
        oracle.apply_ops(st, np.array([[oracle.OP_EDGE_ADD, 0, 1, 0], [oracle.OP_EDGE_ADD, 0, 2, 0]], np.int32))
    with pytest.raises(oracle.UpdateRejected):
        oracle.apply_ops(st, np.array([[oracle.OP_EDGE_ADD, 0, 3, 0]], np.int32))
    with pytest.raises(oracle.UpdateRejected):
        oracle.apply_ops(st, np.array([[9, 0, 1, 0]], np.int32))


def _multiset(state):
    return sorted(zip(state["src"].tolist(), state["dst"].tolist(), state["elabel"].tolist()))


@pytest.mark.parametrize("seed", range(6))
def test_batch_applier_agrees_with_sequential_apply_ops(seed):
    # the C++ applier used for large graphs must give what apply_ops gives, batch by batch
    rng = np.random.default_rng(seed)
    n = 12
    m = 30
    state = dict(n=n, alive=(rng.random(n) < 0.9).astype(np.uint8), vlabel=rng.integers(0, 3, n).astype(np.int32))
    live = np.flatnonzero(state["alive"])
    s = rng.choice(live, m)
    d = rng.choice(live, m)
    state.update(src=s.astype(np.int32), dst=d.astype(np.int32), elabel=rng.integers(0, 3, m).astype(np.int32))
    batches = []
    for _ in range(8):
        ops = []
        for _ in range(int(rng.integers(1, 12))):
            kind = int(rng.choice([0, 0, 1, 1, 2, 3], p=[0.25, 0.1, 0.25, 0.15, 0.15, 0.1]))
            a, b, lab = int(rng.integers(-1, n + 1)) if rng.random() < 0.05 else int(rng.integers(0, n)), \
                int(rng.integers(0, n)), int(rng.integers(0, 3))
            if kind == 1 and len(state["src"]) and rng.random() < 0.7:
                i = int(rng.integers(len(state["src"])))
                a, b, lab = int(state["src"][i]), int(state["dst"][i]), int(state["elabel"][i])
            ops.append((kind, a, b, lab))
        batches.append(np.array(ops, np.int32))
    want = state
    want_rejected = []
    for i, ops in enumerate(batches):
        try:
            want = oracle.apply_ops(want, ops)
        except oracle.UpdateRejected:
            want_rejected.append(i)
    got, rejected = oracle.apply_batches(state, batches)
    assert rejected == want_rejected
    assert _multiset(got) == _multiset(want)
    assert np.array_equal(got["alive"], want["alive"]) and np.array_equal(got["vlabel"], want["vlabel"])
