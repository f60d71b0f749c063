"""Algorithm 4 taken literally (bisim_literal_alg4) against the oracle's
restatement of the printed algorithm (two identifier tracks; the last round
without edge labels). The definition's partition must refine it.
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


def _ctx(B, g, alive=None, **opts):
    return B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                                alive=None if alive is None else _dev(alive),
                                options=B.default_options(**opts) if opts else None)


def test_literal_worked_example_and_counterexample(B):
    gf = parse_golden("fig3_worked_example.txt")
    s, d, l = edges_to_arrays(gf["edges"])
    g = dict(n=gf["n"], src=s, dst=d, elabel=l, vlabel=np.array(gf["vlabel"]["T"], np.int32))
    ctx = _ctx(B, g)
    P, blocks = B.bisim_literal_alg4(ctx, 2)
    assert P.cpu().numpy().tolist() == gf["expect"][("T", 2)].tolist() and blocks == 3
    B.summarize_destroy(ctx)
    s, d, l = edges_to_arrays([(0, 2, 0), (0, 3, 1), (1, 3, 0), (1, 2, 1), (2, 4, 2), (3, 5, 3)])
    g = dict(n=6, src=s, dst=d, elabel=l, vlabel=np.zeros(6, np.int32))
    ctx = _ctx(B, g)
    lit, _ = B.bisim_literal_alg4(ctx, 2)
    B.bisim_iterate(ctx, 2, 0)
    P = B.get_partition(ctx).cpu().numpy()
    lit = lit.cpu().numpy()
    assert lit[0] == lit[1] and P[0] != P[1]
    assert lit.tolist() == oracle.literal_alg4(6, s, d, l, g["vlabel"], 2).tolist()
    B.summarize_destroy(ctx)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_literal_matches_the_oracle_at_every_k(B, seed):
    g = graphgen.uniform_graph(n=3000, m=9000, n_elabels=3, n_vlabels=2, seed=70 + seed)
    alive = (np.random.default_rng(seed).random(g["n"]) > 0.05).astype(np.uint8)
    keep = alive[g["src"]].astype(bool) & alive[g["dst"]].astype(bool)
    g = dict(g, src=g["src"][keep], dst=g["dst"][keep], elabel=g["elabel"][keep])
    ctx = _ctx(B, g, alive=alive)
    for k in range(0, 5):
        lit, blocks = B.bisim_literal_alg4(ctx, k)
        want = oracle.literal_alg4(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k, alive=alive)
        assert np.array_equal(lit.cpu().numpy(), want), k
        assert blocks == len(np.unique(want[want >= 0]))
    # the context's own partition is untouched
    B.bisim_iterate(ctx, 2, 0)
    P, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], 2, alive=alive)
    assert np.array_equal(B.get_partition(ctx).cpu().numpy(), P)
    B.summarize_destroy(ctx)


def test_literal_on_a_powerlaw_graph_and_with_collisions(B):
    g = graphgen.powerlaw_graph(n=40_000, m=300_000, dmax=20_000, n_elabels=20, n_vlabels=4, seed=75)
    for opts in ({}, {"hash_bits": 12}):
        ctx = _ctx(B, g, **opts)
        for k in (2, 3):
            lit, _ = B.bisim_literal_alg4(ctx, k)
            want = oracle.literal_alg4(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k)
            assert np.array_equal(lit.cpu().numpy(), want), (opts, k)
        B.summarize_destroy(ctx)


def test_literal_follows_the_direction_mode(B):
    g = graphgen.uniform_graph(n=1500, m=5000, n_elabels=3, n_vlabels=2, seed=76)
    ctx = _ctx(B, g, direction=B.DIR_BACKWARD)
    lit, _ = B.bisim_literal_alg4(ctx, 3)
    want = oracle.literal_alg4(g["n"], g["dst"], g["src"], g["elabel"], g["vlabel"], 3)
    assert np.array_equal(lit.cpu().numpy(), want)
    B.summarize_destroy(ctx)
