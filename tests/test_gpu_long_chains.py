"""Long k-chaining on the GPU: hundreds of refinement rounds.

The hash-messaging method exists for long chains of k (Section 3.3): on a
directed path with uniform labels every round splits exactly one vertex off,
so the fixpoint needs as many rounds as the path is long. The closed form
(one directed path of m+1 vertices, one vertex label, one edge label):

    after round i the vertices at distance >= i from the sink form one block,
    every vertex closer to the sink is alone, so there are min(i+1, m+1)
    blocks, and the fixpoint is reached at r = m.

These tests run that form at m = 1000 through the captured device-side round
loop (table epochs wrap every 15 rounds, the active list shrinks by one
vertex per round) and through host-driven rounds, and many identical paths
(every vertex active in every round) against the oracle.
"""

import numpy as np
import pytest

import oracle

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


def _paths(n_paths, length):
    """n_paths directed paths of `length` vertices (path-major ids), uniform labels."""
    base = (np.arange(n_paths, dtype=np.int64) * length)[:, None]
    src = (base + np.arange(length - 1)[None, :]).reshape(-1).astype(np.int32)
    n = n_paths * length
    return dict(n=n, src=src, dst=(src + 1).astype(np.int32), elabel=np.zeros(len(src), np.int32),
                vlabel=np.zeros(n, np.int32))


def _closed_form(m, k):
    """Canonical partition of one path of m+1 vertices (sink m) after k rounds."""
    i = np.arange(m + 1)
    dist = m - i
    return np.where(dist >= k, 0, i).astype(np.int32)


@pytest.mark.parametrize("eager", [False, True], ids=["captured-loop", "eager"])
def test_path_of_1001_vertices_needs_exactly_1000_rounds(B, eager):
    m = 1000
    g = _paths(1, m + 1)
    flags = B.FLAG_EAGER if eager else 0
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                               options=B.default_options(flags=flags))
    rounds, blocks = B.bisim_iterate(ctx, B.FIXPOINT, 5000)
    assert rounds == m and blocks == m + 1
    assert B.bisim_get_stats(ctx)["rounds_executed"] == m + 1
    assert np.array_equal(B.get_partition(ctx).cpu().numpy(), _closed_form(m, m))
    # sampled rounds, across epoch wraps (every 15) and past the fixpoint
    for k in (1, 2, 14, 15, 16, 17, 30, 31, 499, 998, 999, 1000, 1001, 1500):
        rounds, blocks = B.bisim_iterate(ctx, k, 0)
        assert rounds == k and blocks == min(k + 1, m + 1), (k, blocks)
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), _closed_form(m, k)), k
    # the fixpoint with a cap below it stops at the cap
    rounds, blocks = B.bisim_iterate(ctx, B.FIXPOINT, 300)
    assert rounds == 300 and blocks == 301
    B.summarize_destroy(ctx)


def test_identical_paths_keep_every_vertex_active_until_the_fixpoint(B):
    # 64 paths of 300 vertices: every block has 64 members, so no vertex is
    # ever alone and the whole graph is listed in all 300 rounds
    g = _paths(64, 300)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    rounds, blocks = B.bisim_iterate(ctx, B.FIXPOINT, 5000)
    want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], oracle.FIXPOINT, 5000)
    assert rounds == wr == 299 and blocks == 300
    assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
    for k in (1, 150, 298):
        B.bisim_iterate(ctx, k, 0)
        want, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], k)
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want), k
    B.summarize_destroy(ctx)


def test_paths_of_mixed_lengths_with_random_labels_match_the_oracle(B):
    rng = np.random.default_rng(77)
    lengths = rng.integers(2, 400, size=60)
    starts = np.concatenate([[0], np.cumsum(lengths)])
    src = np.concatenate([np.arange(a, b - 1) for a, b in zip(starts[:-1], starts[1:])]).astype(np.int32)
    n = int(starts[-1])
    # rare marks: a few edge labels and vertex labels differ, so blocks merge
    # across paths and split over hundreds of rounds
    g = dict(n=n, src=src, dst=(src + 1).astype(np.int32),
             elabel=(rng.random(len(src)) < 0.002).astype(np.int32),
             vlabel=(rng.random(n) < 0.003).astype(np.int32))
    for eager in (False, True):
        ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                                   options=B.default_options(flags=B.FLAG_EAGER if eager else 0))
        rounds, blocks = B.bisim_iterate(ctx, B.FIXPOINT, 5000)
        want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], oracle.FIXPOINT, 5000)
        assert rounds == wr and rounds > 100
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
        B.summarize_destroy(ctx)
