"""The autotune cache on a GPU: the first context of a shape is tuned, a second
context of the same graph takes the stored settings through bisim_retune, and
both refine to the oracle's partition."""

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen

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


def test_second_context_of_a_shape_reuses_the_tuned_settings(B, tmp_path):
    from paper_2111_12493_gb300 import tuning
    g = graphgen.powerlaw_graph(n=60_000, m=500_000, dmax=30_000, n_elabels=16, n_vlabels=4, seed=31)
    want, wr, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], oracle.FIXPOINT, 10)
    cache = tuning.TuneCache(str(tmp_path / "tune.json"))
    results = []
    for _ in range(2):
        ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
        settings, hit = tuning.autotune_cached(ctx, cache, rounds=1)
        rounds, _ = B.bisim_iterate(ctx, B.FIXPOINT, 10)
        assert rounds == wr
        assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want)
        B.summarize_destroy(ctx)
        results.append((settings, hit))
    assert results[0][1] is False and results[1][1] is True
    assert results[0][0] == results[1][0]


def test_retune_changes_the_layout_not_the_result(B):
    g = graphgen.powerlaw_graph(n=40_000, m=300_000, dmax=20_000, n_elabels=8, n_vlabels=3, seed=32)
    want, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], 3)
    ctx = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    try:
        for settings in (dict(small_max_degree=8, mid_max_degree=512, hub_chunk=256),
                         dict(small_max_degree=32, mid_max_degree=8192, hub_chunk=4096)):
            B.bisim_retune(ctx, **settings)
            B.bisim_iterate(ctx, 3, 0)
            assert np.array_equal(B.get_partition(ctx).cpu().numpy(), want), settings
            stats = B.bisim_get_stats(ctx)
            assert stats["n_hub"] > 0 if settings["mid_max_degree"] == 512 else True
    finally:
        B.summarize_destroy(ctx)
