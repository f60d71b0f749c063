"""The allocation-free round (bisim_refine_round_noalloc) against the regular path.

The allocation-free entry point serves callers that cannot allocate device
memory (a plugin inside another runtime that owns the device heap, or a loop
that reserves every buffer up front). Its output must equal what the regular
entry points compute: two calls in a row, raw vertex labels -> P_1 -> P_2,
compared bit for bit with bisim_iterate at k = 1 and k = 2. This file is
collected last so that a stop-at-first-failure run has run everything else.
"""

import numpy as np
import pytest

from paper_2111_12493_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_12493_gb300 import bisim
    return bisim


def _csr(g):
    order = np.argsort(g["src"], kind="stable")
    rp = np.zeros(g["n"] + 1, np.int64)
    rp[1:] = np.cumsum(np.bincount(g["src"], minlength=g["n"]))
    return rp, g["dst"][order].astype(np.int32), g["elabel"][order].astype(np.int32)


@pytest.mark.parametrize("seed", [0, 1])
def test_two_noalloc_rounds_match_bisim_iterate(B, seed):
    import torch
    g = graphgen.powerlaw_graph(n=60_000, m=600_000, dmax=6_000, n_elabels=40, n_vlabels=8, seed=100 + seed)
    rp, col, lab = (torch.from_numpy(a).cuda() for a in _csr(g))
    vl = torch.from_numpy(g["vlabel"]).cuda()

    expected = []
    ctx = B.summarize_init(g["n"], rp, col, lab, vl)
    for k in (1, 2):
        _, blocks = B.bisim_iterate(ctx, k, 10)
        expected.append((B.get_partition(ctx).cpu().numpy(), blocks))
    B.summarize_destroy(ctx)

    p1 = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    p2 = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    b1 = B.bisim_refine_round_noalloc(g["n"], rp, col, lab, vl, p1)
    b2 = B.bisim_refine_round_noalloc(g["n"], rp, col, lab, p1, p2)
    assert np.array_equal(p1.cpu().numpy(), expected[0][0]) and b1 == expected[0][1]
    assert np.array_equal(p2.cpu().numpy(), expected[1][0]) and b2 == expected[1][1]


def test_noalloc_rejects_oversized_graphs(B):
    import torch
    n = 70_000
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    lab = torch.zeros(0, dtype=torch.int32, device="cuda")
    pin = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BisimError) as ei:
        B.bisim_refine_round_noalloc(n, rp, col, lab, pin, out)
    assert ei.value.status == 1 and "limit" in ei.value.message
