"""The allocation-free round (bisim_refine_round_noalloc).

Some callers cannot allocate device memory: a plugin inside another runtime
that owns the device heap, or a loop that reserves every buffer up front
because an allocation may synchronise the device or fail under fragmentation.
For them the library runs one refinement round with its scratch in a fixed
array compiled into the library. Its output must equal what the regular entry
point (bisim_iterate) computes and what the CPU oracle computes: two calls in
a row, raw vertex labels -> P_1 -> P_2, compared bit for bit. The array keeps
the last call's contents, so calls are also checked after a larger call has
left it dirty, and at the exact size limits. Every rejection must happen
before any kernel touches the caller's arrays.

This file is collected last so that a stop-at-first-failure run has run every
other test before it.
"""

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen

pytestmark = pytest.mark.gpu

MAX_N = 65536
MAX_M = 1 << 20
MAX_DEG = 8192


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


def _dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _two_rounds(B, g):
    """P_1 and P_2 from the allocation-free round, with their block counts."""
    import torch
    rp, col, lab, vl = _dev(*_csr(g), g["vlabel"])
    p1 = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    p2 = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    b1 = B.bisim_refine_round_noalloc(g["n"], rp, col, lab, vl, p1)
    b2 = B.bisim_refine_round_noalloc(g["n"], rp, col, lab, p1, p2)
    return (p1.cpu().numpy(), b1), (p2.cpu().numpy(), b2)


def _oracle_rounds(g):
    P0 = g["vlabel"]          # any labelling of the label partition: the round only compares ids
    P1 = oracle.refine_round(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], P0)
    P2 = oracle.refine_round(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], P1)
    return P1, P2


def _check_against_oracle(B, g):
    (p1, b1), (p2, b2) = _two_rounds(B, g)
    w1, w2 = _oracle_rounds(g)
    assert np.array_equal(p1, w1) and b1 == len(np.unique(w1))
    assert np.array_equal(p2, w2) and b2 == len(np.unique(w2))


@pytest.mark.parametrize("seed", [0, 1])
def test_two_noalloc_rounds_match_bisim_iterate_and_the_oracle(B, seed):
    g = graphgen.powerlaw_graph(n=60_000, m=600_000, dmax=6_000, n_elabels=40, n_vlabels=8, seed=100 + seed)
    rp, col, lab, vl = _dev(*_csr(g), g["vlabel"])
    expected = []
    ctx = B.summarize_init(g["n"], rp, col, lab, vl)
    for k in (1, 2):
        _, blocks = B.bisim_iterate(ctx, k, 10)
        expected.append((B.get_partition(ctx).cpu().numpy(), blocks))
    B.summarize_destroy(ctx)
    (p1, b1), (p2, b2) = _two_rounds(B, g)
    assert np.array_equal(p1, expected[0][0]) and b1 == expected[0][1]
    assert np.array_equal(p2, expected[1][0]) and b2 == expected[1][1]
    w1, w2 = _oracle_rounds(g)
    assert np.array_equal(p1, w1) and np.array_equal(p2, w2)


def test_noalloc_at_the_exact_size_limits(B):
    # n = 65536 fills the whole 2n-slot table; m = 2^20 the whole list array
    g = graphgen.powerlaw_graph(n=MAX_N, m=MAX_M, dmax=MAX_DEG, n_elabels=30, n_vlabels=6, seed=140)
    assert g["n"] == MAX_N and len(g["src"]) == MAX_M
    assert np.bincount(g["src"], minlength=g["n"]).max() <= MAX_DEG
    (p1, b1), _ = _two_rounds(B, g)
    rp, col, lab, vl = _dev(*_csr(g), g["vlabel"])
    ctx = B.summarize_init(g["n"], rp, col, lab, vl)
    _, blocks = B.bisim_iterate(ctx, 1, 10)
    assert np.array_equal(p1, B.get_partition(ctx).cpu().numpy()) and b1 == blocks
    B.summarize_destroy(ctx)
    _check_against_oracle(B, g)


def test_noalloc_after_a_larger_call_left_the_array_dirty(B):
    big = graphgen.powerlaw_graph(n=MAX_N, m=500_000, dmax=4_000, n_elabels=20, n_vlabels=5, seed=141)
    small = graphgen.uniform_graph(n=1_000, m=5_000, n_elabels=4, n_vlabels=3, seed=142)
    _check_against_oracle(B, big)
    _check_against_oracle(B, small)
    _check_against_oracle(B, big)


def _rejected(B, *args, match=None):
    with pytest.raises(B.BisimError) as ei:
        B.bisim_refine_round_noalloc(*args)
    assert ei.value.status == 1, ei.value
    if match:
        assert match in ei.value.message, ei.value.message


def test_noalloc_rejects_oversized_graphs(B):
    import torch
    n = MAX_N + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    lab = torch.zeros(0, dtype=torch.int32, device="cuda")
    pin = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _rejected(B, n, rp, col, lab, pin, out, match="limit")
    # one edge over the limit
    n = 100
    m = MAX_M + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    rp[1:] = m
    col = torch.zeros(m, dtype=torch.int32, device="cuda")
    lab = torch.zeros(m, dtype=torch.int32, device="cuda")
    _rejected(B, n, rp, col, lab, torch.zeros(n, dtype=torch.int32, device="cuda"),
              torch.empty(n, dtype=torch.int32, device="cuda"), match="limit")


def test_noalloc_rejects_malformed_input_and_leaves_the_output_alone(B):
    import torch
    g = graphgen.uniform_graph(n=500, m=3_000, n_elabels=4, n_vlabels=3, seed=143)
    rp, col, lab = _csr(g)
    n = g["n"]
    vl = torch.from_numpy(g["vlabel"]).cuda()
    sentinel = torch.full((n,), 7, dtype=torch.int32, device="cuda")

    def run(rp_, col_, lab_, bin_=vl, bout=sentinel, n_=n):
        _rejected(B, n_, rp_, col_, lab_, bin_, bout)
        assert bool((sentinel == 7).all())

    d_rp, d_col, d_lab = _dev(rp, col, lab)
    # row_ptr not a prefix sum of [0, m]: decreasing, wrong end, wrong start
    bad = rp.copy(); bad[10], bad[11] = bad[11], bad[10] - 1
    run(*_dev(bad), d_col, d_lab)
    bad = rp.copy(); bad[-1] -= 1
    run(*_dev(bad), d_col, d_lab)
    bad = rp.copy(); bad[0] = 1
    run(*_dev(bad), d_col, d_lab)
    # a target out of range, and a negative one
    for v in (n, -1):
        bad = col.copy(); bad[17] = v
        run(d_rp, *_dev(bad), d_lab)
    # block_in and block_out the same array
    same = vl.clone()
    _rejected(B, n, d_rp, d_col, d_lab, same, same, match="differ")
    # host arrays (pinned and pageable)
    run(d_rp, d_col, d_lab, bin_=vl.cpu().pin_memory())
    run(d_rp.cpu(), d_col, d_lab)
    _rejected(B, n, d_rp, d_col, d_lab, vl, torch.empty(n, dtype=torch.int32).pin_memory())
    # one out-degree above the limit
    m = MAX_DEG + 1
    rp2 = np.zeros(11, np.int64)
    rp2[1:] = m
    col2 = np.full(m, 3, np.int32)
    lab2 = np.zeros(m, np.int32)
    out2 = torch.full((10,), 7, dtype=torch.int32, device="cuda")
    _rejected(B, 10, *_dev(rp2, col2, lab2), torch.zeros(10, dtype=torch.int32, device="cuda"), out2,
              match="8192")
    assert bool((out2 == 7).all())


def test_noalloc_rejects_memory_of_another_device(B):
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    g = graphgen.uniform_graph(n=200, m=1_000, n_elabels=4, n_vlabels=3, seed=144)
    rp, col, lab = _csr(g)
    with torch.cuda.device(0):
        d_rp, d_col, d_lab = (torch.from_numpy(a).to("cuda:1") for a in (rp, col, lab))
        vl = torch.from_numpy(g["vlabel"]).to("cuda:0")
        out = torch.empty(g["n"], dtype=torch.int32, device="cuda:0")
        _rejected(B, g["n"], d_rp, d_col, d_lab, vl, out, match="current device")
