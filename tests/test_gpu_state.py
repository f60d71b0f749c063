"""Export and import of a context's state (bisim_export_state /
bisim_import_state).

Update batches applied to an imported context must continue exactly where
the exported context stood: after more batches, both contexts hold the same
partition, and by Theorem 2 (Section 3.2.2) it equals the oracle's batch run
on the edited graph. A blob that is not an exported state is rejected.
"""

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


def _state(g):
    return dict(n=g["n"], alive=np.ones(g["n"], np.uint8), vlabel=g["vlabel"].copy(), src=g["src"], dst=g["dst"],
                elabel=g["elabel"])


def _batches(rng, state, count):
    from test_gpu_updates import random_batch
    out = []
    for _ in range(count):
        ops = random_batch(rng, state, int(rng.integers(1, 60)))
        try:
            state = oracle.apply_ops(state, ops)
        except oracle.UpdateRejected:
            continue
        out.append(ops)
    return out, state


@pytest.mark.parametrize("opts,mode,keep", [({}, "forward", None),
                                            ({"direction": 2, "label_filter": [0, 2, 3]}, "both", [0, 2, 3])])
def test_import_resumes_update_batches(B, opts, mode, keep):
    rng = np.random.default_rng(81)
    g = graphgen.uniform_graph(n=400, m=1400, n_elabels=4, n_vlabels=3, seed=82)
    state = _state(g)
    A = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]),
                             options=B.default_options(k_incremental=2, **opts))
    B.apply_updates(A, _dev(np.zeros((0, 4), np.int32)))
    first, state = _batches(rng, state, 5)
    for ops in first:
        B.apply_updates(A, _dev(ops))
    blob = B.bisim_export_state(A)
    C = B.bisim_import_state(blob)
    assert np.array_equal(B.get_partition(C).cpu().numpy(), B.get_partition(A).cpu().numpy())
    # the imported context exports the same state again
    assert B.bisim_export_state(C) == blob
    second, state = _batches(rng, state, 6)
    for ops in second:
        B.apply_updates(A, _dev(ops))
        B.apply_updates(C, _dev(ops))
    want, _, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"], 2,
                               alive=state["alive"], direction=mode, label_filter=keep)
    got_a = B.get_partition(A).cpu().numpy()
    got_c = B.get_partition(C).cpu().numpy()
    assert np.array_equal(got_c, want) and np.array_equal(got_a, want)
    assert B.bisim_get_stats(C)["updates_applied"] == B.bisim_get_stats(A)["updates_applied"]
    B.summarize_destroy(A)
    B.summarize_destroy(C)


def test_export_without_incremental_state(B):
    g = graphgen.powerlaw_graph(n=20_000, m=150_000, dmax=10_000, n_elabels=20, n_vlabels=4, seed=83)
    A = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    B.bisim_iterate(A, 3, 0)
    C = B.bisim_import_state(B.bisim_export_state(A))
    want, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], 3)
    assert np.array_equal(B.get_partition(C).cpu().numpy(), want)
    # the imported graph refines like the original, and takes update batches
    B.bisim_iterate(C, B.FIXPOINT, 10)
    want, _, _ = oracle.refine(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], oracle.FIXPOINT, 10)
    assert np.array_equal(B.get_partition(C).cpu().numpy(), want)
    state = _state(g)
    ops = np.array([[0, 5, 7, 1], [3, 11, 0, 0], [1, 5, 7, 1]], np.int32)
    B.apply_updates(C, _dev(ops))
    state = oracle.apply_ops(state, ops)
    want, _, _ = oracle.refine(state["n"], state["src"], state["dst"], state["elabel"], state["vlabel"], 2,
                               alive=state["alive"])
    assert np.array_equal(B.get_partition(C).cpu().numpy(), want)
    B.summarize_destroy(A)
    B.summarize_destroy(C)


def test_import_rejects_what_is_not_a_state(B):
    g = graphgen.uniform_graph(n=100, m=300, seed=84)
    A = B.summarize_init_coo(g["n"], _dev(g["src"]), _dev(g["dst"]), _dev(g["elabel"]), _dev(g["vlabel"]))
    blob = B.bisim_export_state(A)
    B.summarize_destroy(A)
    for bad in (blob[:-8], blob + b"\0" * 8, b"X" + blob[1:], b"\0" * 32):
        with pytest.raises(B.BisimError) as ei:
            B.bisim_import_state(bad)
        assert ei.value.status == 1
