"""The request loop on the GPU: summarization and update requests for several
resident graphs run concurrently on separate streams, and every result equals
both the result of the same request sequence run alone and the oracle's."""

import time

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_12493_gb300 import serving
    return serving


def _ops(rng, n, src, dst, lab, size, n_elabels):
    ops = []
    for _ in range(size):
        r = rng.random()
        if r < 0.65 or len(src) == 0:
            ops.append((0, rng.integers(n), rng.integers(n), rng.integers(n_elabels)))
        elif r < 0.95:
            i = rng.integers(len(src))
            ops.append((1, src[i], dst[i], lab[i]))
        else:
            ops.append((2, rng.integers(n), 0, rng.integers(3)))      # relabel a live vertex
    return np.array(ops, np.int32).reshape(-1, 4)


def _workload(seed=0):
    import torch
    rng = np.random.default_rng(seed)
    graphs = [graphgen.uniform_graph(n=300, m=900, n_elabels=4, n_vlabels=3, seed=11),
              graphgen.uniform_graph(n=2000, m=7000, n_elabels=4, n_vlabels=3, seed=12),
              graphgen.powerlaw_graph(n=20_000, m=200_000, dmax=20_000, n_elabels=8, n_vlabels=3, seed=13),
              graphgen.uniform_graph(n=50, m=100, n_elabels=2, n_vlabels=3, seed=14)]
    seqs = {}
    for g, G in enumerate(graphs):
        n = G["n"]
        k = [2, 1, 2, 3][g]
        reqs = [("summarize", dict(n=n, src=G["src"], dst=G["dst"], elabel=G["elabel"], vlabel=G["vlabel"], k=k))]
        for _ in range(4):
            size = int(rng.integers(1, 400))
            reqs.append(("update", _ops(rng, n, G["src"], G["dst"], G["elabel"], size, 8)))
        seqs[g] = reqs
    return seqs


def _submit(server, g, kind, payload):
    import torch
    if kind == "summarize":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
        return server.summarize(g, payload["n"], t(payload["src"]), t(payload["dst"]), t(payload["elabel"]),
                                t(payload["vlabel"]), k=payload["k"], keep=True, k_incremental=payload["k"])
    return server.update(g, torch.from_numpy(payload))


def _oracle_results(seqs):
    out = {}
    for g, reqs in seqs.items():
        p = reqs[0][1]
        st = dict(n=p["n"], alive=np.ones(p["n"], np.uint8), vlabel=p["vlabel"].copy(), src=p["src"],
                  dst=p["dst"], elabel=p["elabel"])
        res = []
        for kind, payload in reqs:
            if kind == "update":
                st = oracle.apply_ops(st, payload)
            P, _, _ = oracle.refine(st["n"], st["src"], st["dst"], st["elabel"], st["vlabel"], p["k"],
                                    alive=st["alive"])
            res.append(P)
        out[g] = res
    return out


def test_results_same_alone_and_in_the_mix(serving):
    seqs = _workload()
    want = _oracle_results(seqs)

    # alone: one slot, one graph after another, each request waited for
    alone = {}
    srv = serving.Server(slots=1)
    for g, reqs in seqs.items():
        alone[g] = [_submit(srv, g, kind, p).result(timeout=300)["partition"].cpu().numpy() for kind, p in reqs]
        srv.release(g).result(timeout=60)
    srv.close()

    # in the mix: four slots, all graphs' requests submitted interleaved without waiting
    srv = serving.Server(slots=4)
    futures = {g: [] for g in seqs}
    rng = np.random.default_rng(5)
    cursors = {g: 0 for g in seqs}
    while any(cursors[g] < len(seqs[g]) for g in seqs):
        g = int(rng.choice([g for g in seqs if cursors[g] < len(seqs[g])]))
        kind, p = seqs[g][cursors[g]]
        futures[g].append(_submit(srv, g, kind, p))
        cursors[g] += 1
        time.sleep(float(rng.random()) * 0.002)
    mixed = {g: [f.result(timeout=300)["partition"].cpu().numpy() for f in futures[g]] for g in seqs}
    concurrent = srv.scheduler.max_concurrent
    srv.close()

    for g in seqs:
        for i in range(len(seqs[g])):
            assert np.array_equal(alone[g][i], want[g][i]), f"alone: graph {g} request {i}"
            assert np.array_equal(mixed[g][i], want[g][i]), f"mix: graph {g} request {i}"
    assert concurrent >= 2


def test_memory_budget_serialises_large_requests(serving):
    import torch
    G = graphgen.uniform_graph(n=5000, m=20_000, seed=21)
    est = serving.estimate_bytes(G["n"], len(G["src"]))
    # room for one summarization at a time
    srv = serving.Server(slots=4, mem_budget=int(est * 1.5))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    futs = [srv.summarize(i, G["n"], t(G["src"]), t(G["dst"]), t(G["elabel"]), t(G["vlabel"]), k=2)
            for i in range(3)]
    res = [f.result(timeout=300)["partition"].cpu().numpy() for f in futs]
    assert srv.scheduler.max_concurrent == 1
    srv.close()
    want, _, _ = oracle.refine(G["n"], G["src"], G["dst"], G["elabel"], G["vlabel"], 2)
    for r in res:
        assert np.array_equal(r, want)
