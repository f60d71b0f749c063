"""Request loop scheduling on the CPU: admission by slots and memory, per-graph
order, and that every result in a concurrent mix equals the result of the same
request sequence run alone. The executor here is an oracle-backed stand-in for
the GPU executor; the GPU version of the mix test is in test_gpu_serving.py."""

import random
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2111_12493_gb300 import graphgen
from paper_2111_12493_gb300.serving import AdmissionError, Request, Scheduler


class OracleExecutor:
    """summarize / update / release on host state, with a random delay so requests overlap."""

    def __init__(self, delay=0.01, seed=0):
        self.states = {}
        self.delay = delay
        self.rng = random.Random(seed)
        self.rng_lock = threading.Lock()
        self.active = set()
        self.active_lock = threading.Lock()
        self.overlap_seen = False

    def __call__(self, req: Request, slot: int):
        with self.active_lock:
            assert req.graph_id not in self.active, "two requests on one graph ran at once"
            self.active.add(req.graph_id)
            if len(self.active) > 1:
                self.overlap_seen = True
        try:
            with self.rng_lock:
                d = self.rng.random() * self.delay
            time.sleep(d)
            p = req.payload
            if req.kind == "summarize":
                st = dict(n=p["n"], alive=np.ones(p["n"], np.uint8), vlabel=p["vlabel"].copy(), src=p["src"],
                          dst=p["dst"], elabel=p["elabel"], k=p["k"])
                if p.get("keep"):
                    self.states[req.graph_id] = st
                return _refine(st)
            if req.kind == "update":
                st = self.states[req.graph_id]
                new = oracle.apply_ops(st, p["ops"])
                new["k"] = st["k"]
                self.states[req.graph_id] = new
                return _refine(new)
            if req.kind == "release":
                self.states.pop(req.graph_id, None)
                return None
            raise ValueError(req.kind)
        finally:
            with self.active_lock:
                self.active.discard(req.graph_id)


def _refine(st):
    P, _, _ = oracle.refine(st["n"], st["src"], st["dst"], st["elabel"], st["vlabel"], st["k"], alive=st["alive"])
    return P


def _edge_ops(rng, n, src, dst, lab, size):
    """Adds among all vertices and deletes of base edges (never rejected)."""
    ops = []
    for _ in range(size):
        if rng.random() < 0.7 or len(src) == 0:
            ops.append((0, rng.integers(n), rng.integers(n), rng.integers(4)))
        else:
            i = rng.integers(len(src))
            ops.append((1, src[i], dst[i], lab[i]))
    return np.array(ops, np.int32).reshape(-1, 4)


def _workload(n_graphs=4, n_updates=5, seed=0):
    rng = np.random.default_rng(seed)
    seqs = {}
    for g in range(n_graphs):
        n = int(rng.integers(50, 400))
        G = graphgen.uniform_graph(n=n, m=3 * n, n_elabels=4, n_vlabels=3, seed=100 + g)
        reqs = [("summarize", dict(n=n, src=G["src"], dst=G["dst"], elabel=G["elabel"], vlabel=G["vlabel"],
                                   k=int(rng.integers(1, 4)), keep=True))]
        for _ in range(n_updates):
            reqs.append(("update", dict(ops=_edge_ops(rng, n, G["src"], G["dst"], G["elabel"],
                                                      int(rng.integers(1, 30))))))
        reqs.append(("release", {}))
        seqs[g] = reqs
    return seqs


def _run_alone(seqs):
    out = {}
    for g, reqs in seqs.items():
        ex = OracleExecutor(delay=0)
        out[g] = [ex(Request(kind, g, payload), 0) for kind, payload in reqs]
    return out


def test_mix_equals_alone():
    seqs = _workload()
    alone = _run_alone(seqs)
    ex = OracleExecutor(delay=0.02, seed=1)
    sched = Scheduler(ex, slots=3, mem_budget=1 << 30)
    futures = {g: [] for g in seqs}
    order = [(g, i) for g in seqs for i in range(len(seqs[g]))]
    # interleave graphs but keep each graph's own order
    rng = random.Random(3)
    cursors = {g: 0 for g in seqs}
    submitted = []
    while len(submitted) < len(order):
        g = rng.choice([g for g in seqs if cursors[g] < len(seqs[g])])
        kind, payload = seqs[g][cursors[g]]
        req = Request(kind, g, payload, mem_bytes=10)
        futures[g].append((req, sched.submit(req)))
        submitted.append((g, cursors[g]))
        cursors[g] += 1
        time.sleep(rng.random() * 0.005)
    for g in seqs:
        for i, (req, fut) in enumerate(futures[g]):
            got = fut.result(timeout=60)
            want = alone[g][i]
            if want is None:
                assert got is None
            else:
                assert np.array_equal(got, want), (g, i)
    sched.close()
    assert ex.overlap_seen and sched.max_concurrent >= 2
    for g in seqs:
        starts = [req.started for req, _ in futures[g]]
        assert starts == sorted(starts), "per-graph order broken"


def test_memory_admission_waits_for_release():
    ex = OracleExecutor(delay=0.0)
    G = graphgen.uniform_graph(n=60, m=150, seed=9)
    pay = dict(n=60, src=G["src"], dst=G["dst"], elabel=G["elabel"], vlabel=G["vlabel"], k=2, keep=True)
    sched = Scheduler(ex, slots=4, mem_budget=100)
    a = Request("summarize", "A", pay, mem_bytes=10, resident_bytes=60)
    sched.submit(a).result(timeout=30)
    assert sched.resident == {"A": 60}
    # needs 50 while only 40 are free: must wait for A's release
    b = Request("summarize", "B", dict(pay, keep=False), mem_bytes=50)
    fb = sched.submit(b)
    time.sleep(0.1)
    assert not fb.done()
    r = Request("release", "A", {})
    sched.submit(r).result(timeout=30)
    fb.result(timeout=30)
    assert b.started >= r.finished
    sched.close()
    assert sched.resident == {}


def test_no_head_of_line_blocking_across_graphs():
    ex = OracleExecutor(delay=0.0)
    G = graphgen.uniform_graph(n=40, m=100, seed=2)
    pay = dict(n=40, src=G["src"], dst=G["dst"], elabel=G["elabel"], vlabel=G["vlabel"], k=1, keep=True)
    sched = Scheduler(ex, slots=2, mem_budget=100)
    sched.submit(Request("summarize", "A", pay, mem_bytes=0, resident_bytes=70)).result(timeout=30)
    big = Request("summarize", "B", dict(pay, keep=False), mem_bytes=60)       # cannot fit yet
    small = Request("summarize", "C", dict(pay, keep=False), mem_bytes=20)     # fits now
    fbig, fsmall = sched.submit(big), sched.submit(small)
    fsmall.result(timeout=30)
    assert not fbig.done()
    # a later request on B's graph must not overtake B
    upd = Request("release", "B", {})
    fupd = sched.submit(upd)
    time.sleep(0.05)
    assert not fupd.done()
    sched.submit(Request("release", "A", {})).result(timeout=30)
    fbig.result(timeout=30)
    fupd.result(timeout=30)
    assert upd.started >= big.finished
    sched.close()


def test_oversize_request_fails_and_others_run():
    ex = OracleExecutor(delay=0.0)
    sched = Scheduler(ex, slots=1, mem_budget=100)
    f = sched.submit(Request("summarize", "X", {}, mem_bytes=200))
    with pytest.raises(AdmissionError):
        f.result(timeout=5)
    G = graphgen.uniform_graph(n=30, m=60, seed=4)
    pay = dict(n=30, src=G["src"], dst=G["dst"], elabel=G["elabel"], vlabel=G["vlabel"], k=2)
    P = sched.submit(Request("summarize", "Y", pay, mem_bytes=10)).result(timeout=30)
    want, _, _ = oracle.refine(30, G["src"], G["dst"], G["elabel"], G["vlabel"], 2)
    assert np.array_equal(P, want)
    sched.close()


def test_executor_error_reaches_the_caller_and_frees_the_slot():
    def boom(req, slot):
        if req.graph_id == "bad":
            raise RuntimeError("device said no")
        return slot

    sched = Scheduler(boom, slots=1, mem_budget=100)
    f1 = sched.submit(Request("update", "bad", {}, mem_bytes=10))
    with pytest.raises(RuntimeError, match="device said no"):
        f1.result(timeout=5)
    assert sched.submit(Request("update", "ok", {}, mem_bytes=10)).result(timeout=5) == 0
    sched.close()
    assert sched.in_flight_bytes == 0 and sched.free_slots == [0]


def test_close_fails_requests_that_can_never_fit():
    ex = OracleExecutor(delay=0.0)
    G = graphgen.uniform_graph(n=30, m=60, seed=4)
    pay = dict(n=30, src=G["src"], dst=G["dst"], elabel=G["elabel"], vlabel=G["vlabel"], k=1, keep=True)
    sched = Scheduler(ex, slots=2, mem_budget=100)
    sched.submit(Request("summarize", "A", pay, resident_bytes=90)).result(timeout=30)
    f = sched.submit(Request("summarize", "B", dict(pay, keep=False), mem_bytes=50))
    time.sleep(0.05)
    sched.close()
    with pytest.raises(AdmissionError):
        f.result(timeout=5)
