"""CPU oracle for exact k-bisimulation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never does, and the oracle shares no code with it.

``bisim_oracle.cpp`` restates the definition of forward k-bisimulation
(Section 2.5, with the chaining parameterization of Section 2.4.2) using exact
signatures: sorted vectors of (edge label, neighbour block) pairs inside an
ordered map, no hashing. ``apply_ops`` restates the update semantics of the
incremental setting (Section 3.2: additions, deletions and modifications of
vertices and edges) as a plain sequential edit of an edge list; by Theorem 2
(Section 3.2.2) an incremental summary must equal the batch summary of the
edited graph, so the oracle for an update batch is the batch oracle run on the
result of ``apply_ops``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bisim_oracle.cpp")
_SRC_THREADS = os.path.join(_HERE, "bisim_oracle_threads.cpp")
_LIB = os.path.join(_HERE, "libbisim_oracle.so")
_lock = threading.Lock()
_lib = None

VARIANT_DEFINITION = 0
VARIANT_DROP_EDGE_LABEL = 1
VARIANT_DROP_SELF = 2
VARIANT_REVERSE = 4
VARIANT_MULTISET = 8
VARIANT_OWN_LABEL = 16

FIXPOINT = -1

# Direction of the edges that make up a vertex's set (Section 2.5): forward
# uses out-edges, backward in-edges, both the two sets with each pair tagged.
DIRECTIONS = {"forward": 0, "backward": 1, "both": 2}

OP_EDGE_ADD = 0
OP_EDGE_DEL = 1
OP_VERTEX_ADD = 2
OP_VERTEX_DEL = 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library with the host C++ compiler."""
    srcs = [_SRC, _SRC_THREADS]
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in srcs):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, *srcs])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            p = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.oracle_refine.argtypes = [i32, p, p, p, i64, p, p, p, i32, i32, i32, i32, p, p, p, p, i32]
            lib.oracle_refine.restype = ctypes.c_int
            lib.oracle_round.argtypes = [i32, p, p, p, i64, p, p, p, p, i32, i32, p]
            lib.oracle_round.restype = ctypes.c_int
            lib.oracle_round_range.argtypes = [i32, p, p, p, i64, p, p, p, p, i32, i32, p]
            lib.oracle_round_range.restype = ctypes.c_int
            lib.oracle_round_threads.argtypes = [i32, p, p, i64, p, p, p, p, i32, p]
            lib.oracle_round_threads.restype = ctypes.c_int
            lib.oracle_label_partition.argtypes = [i32, p, p, p, p]
            lib.oracle_label_partition.restype = ctypes.c_int
            lib.oracle_apply_ops.argtypes = [i32, p, p, i64, p, p, p, i32, p, p, i64, p, p, p, p, p]
            lib.oracle_apply_ops.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _filtered(src, dst, elabel, label_filter):
    """The edges whose label is in label_filter (all edges when it is None)."""
    if label_filter is None:
        return src, dst, elabel
    keep = np.isin(np.asarray(elabel), np.asarray(label_filter, dtype=np.int64))
    return np.asarray(src)[keep], np.asarray(dst)[keep], np.asarray(elabel)[keep]


def refine(n, src, dst, elabel, vlabel, k, cap=10_000, alive=None, graph=None,
           variant=VARIANT_DEFINITION, history=False, direction="forward", label_filter=None):
    """Exact partition after k rounds (k >= 0) or at the fixpoint (k = FIXPOINT).

    Returns (P, rounds, executed[, history]) where P is int32 [n] of canonical
    block ids (smallest vertex id of the block, -1 for dead vertices).
    `direction` picks the edges of a vertex's set (forward, backward, both);
    `label_filter`, when given, keeps only the edges with one of its labels.
    """
    lib = _load()
    src, dst, elabel = _filtered(src, dst, elabel, label_filter)
    src, dst, elabel, vlabel, graph = map(_i32, (src, dst, elabel, vlabel, graph))
    alive = None if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
    m = len(src)
    P = np.empty(n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    executed = ctypes.c_int32(0)
    rows = (k if k >= 0 else cap) + 1
    hist = np.full((rows, n), -2, dtype=np.int32) if history else None
    rc = lib.oracle_refine(n, _ptr(alive), _ptr(vlabel), _ptr(graph), m, _ptr(src), _ptr(dst),
                           _ptr(elabel), k, cap, variant, DIRECTIONS[direction], _ptr(P), ctypes.byref(rounds),
                           ctypes.byref(executed), _ptr(hist), rows if history else 0)
    if rc != 0:
        raise ValueError(f"oracle_refine rejected its input (code {rc})")
    if history:
        return P, rounds.value, executed.value, hist[: rounds.value + 1]
    return P, rounds.value, executed.value


def refine_round(n, src, dst, elabel, vlabel, P, alive=None, graph=None, variant=VARIANT_DEFINITION,
                 direction="forward", label_filter=None):
    """One exact refinement round from partition P."""
    lib = _load()
    src, dst, elabel = _filtered(src, dst, elabel, label_filter)
    src, dst, elabel, vlabel, graph, P = map(_i32, (src, dst, elabel, vlabel, graph, P))
    alive = None if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
    out = np.empty(n, dtype=np.int32)
    rc = lib.oracle_round(n, _ptr(alive), _ptr(vlabel), _ptr(graph), len(src), _ptr(src),
                          _ptr(dst), _ptr(elabel), _ptr(P), variant, DIRECTIONS[direction], _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_round rejected its input (code {rc})")
    return out


def refine_round_range(n, src, dst, elabel, vlabel, P, v0, v1, out=None, alive=None, graph=None):
    """One exact round restricted to the vertices [v0, v1) (block ids: smallest
    vertex of the range with the same signature); `out` outside the range is
    left as it is. The CPU baseline times ranges of a large graph with it."""
    lib = _load()
    src, dst, elabel, vlabel, graph, P = map(_i32, (src, dst, elabel, vlabel, graph, P))
    alive = None if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
    out = np.full(n, -2, dtype=np.int32) if out is None else out
    rc = lib.oracle_round_range(n, _ptr(alive), _ptr(vlabel), _ptr(graph), len(src), _ptr(src), _ptr(dst),
                                _ptr(elabel), _ptr(P), int(v0), int(v1), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_round_range rejected its input (code {rc})")
    return out


def refine_round_threads(n, src, dst, elabel, P, threads=0, alive=None, graph=None):
    """The same round as refine_round on `threads` host threads (0: all of them);
    a CPU baseline that uses every core, pinned to refine_round by the tests."""
    lib = _load()
    src, dst, elabel, graph, P = map(_i32, (src, dst, elabel, graph, P))
    alive = None if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
    out = np.empty(n, dtype=np.int32)
    rc = lib.oracle_round_threads(n, _ptr(alive), _ptr(graph), len(src), _ptr(src), _ptr(dst), _ptr(elabel),
                                  _ptr(P), int(threads), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_round_threads rejected its input (code {rc})")
    return out


def literal_alg4(n, src, dst, elabel, vlabel, k, alive=None):
    """Algorithm 4 (Section 3.3.1) as printed, with exact identifiers.

    Two identifiers per vertex start from the label partition. For k = 1 one
    round gives id_s <- (own id_s, {(label, neighbour id_o)}). For k >= 2,
    rounds 1 .. k-1 give id_s <- (own id_s, {(label, neighbour id_s)}) and
    id_o <- {(label, neighbour id_o)} in round 1, {neighbour id_o} after it (no
    own term); the final round gives id_s <- (own id_s, {neighbour id_o}). A
    vertex that receives no message (no live out-edge) keeps its identifiers.
    Identifiers are compared exactly (the paper assumes unique hashes), so each
    is a partition; returns canonical ids (smallest member, -1 if dead).
    Plain Python: tuples and frozensets in dicts.
    """
    live = [True] * n if alive is None else [bool(a) for a in np.asarray(alive).tolist()]
    out = [[] for _ in range(n)]
    for u, w, l in zip(np.asarray(src).tolist(), np.asarray(dst).tolist(), np.asarray(elabel).tolist()):
        if live[u] and live[w]:
            out[u].append((int(l), w))

    def canon(key):
        first = {}
        return [first.setdefault(key(v), v) if live[v] else -1 for v in range(n)]

    ids = ido = canon(lambda v: int(vlabel[v]))
    if k == 0:
        return np.array(ids, np.int32)
    if k == 1:
        return np.array(canon(lambda v: (ids[v], frozenset((l, ido[w]) for l, w in out[v]))), np.int32)
    for i in range(1, k):
        new_s = canon(lambda v: (ids[v], frozenset((l, ids[w]) for l, w in out[v])))
        if i == 1:
            new_o = canon(lambda v: ("msg", frozenset((l, ido[w]) for l, w in out[v])) if out[v] else ("keep", ido[v]))
        else:
            new_o = canon(lambda v: ("msg", frozenset(ido[w] for _, w in out[v])) if out[v] else ("keep", ido[v]))
        ids, ido = new_s, new_o
    return np.array(canon(lambda v: (ids[v], frozenset(ido[w] for _, w in out[v]))), np.int32)


def summary_edges(src, dst, elabel, P, label_filter=None):
    """Edges of the summary graph of partition P (Section 2.6): one per distinct
    (P[u], l, P[w]) over the edges (u, w, l) whose endpoints are in a block,
    sorted lexicographically. Plain Python: a set of tuples."""
    src, dst, elabel = _filtered(src, dst, elabel, label_filter)
    out = set()
    for u, w, l in zip(np.asarray(src).tolist(), np.asarray(dst).tolist(), np.asarray(elabel).tolist()):
        a, b = int(P[u]), int(P[w])
        if a >= 0 and b >= 0:
            out.add((a, int(l), b))
    return sorted(out)


def block_sizes(P):
    """The count payload (Section 3.1): vertices per block id, 0 for ids that name no block."""
    sizes = [0] * len(P)
    for b in np.asarray(P).tolist():
        if b >= 0:
            sizes[b] += 1
    return np.array(sizes, dtype=np.int32)


def label_partition(n, vlabel, alive=None, graph=None):
    lib = _load()
    vlabel, graph = _i32(vlabel), _i32(graph)
    alive = None if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
    out = np.empty(n, dtype=np.int32)
    lib.oracle_label_partition(n, _ptr(alive), _ptr(vlabel), _ptr(graph), _ptr(out))
    return out


def refine_batched(b, k, cap=10_000):
    """Each graph of a batched set refined on its own; ids are graph-local minima."""
    vo, eo = b["vertex_offsets"], b["edge_offsets"]
    out = np.empty(int(vo[-1]), dtype=np.int32)
    for g in range(b["n_graphs"]):
        v0, v1, e0, e1 = int(vo[g]), int(vo[g + 1]), int(eo[g]), int(eo[g + 1])
        P, _, _ = refine(v1 - v0, b["src_local"][e0:e1], b["dst_local"][e0:e1],
                         b["elabel"][e0:e1], b["vlabel"][v0:v1], k, cap)
        out[v0:v1] = P
    return out


class UpdateRejected(ValueError):
    """A batch that names an invalid vertex or operation; nothing was applied."""


def apply_ops(state: dict, ops: np.ndarray) -> dict:
    """Apply an update batch with sequential semantics; returns a new state.

    state: dict(n, alive uint8[n], vlabel int32[n], src, dst, elabel int32[m]).
    ops:   int32 [n_ops, 4] rows (kind, a, b, label):
      EDGE_ADD (a -> b, label): both endpoints in range and alive, else the whole
                                 batch is rejected.
      EDGE_DEL (a -> b, label): removes one matching edge; a no-op if none exists.
      VERTEX_ADD (a, label):     makes a alive with this label (relabels if alive).
      VERTEX_DEL (a):            removes a and every edge incident to it.
    Ids out of range or unknown kinds reject the whole batch.
    """
    n = int(state["n"])
    alive = [bool(x) for x in state["alive"]]
    vlabel = [int(x) for x in state["vlabel"]]
    edges = list(zip((int(x) for x in state["src"]), (int(x) for x in state["dst"]),
                     (int(x) for x in state["elabel"])))
    # index: edge tuple -> list of live positions (a multiset)
    where: dict = {}
    for i, e in enumerate(edges):
        where.setdefault(e, []).append(i)
    live = [True] * len(edges)
    incident: dict = {}
    for i, (s, d, _) in enumerate(edges):
        incident.setdefault(s, []).append(i)
        if d != s:
            incident.setdefault(d, []).append(i)
    for row in np.asarray(ops, dtype=np.int64).reshape(-1, 4):
        kind, a, b, lab = (int(x) for x in row)
        if kind == OP_EDGE_ADD:
            if not (0 <= a < n and 0 <= b < n) or not alive[a] or not alive[b]:
                raise UpdateRejected(f"EDGE_ADD with invalid endpoint ({a}, {b})")
            i = len(edges)
            e = (a, b, lab)
            edges.append(e)
            live.append(True)
            where.setdefault(e, []).append(i)
            incident.setdefault(a, []).append(i)
            if b != a:
                incident.setdefault(b, []).append(i)
        elif kind == OP_EDGE_DEL:
            if not (0 <= a < n and 0 <= b < n):
                raise UpdateRejected(f"EDGE_DEL with out-of-range endpoint ({a}, {b})")
            lst = where.get((a, b, lab), [])
            while lst and not live[lst[-1]]:
                lst.pop()
            if lst:
                live[lst.pop()] = False
        elif kind == OP_VERTEX_ADD:
            if not (0 <= a < n):
                raise UpdateRejected(f"VERTEX_ADD with out-of-range vertex {a}")
            alive[a] = True
            vlabel[a] = lab
        elif kind == OP_VERTEX_DEL:
            if not (0 <= a < n):
                raise UpdateRejected(f"VERTEX_DEL with out-of-range vertex {a}")
            alive[a] = False
            for i in incident.get(a, []):
                live[i] = False
        else:
            raise UpdateRejected(f"unknown op kind {kind}")
    keep = [e for e, ok in zip(edges, live) if ok]
    arr = np.array(keep, dtype=np.int32).reshape(-1, 3)
    return dict(n=n, alive=np.array(alive, dtype=np.uint8), vlabel=np.array(vlabel, dtype=np.int32),
                src=arr[:, 0].copy(), dst=arr[:, 1].copy(), elabel=arr[:, 2].copy())


def apply_batches(state: dict, batches: list) -> tuple:
    """Apply update batches in order (C++ restatement of ``apply_ops`` for large graphs).

    A rejected batch changes nothing and the later ones still apply, as on
    the device. Returns (new state, list of rejected batch indices).
    """
    lib = _load()
    n = int(state["n"])
    alive = np.array(state["alive"], dtype=np.uint8, copy=True)
    vlabel = np.array(state["vlabel"], dtype=np.int32, copy=True)
    src, dst, lab = (_i32(state[k]) for k in ("src", "dst", "elabel"))
    ops = [np.ascontiguousarray(np.asarray(b, dtype=np.int32).reshape(-1, 4)) for b in batches]
    offsets = np.zeros(len(ops) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([len(o) for o in ops])
    allops = np.concatenate(ops) if ops else np.zeros((0, 4), np.int32)
    allops = np.ascontiguousarray(allops, dtype=np.int32)
    cap = len(src) + int(offsets[-1]) + 1
    osrc, odst, olab = (np.empty(cap, dtype=np.int32) for _ in range(3))
    out_m = ctypes.c_int64(0)
    rejected = np.zeros(max(1, len(ops)), dtype=np.uint8)
    rc = lib.oracle_apply_ops(n, _ptr(alive), _ptr(vlabel), len(src), _ptr(src), _ptr(dst), _ptr(lab), len(ops),
                              _ptr(offsets), _ptr(allops), cap, _ptr(osrc), _ptr(odst), _ptr(olab),
                              ctypes.byref(out_m), _ptr(rejected))
    if rc != 0:
        raise ValueError(f"oracle_apply_ops failed (code {rc})")
    k = out_m.value
    new = dict(n=n, alive=alive, vlabel=vlabel, src=osrc[:k].copy(), dst=odst[:k].copy(), elabel=olab[:k].copy())
    return new, [i for i in range(len(ops)) if rejected[i]]
