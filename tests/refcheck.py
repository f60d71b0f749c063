"""Independent reference checks used to pin the oracle (pure Python, tiny inputs).

Nothing here calls the oracle or the CUDA path. Each routine restates a
different characterisation of the same partition:

* ``brute_force``: the pairwise relation of Section 2.5, iterated k times.
  R_0 relates vertices with equal labels; R_j keeps a pair (u, v) of R_{j-1}
  iff every l-edge of u is matched by an l-edge of v to an R_{j-1}-related
  target, and vice versa (the symmetric clause of the Complex Schema Element
  definition, Section 2.4.1).
* ``coarsest_stable``: the relational coarsest partition of Paige and Tarjan
  (cited in Section 2.5), computed by naive splitting: a block X is split by a
  splitter (B, l) into the vertices that have an l-edge into B and those that
  have none, until no splitter splits any block.
* ``parse_golden``: reader for the small text fixtures under tests/golden/.
"""

from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def canonical(ids) -> np.ndarray:
    """Relabel a partition (any ids; -1 = no block) so each block is named by its smallest member."""
    ids = list(ids)
    first = {}
    out = []
    for v, b in enumerate(ids):
        if b == -1:
            out.append(-1)
            continue
        if b not in first:
            first[b] = v
        out.append(first[b])
    return np.array(out, dtype=np.int32)


def brute_force(n, edges, vlabel, k, alive=None, direction="forward"):
    """Canonical ids of the k-bisimulation classes from the pairwise definition.

    direction: "forward" matches out-edges, "backward" in-edges (Section 2.5),
    "both" matches the out-edges and, separately, the in-edges."""
    alive = [True] * n if alive is None else [bool(a) for a in alive]
    out = [[] for _ in range(n)]
    for s, d, l in edges:
        if alive[s] and alive[d]:
            # the edge's label carries its direction as seen from the vertex
            if direction in ("forward", "both"):
                out[s].append(((l, "out"), d))
            if direction in ("backward", "both"):
                out[d].append(((l, "in"), s))
    R = [[alive[u] and alive[v] and vlabel[u] == vlabel[v] for v in range(n)] for u in range(n)]
    history = [R]
    for _ in range(k):
        R2 = [[False] * n for _ in range(n)]
        for u in range(n):
            for v in range(n):
                if not R[u][v]:
                    continue
                fwd = all(any(l2 == l and R[a][b] for (l2, b) in out[v]) for (l, a) in out[u])
                bwd = all(any(l2 == l and R[a][b] for (l2, a) in out[u]) for (l, b) in out[v])
                R2[u][v] = fwd and bwd
        R = R2
        history.append(R)
    res = []
    for Rj in history:
        ids = [(-1 if not alive[u] else min(v for v in range(n) if Rj[u][v])) for u in range(n)]
        res.append(np.array(ids, dtype=np.int32))
    return res


def coarsest_stable(n, edges, vlabel, alive=None):
    """Coarsest refinement of the label partition stable under every (block, label) splitter."""
    alive = [True] * n if alive is None else [bool(a) for a in alive]
    live_edges = [(s, d, l) for (s, d, l) in edges if alive[s] and alive[d]]
    labels = sorted({l for (_, _, l) in live_edges})
    block = {}
    nxt = 0
    bid = [-1] * n
    for v in range(n):
        if not alive[v]:
            continue
        key = vlabel[v]
        if key not in block:
            block[key] = nxt
            nxt += 1
        bid[v] = block[key]
    changed = True
    while changed:
        changed = False
        for B in sorted(set(b for b in bid if b >= 0)):
            for l in labels:
                pre = {s for (s, d, ll) in live_edges if ll == l and bid[d] == B}
                groups = {}
                for v in range(n):
                    if bid[v] >= 0:
                        groups.setdefault(bid[v], []).append(v)
                for X, members in groups.items():
                    inside = [v for v in members if v in pre]
                    if 0 < len(inside) < len(members):
                        for v in inside:
                            bid[v] = nxt
                        nxt += 1
                        changed = True
    return canonical(bid)


def parse_golden(name):
    """Read a fixture: n, edges, labelled modes, expectations and op rows."""
    g = dict(n=0, edges=[], vlabel={}, expect={}, ops={}, summary={}, sizes={})
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "n":
                g["n"] = int(tok[1])
            elif tok[0] == "edge":
                g["edges"].append(tuple(int(x) for x in tok[1:4]))
            elif tok[0] == "vlabel":
                g["vlabel"][tok[1]] = [int(x) for x in tok[2:]]
            elif tok[0] == "expect":
                g["expect"][(tok[1], int(tok[2]))] = np.array([int(x) for x in tok[3:]], dtype=np.int32)
            elif tok[0] == "op":
                g["ops"].setdefault(tok[1], []).append([int(x) for x in tok[2:6]])
            elif tok[0] == "summary":
                g["summary"].setdefault(int(tok[1]), []).append(tuple(int(x) for x in tok[2:5]))
            elif tok[0] == "sizes":
                g["sizes"][int(tok[1])] = np.array([int(x) for x in tok[2:]], dtype=np.int32)
    return g


def edges_to_arrays(edges):
    a = np.array(edges, dtype=np.int32).reshape(-1, 3)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()
