// CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, single-threaded restatement of forward k-bisimulation on a
// directed edge-labelled multigraph, written from the definition in the
// paper's Section 2.5 ("Bisimulation") together with the chaining
// parameterization (Definition "Chaining parameterization", Section 2.4.2) and
// the Complex Schema Element's "and vice versa" clause (Definition "Complex
// Schema Element", Section 2.4.1). Algorithm 4 (Section 3.3.1) claims to reach
// exactly this partition using hashed identifiers; the oracle therefore uses no
// hashing at all: every signature is kept whole as a sorted vector inside an
// ordered map.
//
// Only the test suite, the smoke check and the CPU-baseline leg of the bench
// may load this library. It shares no code, header, table or helper with the
// CUDA path.
//
// Definition followed (one int32 label per vertex, one per edge; UNTYPED = -1
// is an ordinary label of its own):
//
//   P_0[v]     = min { u alive : (g[u], L[u]) = (g[v], L[v]) }       (label partition)
//   S_i(v)     = set of pairs (l, P_i[w]) over out-edges (v, w, l)   (duplicates count once)
//                (backward: over in-edges (w, v, l); both: the two sets, each pair tagged
//                with its direction)
//   sig_i(v)   = (P_i[v], S_i(v))
//   P_{i+1}[v] = min { u alive : sig_i(u) = sig_i(v) }
//
// Block ids are canonical: the smallest vertex id in the block. Dead vertices
// get -1 and never appear in any block. g[] is an optional graph id used for a
// disjoint union of independent graphs, so that no block crosses two graphs.
//
// Fixpoint: the smallest r with P_{r+1} == P_r, capped at `cap`; the result is
// P_r and r (P_cap and cap if the cap is reached first).
//
// The `variant` bits exist so tests can plant a mistake in the oracle and show
// that the pins catch it; variant 0 is the definition. VARIANT_OWN_LABEL is the
// one legitimate alternative: it keys the own-state term on (g[v], L[v])
// instead of P_i[v], which yields the same partition (both refine P_0).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

namespace {

enum : int32_t {
    VARIANT_DEFINITION = 0,
    VARIANT_DROP_EDGE_LABEL = 1,   // planted mistake: pairs lose their edge label
    VARIANT_DROP_SELF = 2,         // planted mistake: own block not part of the signature
    VARIANT_REVERSE = 4,           // planted mistake: follows in-edges (backward bisimulation)
    VARIANT_MULTISET = 8,          // planted mistake: duplicates are not removed
    VARIANT_OWN_LABEL = 16,        // legitimate: own term is the vertex label, not P_i[v]
};

// (direction, edge label, neighbour block); direction 0 = an out-edge, 1 = an in-edge
using Pair = std::tuple<int32_t, int32_t, int32_t>;
using Signature = std::tuple<int32_t, int32_t, std::vector<Pair>>;  // (own a, own b, S)

// Which edges make up a vertex's set (Section 2.5: forward bisimulation uses
// outgoing edges, backward bisimulation incoming ones; both = the two sets
// together, each pair tagged with its direction).
enum : int32_t { DIR_FORWARD = 0, DIR_BACKWARD = 1, DIR_BOTH = 2 };

struct Graph {
    int32_t n;
    const uint8_t* alive;      // nullable: all alive
    const int32_t* vlabel;
    const int32_t* gid;        // nullable: one graph
    int64_t m;
    const int32_t* src;
    const int32_t* dst;
    const int32_t* elabel;

    bool is_alive(int32_t v) const { return alive == nullptr || alive[v] != 0; }
    int32_t graph_of(int32_t v) const { return gid == nullptr ? 0 : gid[v]; }
};

// P_0: vertices with equal (graph, label) share a block (Section 2.5, labelled variant).
void label_partition(const Graph& G, int32_t* P0) {
    std::map<std::pair<int32_t, int32_t>, int32_t> first;
    for (int32_t v = 0; v < G.n; ++v) {
        if (!G.is_alive(v)) { P0[v] = -1; continue; }
        auto key = std::make_pair(G.graph_of(v), G.vlabel[v]);
        auto it = first.find(key);
        if (it == first.end()) it = first.emplace(key, v).first;   // ascending v: first is min
        P0[v] = it->second;
    }
}

// One refinement round: vertices stay together iff they were together and
// their sets of (direction, edge label, neighbour block) agree. Only the
// vertices of [v0, v1) are refined (the whole round is [0, n)); a vertex range
// lets the CPU baseline time a bounded part of a large graph's round.
void refine_round(const Graph& G, const int32_t* P, int32_t variant, int32_t* Pnext, int32_t v0, int32_t v1,
                  int32_t direction = DIR_FORWARD) {
    std::vector<std::vector<Pair>> S(G.n);
    for (int64_t e = 0; e < G.m; ++e) {
        int32_t v = G.src[e], w = G.dst[e];
        if (!G.is_alive(v) || !G.is_alive(w)) continue;
        if (variant & VARIANT_REVERSE) std::swap(v, w);
        int32_t l = (variant & VARIANT_DROP_EDGE_LABEL) ? 0 : G.elabel[e];
        if (direction != DIR_BACKWARD && v >= v0 && v < v1) S[v].emplace_back(0, l, P[w]);   // out-edge of v
        if (direction != DIR_FORWARD && w >= v0 && w < v1) S[w].emplace_back(1, l, P[v]);    // in-edge of w
    }
    for (int32_t v = v0; v < v1; ++v) {
        std::sort(S[v].begin(), S[v].end());
        if (!(variant & VARIANT_MULTISET))
            S[v].erase(std::unique(S[v].begin(), S[v].end()), S[v].end());
    }
    std::map<Signature, int32_t> rep;
    for (int32_t v = v0; v < v1; ++v) {
        if (!G.is_alive(v)) { Pnext[v] = -1; continue; }
        int32_t a = P[v], b = 0;
        if (variant & VARIANT_OWN_LABEL) { a = G.graph_of(v); b = G.vlabel[v]; }
        if (variant & VARIANT_DROP_SELF) { a = 0; b = 0; }
        Signature sig(a, b, std::move(S[v]));
        auto it = rep.find(sig);
        if (it == rep.end()) it = rep.emplace(std::move(sig), v).first;  // ascending v: min
        Pnext[v] = it->second;
    }
}

bool same(const std::vector<int32_t>& a, const std::vector<int32_t>& b) { return a == b; }

}  // namespace

extern "C" {

// Returns 0 on success, nonzero on invalid arguments.
// k >= 0: run exactly k rounds. k < 0: run to the fixpoint (at most `cap` rounds).
// out_P: int32[n]. out_rounds: k, or the fixpoint round r. out_executed: rounds
// actually computed (k, r+1 when the fixpoint was detected, or cap).
// history: nullable int32[(max_rounds+1) * n]; row i receives P_i.
int oracle_refine(int32_t n, const uint8_t* alive, const int32_t* vlabel, const int32_t* gid,
                  int64_t m, const int32_t* src, const int32_t* dst, const int32_t* elabel,
                  int32_t k, int32_t cap, int32_t variant, int32_t direction,
                  int32_t* out_P, int32_t* out_rounds, int32_t* out_executed,
                  int32_t* history, int32_t history_rows) {
    if (direction < DIR_FORWARD || direction > DIR_BOTH) return 1;
    if (n < 0 || m < 0 || (n > 0 && (vlabel == nullptr || out_P == nullptr))) return 1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return 2;
    Graph G{n, alive, vlabel, gid, m, src, dst, elabel};
    std::vector<int32_t> P(n), Q(n);
    label_partition(G, P.data());
    auto record = [&](int32_t row, const std::vector<int32_t>& X) {
        if (history != nullptr && row < history_rows)
            std::memcpy(history + static_cast<int64_t>(row) * n, X.data(), sizeof(int32_t) * n);
    };
    record(0, P);
    int32_t rounds = 0, executed = 0;
    if (k >= 0) {
        for (int32_t i = 0; i < k; ++i) {
            refine_round(G, P.data(), variant, Q.data(), 0, n, direction);
            P.swap(Q);
            ++executed;
            record(executed, P);
        }
        rounds = k;
    } else {
        rounds = cap;
        for (int32_t i = 0; i < cap; ++i) {
            refine_round(G, P.data(), variant, Q.data(), 0, n, direction);
            ++executed;
            if (same(P, Q)) { rounds = i; break; }
            P.swap(Q);
            record(executed, P);
        }
    }
    if (n > 0) std::memcpy(out_P, P.data(), sizeof(int32_t) * n);
    if (out_rounds) *out_rounds = rounds;
    if (out_executed) *out_executed = executed;
    return 0;
}

// One round from a given partition P (int32[n], -1 for dead vertices):
// writes P_next. Used to check a refinement round at sizes where a full run
// from P_0 would take too long.
int oracle_round(int32_t n, const uint8_t* alive, const int32_t* vlabel, const int32_t* gid,
                 int64_t m, const int32_t* src, const int32_t* dst, const int32_t* elabel,
                 const int32_t* P, int32_t variant, int32_t direction, int32_t* out_P) {
    if (n < 0 || m < 0 || direction < DIR_FORWARD || direction > DIR_BOTH) return 1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return 2;
    Graph G{n, alive, vlabel, gid, m, src, dst, elabel};
    refine_round(G, P, variant, out_P, 0, n, direction);
    return 0;
}

// The same round restricted to the vertices [v0, v1): their signatures over
// the whole P, each numbered by the smallest vertex of the range with the same
// signature; out_P outside the range is left untouched. On [0, n) it is
// oracle_round. The CPU baseline times consecutive ranges of a large graph as
// bounded samples of one round (the per-vertex work is the round's; only the
// map is smaller).
int oracle_round_range(int32_t n, const uint8_t* alive, const int32_t* vlabel, const int32_t* gid,
                       int64_t m, const int32_t* src, const int32_t* dst, const int32_t* elabel,
                       const int32_t* P, int32_t v0, int32_t v1, int32_t* out_P) {
    if (n < 0 || m < 0 || v0 < 0 || v1 > n || v0 > v1) return 1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return 2;
    Graph G{n, alive, vlabel, gid, m, src, dst, elabel};
    refine_round(G, P, VARIANT_DEFINITION, out_P, v0, v1);
    return 0;
}

// The label partition P_0 alone.
int oracle_label_partition(int32_t n, const uint8_t* alive, const int32_t* vlabel,
                           const int32_t* gid, int32_t* out_P) {
    if (n < 0) return 1;
    Graph G{n, alive, vlabel, gid, 0, nullptr, nullptr, nullptr};
    label_partition(G, out_P);
    return 0;
}

}  // extern "C"

// Update batches with sequential semantics (the incremental setting of Section
// 3.2: additions, deletions and modifications of vertices and edges), restated
// for graphs too large for the Python restatement `apply_ops`, which it must
// agree with:
//   EDGE_ADD (a, b, l)  both endpoints in range and alive at that point of the
//                        batch, else the whole batch is rejected
//   EDGE_DEL (a, b, l)  removes one live edge (a, b, l); nothing if none is left
//   VERTEX_ADD (a, l)   makes a alive with label l (relabels a live vertex)
//   VERTEX_DEL (a)      makes a dead and removes every live edge at a
// Ids out of range or unknown kinds reject the batch. A rejected batch changes
// nothing; the others apply in order. Edges come out in input order (removed
// ones dropped) followed by the added ones still live.
namespace {

struct EdgeKey {
    int32_t s, d, l;
    bool operator<(const EdgeKey& o) const { return std::tie(s, d, l) < std::tie(o.s, o.d, o.l); }
};

}  // namespace

extern "C" int oracle_apply_ops(int32_t n, uint8_t* alive, int32_t* vlabel, int64_t m, const int32_t* src,
                                const int32_t* dst, const int32_t* elab, int32_t n_batches,
                                const int64_t* batch_offsets, const int32_t* ops, int64_t cap, int32_t* out_src,
                                int32_t* out_dst, int32_t* out_label, int64_t* out_m, uint8_t* rejected) {
    if (n < 0 || m < 0 || n_batches < 0) return 1;
    std::vector<int32_t> es(src, src + m), ed(dst, dst + m), el(elab, elab + m);
    std::vector<uint8_t> live(static_cast<size_t>(m), 1);
    // only the keys some EDGE_DEL names and the vertices some VERTEX_DEL names need an index
    std::set<EdgeKey> del_keys;
    std::set<int32_t> del_vertices;
    const int64_t total = batch_offsets[n_batches];
    for (int64_t i = 0; i < total; ++i) {
        const int32_t* o = ops + 4 * i;
        if (o[0] == 1) del_keys.insert(EdgeKey{o[1], o[2], o[3]});
        if (o[0] == 3) del_vertices.insert(o[1]);
    }
    std::map<EdgeKey, std::vector<int64_t>> by_key;      // live edge indices per named key
    std::map<int32_t, std::vector<int64_t>> incident;    // edge indices per named vertex
    auto index_edge = [&](int64_t i) {
        const EdgeKey k{es[i], ed[i], el[i]};
        if (del_keys.count(k)) by_key[k].push_back(i);
        if (del_vertices.count(es[i])) incident[es[i]].push_back(i);
        if (ed[i] != es[i] && del_vertices.count(ed[i])) incident[ed[i]].push_back(i);
    };
    for (int64_t i = 0; i < m; ++i) index_edge(i);
    for (int32_t b = 0; b < n_batches; ++b) {
        const int64_t lo = batch_offsets[b], hi = batch_offsets[b + 1];
        // dry run: the alive state each op sees, and the ops' validity
        std::map<int32_t, uint8_t> shadow;
        auto is_alive = [&](int32_t v) {
            auto it = shadow.find(v);
            return it != shadow.end() ? it->second != 0 : alive[v] != 0;
        };
        bool ok = true;
        for (int64_t i = lo; i < hi && ok; ++i) {
            const int32_t* o = ops + 4 * i;
            const int32_t kind = o[0], a = o[1], c = o[2];
            const bool ra = a >= 0 && a < n, rc = c >= 0 && c < n;
            if (kind == 0) ok = ra && rc && is_alive(a) && is_alive(c);
            else if (kind == 1) ok = ra && rc;
            else if (kind == 2) { ok = ra; if (ok) shadow[a] = 1; }
            else if (kind == 3) { ok = ra; if (ok) shadow[a] = 0; }
            else ok = false;
        }
        rejected[b] = ok ? 0 : 1;
        if (!ok) continue;
        for (int64_t i = lo; i < hi; ++i) {
            const int32_t* o = ops + 4 * i;
            const int32_t kind = o[0], a = o[1], c = o[2], l = o[3];
            if (kind == 0) {
                es.push_back(a);
                ed.push_back(c);
                el.push_back(l);
                live.push_back(1);
                index_edge(static_cast<int64_t>(es.size()) - 1);
            } else if (kind == 1) {
                auto it = by_key.find(EdgeKey{a, c, l});
                if (it == by_key.end()) continue;
                std::vector<int64_t>& lst = it->second;
                while (!lst.empty() && !live[lst.back()]) lst.pop_back();
                if (!lst.empty()) {
                    live[lst.back()] = 0;
                    lst.pop_back();
                }
            } else if (kind == 2) {
                alive[a] = 1;
                vlabel[a] = l;
            } else {
                alive[a] = 0;
                auto it = incident.find(a);
                if (it != incident.end())
                    for (int64_t e : it->second) live[e] = 0;
            }
        }
    }
    int64_t k = 0;
    for (size_t i = 0; i < es.size(); ++i) {
        if (!live[i]) continue;
        if (k >= cap) return 2;
        out_src[k] = es[i];
        out_dst[k] = ed[i];
        out_label[k] = el[i];
        ++k;
    }
    *out_m = k;
    return 0;
}
