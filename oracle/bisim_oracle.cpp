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

using Pair = std::pair<int32_t, int32_t>;                       // (edge label, neighbour block)
using Signature = std::tuple<int32_t, int32_t, std::vector<Pair>>;  // (own a, own b, S)

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
// their sets of (edge label, neighbour block) agree.
void refine_round(const Graph& G, const int32_t* P, int32_t variant, int32_t* Pnext) {
    std::vector<std::vector<Pair>> S(G.n);
    for (int64_t e = 0; e < G.m; ++e) {
        int32_t v = G.src[e], w = G.dst[e];
        if (!G.is_alive(v) || !G.is_alive(w)) continue;
        if (variant & VARIANT_REVERSE) std::swap(v, w);
        int32_t l = (variant & VARIANT_DROP_EDGE_LABEL) ? 0 : G.elabel[e];
        S[v].emplace_back(l, P[w]);
    }
    for (int32_t v = 0; v < G.n; ++v) {
        std::sort(S[v].begin(), S[v].end());
        if (!(variant & VARIANT_MULTISET))
            S[v].erase(std::unique(S[v].begin(), S[v].end()), S[v].end());
    }
    std::map<Signature, int32_t> rep;
    for (int32_t v = 0; v < G.n; ++v) {
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
                  int32_t k, int32_t cap, int32_t variant,
                  int32_t* out_P, int32_t* out_rounds, int32_t* out_executed,
                  int32_t* history, int32_t history_rows) {
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
            refine_round(G, P.data(), variant, Q.data());
            P.swap(Q);
            ++executed;
            record(executed, P);
        }
        rounds = k;
    } else {
        rounds = cap;
        for (int32_t i = 0; i < cap; ++i) {
            refine_round(G, P.data(), variant, Q.data());
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
// from P_0 would take too long. If `vertex_begin < vertex_end` the signature
// map is built over all vertices but only [vertex_begin, vertex_end) is
// written -- the other entries of out_P are left untouched.
int oracle_round(int32_t n, const uint8_t* alive, const int32_t* vlabel, const int32_t* gid,
                 int64_t m, const int32_t* src, const int32_t* dst, const int32_t* elabel,
                 const int32_t* P, int32_t variant, int32_t* out_P) {
    if (n < 0 || m < 0) return 1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return 2;
    Graph G{n, alive, vlabel, gid, m, src, dst, elabel};
    refine_round(G, P, variant, out_P);
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
