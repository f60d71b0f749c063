// CPU BASELINE ON ALL HOST CORES -- TEST AND BENCHMARK INFRASTRUCTURE ONLY.
//
// One refinement round of the oracle's definition (Section 2.5 with the
// chaining parameterization of Section 2.4.2; see bisim_oracle.cpp) computed
// by several host threads, so that the benchmark can report a CPU number that
// uses every core next to the single-threaded oracle. The arithmetic is the
// oracle's, unchanged: whole signatures (own block, sorted unique vector of
// (edge label, neighbour block) pairs) in ordered maps, no hashing decides
// anything. Only the work is divided:
//
//   1. the out-edges' pairs are gathered per source vertex (edge ranges per
//      thread; counts, a prefix sum and a second pass that places each pair);
//   2. every vertex's pairs are sorted and deduplicated (vertex ranges);
//   3. each vertex is given a shard by a hash of its signature, which only
//      decides which thread handles it;
//   4. each thread builds the ordered map of its shard, visiting its vertices
//      in ascending order, so the first vertex that inserts a signature is the
//      smallest one: P_{i+1}[v] = min{u : sig(u) = sig(v)} as in the oracle.
//
// Equal signatures always fall into the same shard, so the result is the
// oracle's round exactly; tests/test_oracle_pins.py checks that on random
// graphs. Shares no code with the CUDA path.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

namespace {

using Pair = std::pair<int32_t, int32_t>;
using Signature = std::pair<int32_t, std::vector<Pair>>;

template <class F>
void run_threads(int32_t threads, F&& body) {
    std::vector<std::thread> pool;
    for (int32_t t = 1; t < threads; ++t) pool.emplace_back(body, t);
    body(0);
    for (auto& th : pool) th.join();
}

// FNV-1a over the signature's integers: picks the shard, nothing else.
uint64_t shard_hash(int32_t own, const std::vector<Pair>& s) {
    uint64_t h = 1469598103934665603ull;
    auto add = [&h](uint32_t x) {
        for (int b = 0; b < 4; ++b) {
            h ^= (x >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    add(static_cast<uint32_t>(own));
    for (const Pair& p : s) {
        add(static_cast<uint32_t>(p.first));
        add(static_cast<uint32_t>(p.second));
    }
    return h;
}

}  // namespace

extern "C" {

// One round from P (int32[n], -1 for dead vertices) on `threads` host threads
// (0: all hardware threads); writes P_next. Returns 0, or nonzero for invalid
// arguments. alive and gid (a graph id per vertex, so that no block crosses
// two graphs) are nullable.
int oracle_round_threads(int32_t n, const uint8_t* alive, const int32_t* gid, int64_t m, const int32_t* src,
                         const int32_t* dst, const int32_t* elabel, const int32_t* P, int32_t threads,
                         int32_t* out_P) {
    if (n < 0 || m < 0) return 1;
    if (threads <= 0) threads = static_cast<int32_t>(std::max(1u, std::thread::hardware_concurrency()));
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return 2;
    auto live = [&](int32_t v) { return alive == nullptr || alive[v] != 0; };
    auto erange = [&](int32_t t) {
        return std::make_pair(m * t / threads, m * (t + 1) / threads);
    };
    auto vrange = [&](int32_t t) {
        return std::make_pair(static_cast<int32_t>(int64_t{n} * t / threads),
                              static_cast<int32_t>(int64_t{n} * (t + 1) / threads));
    };

    // 1. pairs per source vertex
    std::vector<std::atomic<int64_t>> cnt(static_cast<size_t>(n) + 1);
    for (auto& c : cnt) c.store(0, std::memory_order_relaxed);
    run_threads(threads, [&](int32_t t) {
        const auto r = erange(t);
        for (int64_t e = r.first; e < r.second; ++e)
            if (live(src[e]) && live(dst[e])) cnt[src[e]].fetch_add(1, std::memory_order_relaxed);
    });
    std::vector<int64_t> off(static_cast<size_t>(n) + 1, 0);
    for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v].load(std::memory_order_relaxed);
    for (int32_t v = 0; v < n; ++v) cnt[v].store(off[v], std::memory_order_relaxed);
    std::vector<Pair> pairs(static_cast<size_t>(off[n]));
    run_threads(threads, [&](int32_t t) {
        const auto r = erange(t);
        for (int64_t e = r.first; e < r.second; ++e) {
            const int32_t v = src[e], w = dst[e];
            if (!live(v) || !live(w)) continue;
            pairs[cnt[v].fetch_add(1, std::memory_order_relaxed)] = Pair(elabel[e], P[w]);
        }
    });

    // 2. sorted unique sets; 3. shards
    std::vector<int64_t> len(n);
    std::vector<uint32_t> shard(n);
    run_threads(threads, [&](int32_t t) {
        const auto r = vrange(t);
        for (int32_t v = r.first; v < r.second; ++v) {
            auto b = pairs.begin() + off[v], e = pairs.begin() + off[v + 1];
            std::sort(b, e);
            len[v] = std::unique(b, e) - b;
            if (live(v)) {
                std::vector<Pair> s(b, b + len[v]);
                const int32_t g = gid == nullptr ? 0 : gid[v];
                shard[v] = static_cast<uint32_t>((shard_hash(P[v], s) ^ (static_cast<uint64_t>(g) << 17)) % threads);
            }
        }
    });

    // 4. one ordered map per shard, vertices in ascending order
    run_threads(threads, [&](int32_t t) {
        std::map<std::pair<int32_t, Signature>, int32_t> rep;
        for (int32_t v = 0; v < n; ++v) {
            if (!live(v)) {
                if (t == 0) out_P[v] = -1;
                continue;
            }
            if (shard[v] != static_cast<uint32_t>(t)) continue;
            const int32_t g = gid == nullptr ? 0 : gid[v];
            std::vector<Pair> s(pairs.begin() + off[v], pairs.begin() + off[v] + len[v]);
            auto key = std::make_pair(g, Signature(P[v], std::move(s)));
            auto it = rep.find(key);
            if (it == rep.end()) it = rep.emplace(std::move(key), v).first;
            out_P[v] = it->second;
        }
    });
    return 0;
}

}  // extern "C"
