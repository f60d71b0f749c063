// Batched contexts: one persistent kernel refines every graph of the batch
// (Algorithm 4's rounds, made exact as in the definition of Section 2.5).
//
// The work queue holds the graphs' vertex segments [voff[g], voff[g+1]) of the
// union, largest first; each CTA takes the next segment and runs that graph's
// rounds to the end (k rounds, or fewer once the graph's block count stops
// changing: then P_{i+1} = P_i and every later round repeats it), with CTA
// barriers between the phases, before it takes the next. Nothing waits on
// another CTA, so one launch refines the whole batch and the result of each
// graph is the one its solo run gives.
//
// One round of one graph:
//   signatures   a vertex alone in its block keeps it (every round refines the
//                last); the other rows are deduplicated in one thread (up to
//                16 edges, pair values in registers), one warp (up to 256, a
//                shared-memory set) or the whole CTA (a shared-memory set, in
//                sub-ranges of a mix of the values when the row is too long
//                for one pass). Rows of one thread insert their hash into the
//                table right away.
//   table        the graph's own region of the signature table; a slot keeps
//                the smallest vertex inserted with its fingerprint.
//   verification every listed vertex against its slot's vertex r: r itself is
//                a block id; otherwise equal own block, equal set size and
//                equal sets (in the thread for rows of up to 8 edges, in a warp
//                up to 32, in the CTA above). A mismatch is a hash collision:
//                the vertex is inserted again at the next level with another
//                salt. The smallest vertex of every slot is final at each level,
//                so the levels end.
// Data written inside the launch is never read through the read-only path:
// block ids with plain loads (a graph's are written and read by its own CTA,
// a barrier apart), the rest with L2 loads (__ldcg).
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

struct SegState {
    unsigned head;                  // next queue entry
    unsigned error;                 // kErr* bits
    unsigned long long blocks;      // blocks of the final partitions, all graphs
    unsigned long long levels;      // collision levels taken, all graphs and rounds
    int32_t rounds;                 // largest result r over the graphs
    int32_t executed;               // most rounds computed for one graph
};

namespace {

constexpr int kSegThreads = 512;
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegSlots = 8192;                         // the CTA's shared-memory set (64 KB)
constexpr int kSegWarpSlots = kSegSlots / kSegWarps;    // a warp's slice of it
constexpr int kSegThreadMax = 16;                       // rows deduplicated by one thread
constexpr int kSegWarpMax = kSegWarpSlots / 2;          // rows deduplicated by one warp
constexpr int kSegInlineMax = 8;                        // rows compared inside the verifying thread
constexpr int kSegSetLimit = kSegSlots * 3 / 4;         // distinct values one split pass of the CTA set may hold
constexpr uint32_t kSegMaxSplits = 1u << 12;
constexpr uint64_t kSaltSplit = 0x13198a2e03707344ull;
constexpr size_t kSegSmem = sizeof(unsigned long long) * kSegSlots;

struct SegArgs {
    const int64_t* voff;            // [G + 1] vertex segments of the union
    const int32_t* order;           // [G] queue: graphs, largest first
    int32_t G;
    const int64_t* re0;             // vertex -> first entry of its row in pe
    const int32_t* rdeg;            // vertex -> row length
    const unsigned long long* pe;   // rows as packed (label << 32 | target) entries (the round layout)
    const int32_t* P0;              // label partition
    int32_t* P[2];                  // round outputs; the final partition ends in P[0]
    unsigned long long* hash;       // [n] signature hash
    int32_t* cnt;                   // [n] |S_v|
    uint32_t* slot;                 // [n] table slot
    uint8_t* own;                   // [n] the vertex was its block's id in the last round
    uint8_t* joined;                // [n] another vertex joined its block in the last round
    int32_t* list[4];               // [n] each; a graph uses its own segment of every list
    Slot* slots;                    // table regions, one per graph
    const int64_t* rbase;
    const uint32_t* rmask;
    uint64_t hmask;                 // hash width mask
    int32_t limit;                  // rounds asked for (k, or the cap of a fixpoint run)
    int32_t fixpoint;
    SegState* st;
};

struct SegShared {
    unsigned n[4];                  // list lengths
    unsigned zero[kSegWarps + 1];   // "value 0 inserted" flags of the sets (per warp; the CTA's last)
    unsigned used;
    unsigned over;
    unsigned long long red_s;
    unsigned red_c;
    int32_t g;
};

__device__ __forceinline__ unsigned seg_lane() { return threadIdx.x & 31u; }

// The block ids of a graph are written and read by its own CTA only, with a
// CTA barrier in between, so the gathers may go through L1.
__device__ __forceinline__ uint64_t seg_pair(const SegArgs& A, const int32_t* Pin, int64_t e) {
    const unsigned long long pk = __ldg(A.pe + e);
    return pair_value(static_cast<int32_t>(pk >> 32), Pin[static_cast<uint32_t>(pk)]);
}

// First entry and length of v's row.
__device__ __forceinline__ int64_t seg_row(const SegArgs& A, int32_t v, int64_t& d) {
    d = __ldg(A.rdeg + v);
    return __ldg(A.re0 + v);
}

// Sub-range of a pair value when a set is built in several passes.
__device__ __forceinline__ uint32_t seg_sub(uint64_t mv, uint32_t splits) {
    return __umulhi(static_cast<uint32_t>(mix64(mv ^ kSaltSplit) >> 32), splits);
}

// Appends v for every lane with f (all 32 lanes call it together).
__device__ __forceinline__ void seg_append(bool f, int32_t v, int32_t* list, unsigned* n) {
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (b == 0u) return;
    const int leader = __ffs(b) - 1;
    unsigned at = 0;
    if (static_cast<int>(seg_lane()) == leader) at = atomicAdd(n, static_cast<unsigned>(__popc(b)));
    at = __shfl_sync(0xffffffffu, at, leader);
    if (f) list[at + __popc(b & ((1u << seg_lane()) - 1u))] = v;
}

__device__ __forceinline__ uint64_t seg_epoch(int& epoch, Slot* slots, int64_t base, uint32_t mask) {
    if (++epoch > static_cast<int>(kEpochCycle)) {      // the region's epochs are used up: clear it
        __syncthreads();
        for (uint32_t j = threadIdx.x; j <= mask; j += kSegThreads) slots[base + j].w = 0ull;
        __syncthreads();
        epoch = 1;
    }
    return static_cast<uint64_t>(epoch) << 32;
}

// Slots of the CTA set for one pass: a single pass over at most `values`
// distinct values gets twice that (so it cannot overflow); split passes get
// the whole set.
__device__ __forceinline__ uint32_t seg_set_size(uint32_t splits, int64_t values) {
    if (splits > 1) return kSegSlots;
    uint32_t sz = 64;
    while (sz < kSegSlots && static_cast<int64_t>(sz) < 2 * values) sz <<= 1;
    return sz;
}

// CTA-wide sum of (c, s); every thread gets the result.
__device__ __forceinline__ void seg_reduce(SegShared& S, unsigned& c, unsigned long long& s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (threadIdx.x == 0) {
        S.red_c = 0u;
        S.red_s = 0ull;
    }
    __syncthreads();
    if (seg_lane() == 0u) {
        atomicAdd(&S.red_c, c);
        atomicAdd(&S.red_s, s);
    }
    __syncthreads();
    c = S.red_c;
    s = S.red_s;
    __syncthreads();
}

// Size and wrap-around sum of the set of pair values of row [e0, e0 + d), by
// the whole CTA. The row's values are split into sub-ranges so that one pass
// holds at most kSegSetLimit distinct values; a pass that overflows restarts
// the row with twice as many sub-ranges. Returns false (and flags the error)
// if even kSegMaxSplits sub-ranges overflow.
__device__ bool seg_cta_set(const SegArgs& A, const int32_t* Pin, int64_t e0, int64_t d, unsigned long long* set,
                            SegShared& S, unsigned& out_c, unsigned long long& out_s) {
    uint32_t splits = 1;
    while (static_cast<int64_t>(splits) * (kSegSetLimit / 2) < d && splits < kSegMaxSplits) splits <<= 1;
    volatile unsigned* over = &S.over;
    for (; splits <= kSegMaxSplits; splits <<= 1) {
        const uint32_t SZ = seg_set_size(splits, d);
        unsigned c = 0;
        unsigned long long s = 0;
        bool o = false;
        for (uint32_t sub = 0; sub < splits && !o; ++sub) {
            for (uint32_t j = threadIdx.x; j < SZ; j += kSegThreads) set[j] = 0ull;
            if (threadIdx.x == 0) {
                S.zero[kSegWarps] = 0u;
                S.used = 0u;
                S.over = 0u;
            }
            __syncthreads();
            for (int64_t j = threadIdx.x; j < d; j += kSegThreads) {
                if (*over) break;
                const uint64_t mv = seg_pair(A, Pin, e0 + j);
                if (splits > 1 && seg_sub(mv, splits) != sub) continue;
                if (smem_set_insert(set, SZ - 1, &S.zero[kSegWarps], mv)) {
                    ++c;
                    s += mv;
                    if (atomicAdd(&S.used, 1u) + 1u > SZ / 4 * 3) *over = 1u;
                }
            }
            __syncthreads();
            o = __syncthreads_or(*over != 0u) != 0;
        }
        if (!o) {
            seg_reduce(S, c, s);
            out_c = c;
            out_s = s;
            return true;
        }
    }
    if (threadIdx.x == 0) atomicOr(&A.st->error, kErrHubFull);
    out_c = 0;
    out_s = 0;
    return false;
}

// Whether the set of row v equals the set of row r, given equal set sizes
// (then S_v inside S_r suffices), by the whole CTA; the same sub-range passes
// over r's values as seg_cta_set. Flags the error and answers false if no
// split fits.
__device__ bool seg_cta_equal(const SegArgs& A, const int32_t* Pin, int64_t ev, int64_t dv, int64_t er, int64_t dr,
                              int32_t c, unsigned long long* set, SegShared& S) {
    uint32_t splits = 1;
    while (static_cast<int64_t>(splits) * (kSegSetLimit / 2) < c && splits < kSegMaxSplits) splits <<= 1;
    volatile unsigned* over = &S.over;
    for (; splits <= kSegMaxSplits; splits <<= 1) {
        const uint32_t SZ = seg_set_size(splits, c);
        bool o = false, miss = false;
        for (uint32_t sub = 0; sub < splits && !o && !miss; ++sub) {
            for (uint32_t j = threadIdx.x; j < SZ; j += kSegThreads) set[j] = 0ull;
            if (threadIdx.x == 0) {
                S.zero[kSegWarps] = 0u;
                S.used = 0u;
                S.over = 0u;
            }
            __syncthreads();
            for (int64_t j = threadIdx.x; j < dr; j += kSegThreads) {
                if (*over) break;
                const uint64_t mv = seg_pair(A, Pin, er + j);
                if (splits > 1 && seg_sub(mv, splits) != sub) continue;
                if (smem_set_insert(set, SZ - 1, &S.zero[kSegWarps], mv) && atomicAdd(&S.used, 1u) + 1u > SZ / 4 * 3)
                    *over = 1u;
            }
            __syncthreads();
            o = __syncthreads_or(*over != 0u) != 0;
            bool my_miss = false;
            if (!o) {
                for (int64_t j = threadIdx.x; j < dv && !my_miss; j += kSegThreads) {
                    const uint64_t mv = seg_pair(A, Pin, ev + j);
                    if (splits > 1 && seg_sub(mv, splits) != sub) continue;
                    my_miss = !smem_set_contains(set, SZ - 1, S.zero[kSegWarps], mv);
                }
            }
            miss = __syncthreads_or(my_miss ? 1 : 0) != 0;
        }
        if (!o) return !miss;
    }
    if (threadIdx.x == 0) atomicOr(&A.st->error, kErrHubFull);
    return false;
}

// v joins the block of r (its representative) in P_{i+1}.
__device__ __forceinline__ void seg_join(const SegArgs& A, int32_t* Pout, int32_t v, int32_t r) {
    Pout[v] = r;
    A.joined[r] = 1;
}

// All rounds of graph g, by the whole CTA.
__device__ void seg_graph(const SegArgs& A, int32_t g, unsigned long long* set, SegShared& S) {
    const int tid = static_cast<int>(threadIdx.x);
    const int warp = tid >> 5;
    const unsigned lane = seg_lane();
    const int64_t v0 = __ldg(A.voff + g), v1 = __ldg(A.voff + g + 1);
    const int32_t ng = static_cast<int32_t>(v1 - v0);
    const int64_t base = __ldg(A.rbase + g);
    const uint32_t mask = __ldg(A.rmask + g);
    int32_t* Lall = A.list[0] + v0;       // round's listed vertices (level 0 input)
    int32_t* Lw = A.list[1] + v0;         // warp rows; then pairs for a warp comparison
    int32_t* Lc = A.list[2] + v0;         // CTA rows; then pairs for a CTA comparison
    int32_t* Lx = A.list[3] + v0;         // next collision level
    unsigned* err = &A.st->error;

    for (uint32_t j = tid; j <= mask; j += kSegThreads) A.slots[base + j].w = 0ull;
    for (int64_t v = v0 + tid; v < v1; v += kSegThreads) A.own[v] = 0;     // nobody is alone before the first round
    int epoch = 0;
    const int32_t* Pin = A.P0;
    int32_t* Pout = A.P[0];
    unsigned long long prev = 0, final_blocks = 0;
    int32_t rounds = A.limit, executed = 0;
    unsigned long long levels = 0;
    bool stopped = false;
    for (int32_t i = 0; i < A.limit; ++i) {
        Pout = A.P[i & 1];
        if (tid == 0) {
            S.n[0] = S.n[1] = S.n[2] = S.n[3] = 0u;
        }
        __syncthreads();
        TableRef t;
        t.slots = A.slots;
        t.mask = mask;
        t.hmask = A.hmask;
        t.epoch = seg_epoch(epoch, A.slots, base, mask);
        unsigned my_blocks = 0, my_prev = 0;
        // ---- signatures; rows of one thread go into the table right away
        for (int64_t b0 = v0; b0 < v1; b0 += kSegThreads) {
            const int64_t v = b0 + tid;
            const bool in = v < v1;
            bool listed = false, wrow = false, crow = false;
            if (in) {
                if (i == 0 && __ldg(A.P0 + v) == static_cast<int32_t>(v)) ++my_prev;
                const bool alone = __ldcg(A.own + v) != 0 && __ldcg(A.joined + v) == 0;
                if (alone) {
                    Pout[v] = static_cast<int32_t>(v);
                    ++my_blocks;
                } else {
                    listed = true;
                    A.own[v] = 0;
                    A.joined[v] = 0;
                    int64_t dl = 0;
                    const int64_t e0 = seg_row(A, static_cast<int32_t>(v), dl);
                    const int d = static_cast<int>(dl);
                    if (dl <= kSegThreadMax) {
                        uint64_t x[kSegThreadMax];
#pragma unroll
                        for (int j = 0; j < kSegThreadMax; ++j) x[j] = j < d ? seg_pair(A, Pin, e0 + j) : 0ull;
                        unsigned c = 0;
                        uint64_t s = 0;
#pragma unroll
                        for (int j = 0; j < kSegThreadMax; ++j) {
                            bool fresh = j < d;
#pragma unroll
                            for (int q = 0; q < j; ++q) fresh = fresh && x[q] != x[j];
                            if (fresh) {
                                ++c;
                                s += x[j];
                            }
                        }
                        const uint64_t h = sig_hash(Pin[v], c, s);
                        A.cnt[v] = static_cast<int32_t>(c);
                        A.hash[v] = h;
                        A.slot[v] = table_insert_in(t, level_hash(h, 0, t.hmask), static_cast<int32_t>(v), base, mask,
                                                    err);
                    } else if (dl <= kSegWarpMax) {
                        wrow = true;
                    } else {
                        crow = true;
                    }
                }
            }
            seg_append(listed, static_cast<int32_t>(v), Lall, &S.n[0]);
            seg_append(wrow, static_cast<int32_t>(v), Lw, &S.n[1]);
            seg_append(crow, static_cast<int32_t>(v), Lc, &S.n[2]);
        }
        __syncthreads();
        // ---- warp rows: one warp per row, a set in the warp's slice
        {
            unsigned long long* tab = set + warp * kSegWarpSlots;
            const unsigned nw = S.n[1];
            for (unsigned q = warp; q < nw; q += kSegWarps) {
                const int32_t v = Lw[q];
                int64_t dl = 0;
                const int64_t e0 = seg_row(A, v, dl);
                const int d = static_cast<int>(dl);
                uint32_t SZ = 64;
                while (SZ < 2u * static_cast<uint32_t>(d)) SZ <<= 1;
                for (uint32_t j = lane; j < SZ; j += 32) tab[j] = 0ull;
                if (lane == 0) S.zero[warp] = 0u;
                __syncwarp();
                unsigned c = 0;
                uint64_t s = 0;
                for (int j0 = 0; j0 < d; j0 += 32) {
                    const int j = j0 + static_cast<int>(lane);
                    bool fresh = false;
                    uint64_t mv = 0;
                    if (j < d) {
                        mv = seg_pair(A, Pin, e0 + j);
                        fresh = smem_set_insert(tab, SZ - 1, &S.zero[warp], mv);
                    }
                    c += static_cast<unsigned>(__popc(__ballot_sync(0xffffffffu, fresh)));
                    if (fresh) s += mv;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) {
                    const uint64_t h = sig_hash(Pin[v], c, s);
                    A.cnt[v] = static_cast<int32_t>(c);
                    A.hash[v] = h;
                    A.slot[v] = table_insert_in(t, level_hash(h, 0, t.hmask), v, base, mask, err);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // ---- CTA rows: the whole CTA per row
        {
            const unsigned nc = S.n[2];
            for (unsigned q = 0; q < nc; ++q) {
                const int32_t v = Lc[q];
                int64_t d = 0;
                const int64_t e0 = seg_row(A, v, d);
                unsigned c = 0;
                unsigned long long s = 0;
                seg_cta_set(A, Pin, e0, d, set, S, c, s);
                if (tid == 0) {
                    const uint64_t h = sig_hash(Pin[v], c, s);
                    A.cnt[v] = static_cast<int32_t>(c);
                    A.hash[v] = h;
                    A.slot[v] = table_insert_in(t, level_hash(h, 0, t.hmask), v, base, mask, err);
                }
                __syncthreads();
            }
        }
        __syncthreads();
        // ---- renumbering: verification, then the collision levels
        int32_t* cur = Lall;
        int32_t* nxt = Lx;
        unsigned count = S.n[0];
        uint32_t level = 0;
        for (;;) {
            if (level > 0) {
                t.epoch = seg_epoch(epoch, A.slots, base, mask);
                for (unsigned q = tid; q < count; q += kSegThreads) {
                    const int32_t v = cur[q];
                    A.slot[v] = table_insert_in(t, level_hash(__ldcg(A.hash + v), level, t.hmask), v, base, mask, err);
                }
            }
            if (tid == 0) S.n[1] = S.n[2] = S.n[3] = 0u;
            __syncthreads();
            for (unsigned b0 = 0; b0 < count; b0 += kSegThreads) {
                const unsigned q = b0 + tid;
                bool small = false, big = false, push = false;
                int32_t v = -1;
                if (q < count) {
                    v = cur[q];
                    const uint32_t sv = __ldcg(A.slot + v);
                    const int32_t r = sv == ~0u ? -1 : static_cast<int32_t>(static_cast<uint32_t>(__ldcg(&A.slots[sv].w)));
                    if (r < v0 || r >= v1) {                   // failed insert, reported through the error bits
                        atomicOr(err, kErrTableFull);
                        Pout[v] = -1;
                    } else if (r == v) {
                        Pout[v] = v;
                        A.own[v] = 1;
                        ++my_blocks;
                    } else if (Pin[v] != Pin[r] || __ldcg(A.cnt + v) != __ldcg(A.cnt + r)) {
                        push = true;
                    } else {
                        int64_t dv = 0, dr = 0;
                        const int64_t ev = seg_row(A, v, dv);
                        const int64_t er = seg_row(A, r, dr);
                        if (dv <= kSegInlineMax && dr <= kSegInlineMax) {
                            uint64_t y[kSegInlineMax];
#pragma unroll
                            for (int j = 0; j < kSegInlineMax; ++j) y[j] = j < dr ? seg_pair(A, Pin, er + j) : 0ull;
                            bool ok = true;
                            for (int64_t j = 0; j < dv && ok; ++j) {
                                const uint64_t a = seg_pair(A, Pin, ev + j);
                                bool f = false;
#pragma unroll
                                for (int k = 0; k < kSegInlineMax; ++k) f = f || (k < dr && y[k] == a);
                                ok = f;
                            }
                            if (ok) seg_join(A, Pout, v, r);
                            else push = true;
                        } else if (dv <= 32 && dr <= 32) {
                            small = true;
                        } else {
                            big = true;
                        }
                    }
                }
                seg_append(push, v, nxt, &S.n[3]);
                seg_append(small, v, Lw, &S.n[1]);
                seg_append(big, v, Lc, &S.n[2]);
            }
            __syncthreads();
            // pairs of rows of at most 32 edges: one warp per pair, lane j holds
            // the j-th value of each row
            {
                const unsigned ns = S.n[1];
                for (unsigned q = warp; q < ns; q += kSegWarps) {
                    const int32_t v = Lw[q];
                    const int32_t r = static_cast<int32_t>(static_cast<uint32_t>(__ldcg(&A.slots[__ldcg(A.slot + v)].w)));
                    int64_t dv = 0, dr = 0;
                    const int64_t ev = seg_row(A, v, dv);
                    const int64_t er = seg_row(A, r, dr);
                    const bool ha = lane < dv, hb = lane < dr;
                    const uint64_t a = ha ? seg_pair(A, Pin, ev + lane) : 0ull;
                    const uint64_t b = hb ? seg_pair(A, Pin, er + lane) : 0ull;
                    bool found = false;
                    for (int k = 0; k < static_cast<int>(dr); ++k) {
                        const uint64_t bk = __shfl_sync(0xffffffffu, b, k);   // every lane takes part in every shuffle
                        found = found || bk == a;
                    }
                    const bool miss = __any_sync(0xffffffffu, ha && !found);
                    seg_append(lane == 0 && miss, v, nxt, &S.n[3]);
                    if (lane == 0 && !miss) seg_join(A, Pout, v, r);
                }
            }
            // longer rows: the whole CTA per pair
            {
                const unsigned nb = S.n[2];
                for (unsigned q = 0; q < nb; ++q) {
                    const int32_t v = Lc[q];
                    const int32_t r = static_cast<int32_t>(static_cast<uint32_t>(__ldcg(&A.slots[__ldcg(A.slot + v)].w)));
                    int64_t dv = 0, dr = 0;
                    const int64_t ev = seg_row(A, v, dv);
                    const int64_t er = seg_row(A, r, dr);
                    const bool eq = seg_cta_equal(A, Pin, ev, dv, er, dr, __ldcg(A.cnt + r), set, S);
                    if (tid == 0) {
                        if (eq) seg_join(A, Pout, v, r);
                        else nxt[atomicAdd(&S.n[3], 1u)] = v;
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            count = S.n[3];
            if (count == 0u) break;
            ++level;
            ++levels;
            if (level > static_cast<uint32_t>(ng) + 1u) {     // cannot happen: every level settles a slot's vertex
                if (tid == 0) atomicOr(err, kErrTableFull);
                break;
            }
            int32_t* tmp = cur;
            cur = nxt;
            nxt = tmp;
            __syncthreads();
        }
        // ---- block count of P_{i+1}; the graph stops at its fixpoint
        unsigned c = my_blocks;
        unsigned long long pv = my_prev;
        seg_reduce(S, c, pv);
        if (i == 0) prev = pv;
        executed = i + 1;
        final_blocks = c;
        if (c == prev) {                     // P_{i+1} refines P_i with as many blocks: P_{i+1} = P_i
            rounds = A.fixpoint ? i : A.limit;
            stopped = true;
        }
        prev = c;
        Pin = Pout;
        __syncthreads();
        if (stopped) break;
    }
    if (executed == 0) {
        final_blocks = 0;
        unsigned c = 0;
        unsigned long long unused = 0;
        for (int64_t v = v0 + tid; v < v1; v += kSegThreads) {
            const int32_t p = __ldg(A.P0 + v);
            A.P[0][v] = p;
            c += p == static_cast<int32_t>(v) ? 1u : 0u;
        }
        seg_reduce(S, c, unused);
        final_blocks = c;
    } else if (Pout != A.P[0]) {
        for (int64_t v = v0 + tid; v < v1; v += kSegThreads) A.P[0][v] = __ldcg(Pout + v);
    }
    if (tid == 0) {
        atomicAdd(&A.st->blocks, final_blocks);
        if (levels) atomicAdd(&A.st->levels, levels);
        atomicMax(&A.st->rounds, rounds);
        atomicMax(&A.st->executed, executed);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSegThreads, 2) k_segments(const SegArgs A) {
    extern __shared__ unsigned long long set[];
    __shared__ SegShared S;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned q = atomicAdd(&A.st->head, 1u);
            S.g = q < static_cast<unsigned>(A.G) ? __ldg(A.order + q) : -1;
        }
        __syncthreads();
        const int32_t g = S.g;
        __syncthreads();
        if (g < 0) return;
        seg_graph(A, g, set, S);
    }
}

__global__ void k_seg_rows(const int32_t* __restrict__ vpos, const int64_t* __restrict__ prp, int32_t n,
                           int64_t* __restrict__ e0, int32_t* __restrict__ deg) {
    const int32_t v = static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v >= n) return;
    const int32_t p = vpos[v];
    const int64_t a = prp[p];
    e0[v] = a;
    deg[v] = static_cast<int32_t>(prp[p + 1] - a);
}

int seg_grid(int32_t G, bool beside_union) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_segments, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSegSmem));
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_segments, kSegThreads, kSegSmem) != cudaSuccess) b = 1;
        per_sm = std::max(b, 1);
        cudaGetLastError();
    }
    return static_cast<int>(std::min<int64_t>(G, static_cast<int64_t>(beside_union ? 1 : per_sm) * std::max(sms, 1)));
}

}  // namespace

bisim_status segment_init(bisim_ctx* ctx, const int64_t* voff_host, const int64_t* eoff_host, int32_t n_graphs,
                          cudaStream_t s) {
    // the queue: largest graphs first (by edges, then vertices), so that the
    // last graphs to start are the small ones
    std::vector<int32_t> order(n_graphs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const int64_t ea = eoff_host[a + 1] - eoff_host[a], eb = eoff_host[b + 1] - eoff_host[b];
        if (ea != eb) return ea > eb;
        return voff_host[a + 1] - voff_host[a] > voff_host[b + 1] - voff_host[b];
    });
    ctx->seg_sorted = order;
    ctx->seg_vcount.resize(n_graphs);
    for (int32_t g = 0; g < n_graphs; ++g) ctx->seg_vcount[g] = voff_host[g + 1] - voff_host[g];
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_order), sizeof(int32_t) * n_graphs, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_big), std::max<size_t>(n_graphs, 1), s)))
        return cuda_error(ctx, e, "alloc graph queue");
    ctx->seg_split = -1;
    return BISIM_OK;
}

// The persistent kernel's queue for a split: the graphs of at most `split`
// vertices, largest first; seg_big flags the others, which the union's round
// kernels refine beside it.
bisim_status segment_queue(bisim_ctx* ctx, int32_t split, cudaStream_t s) {
    if (ctx->seg_split == split) return BISIM_OK;
    const int32_t G = ctx->n_graphs;
    std::vector<int32_t> queue;
    std::vector<uint8_t> big(G, 0);
    queue.reserve(G);
    for (int32_t g : ctx->seg_sorted) {
        if (ctx->seg_vcount[g] <= split) queue.push_back(g);
        else big[g] = 1;
    }
    ctx->seg_n_small = static_cast<int32_t>(queue.size());
    if (!queue.empty())
        cudaMemcpyAsync(ctx->seg_order, queue.data(), sizeof(int32_t) * queue.size(), cudaMemcpyHostToDevice, s);
    if (G > 0) cudaMemcpyAsync(ctx->seg_big, big.data(), G, cudaMemcpyHostToDevice, s);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "upload graph queue");   // the host vectors die here
    ctx->seg_split = split;
    return BISIM_OK;
}

bool segment_usable(const bisim_ctx* ctx) {
    return ctx->gid != nullptr && ctx->rtable != nullptr && ctx->seg_order != nullptr &&
           !(ctx->opt.flags & BISIM_FLAG_UNION_ROUNDS);
}

bisim_status segment_rounds(bisim_ctx* ctx, int32_t k, int32_t cap, cudaStream_t s, int32_t* out_rounds,
                            int32_t* out_executed, int64_t* out_blocks) {
    const int32_t n = ctx->n;
    const bool fixpoint = k == BISIM_FIXPOINT;
    const int32_t limit = fixpoint ? cap : k;
    cudaError_t e;
    bisim_status pst = dense_prepare(ctx, s);        // the rows in the round layout (built by init)
    if (pst != BISIM_OK) return pst;
    if (ctx->seg_hash == nullptr) {
        const size_t nv = static_cast<size_t>(std::max(n, 1));
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_hash), sizeof(unsigned long long) * nv, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_own), nv, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_joined), nv, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_lists), sizeof(int32_t) * 4 * nv, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_state), sizeof(SegState), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_e0), sizeof(int64_t) * nv, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_deg), sizeof(int32_t) * nv, s)))
            return cuda_error(ctx, e, "alloc batched round state");
        if (ctx->seg_host == nullptr && (ctx->seg_host = pinned_take()) == nullptr)
            return set_error(ctx, BISIM_ENOMEM, "pinned host memory for the batched round state");
        ctx->stats.device_bytes = ctx->device_bytes;
    }
    if (ctx->opt.mem_budget_bytes > 0 && ctx->device_bytes > ctx->opt.mem_budget_bytes)
        return set_error(ctx, BISIM_ENOMEM, "context exceeds the memory budget");
    if (ctx->seg_rows_version != ctx->layout_version && n > 0) {
        // every vertex's row by vertex id (the layout keeps rows by position)
        BISIM_SITE(site_r, "segment_rows");
        Launch L(site_r, s, n, 0, 24.0 * n);
        k_seg_rows<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(ctx->dvpos, ctx->dprp, n, ctx->seg_e0,
                                                                         ctx->seg_deg);
        ctx->seg_rows_version = ctx->layout_version;
    }
    bisim_status st;
    if ((st = segment_queue(ctx, ctx->opt.batch_split, s)) != BISIM_OK) return st;
    const int32_t n_small = ctx->seg_n_small;
    const bool any_big = n_small < ctx->n_graphs;
    if (any_big && (n_small == 0 || limit <= 0)) {
        // every graph above the split: the union's round kernels alone
        int64_t prev = 0, dropped = 0, blocks = 0;
        int32_t rounds = 0, executed = 0;
        if ((st = dense_rounds_begin(ctx, s, nullptr, &prev, &dropped)) != BISIM_OK ||
            (st = dense_rounds_run(ctx, k, cap, s, prev, &rounds, &executed, &blocks, true)) != BISIM_OK)
            return st;
        ctx->cur_k = rounds;
        ctx->stats.rounds = rounds;
        ctx->stats.rounds_executed = executed;
        ctx->stats.num_blocks = blocks;
        *out_rounds = rounds;
        *out_executed = executed;
        *out_blocks = blocks;
        return BISIM_OK;
    }
    // graphs above the split (if any) go through the union's round kernels on
    // the caller's stream while the persistent kernel takes the others on a
    // second stream: the two touch disjoint vertices and table regions (the
    // persistent kernel's in a table of its own, since the union's rounds
    // clear theirs whole)
    const bool hybrid = any_big;
    int64_t prev_u = 0, dropped = 0;
    cudaStream_t ks = s;
    if (hybrid) {
        if ((st = dense_rounds_begin(ctx, s, ctx->seg_big, &prev_u, &dropped)) != BISIM_OK) return st;
        if (ctx->seg_table == nullptr &&
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->seg_table), sizeof(Slot) * ctx->n_rslots, s)))
            return cuda_error(ctx, e, "alloc the persistent kernel's table");
        if (ctx->seg_stream == nullptr &&
            ((e = cudaStreamCreateWithFlags(reinterpret_cast<cudaStream_t*>(&ctx->seg_stream), cudaStreamNonBlocking)) ||
             (e = cudaEventCreateWithFlags(reinterpret_cast<cudaEvent_t*>(&ctx->seg_events[0]), cudaEventDisableTiming)) ||
             (e = cudaEventCreateWithFlags(reinterpret_cast<cudaEvent_t*>(&ctx->seg_events[1]), cudaEventDisableTiming))))
            return cuda_error(ctx, e, "create the persistent kernel's stream");
        ctx->stats.device_bytes = ctx->device_bytes;
        if (ctx->opt.mem_budget_bytes > 0 && ctx->device_bytes > ctx->opt.mem_budget_bytes)
            return set_error(ctx, BISIM_ENOMEM, "context exceeds the memory budget");
        ks = static_cast<cudaStream_t>(ctx->seg_stream);
    }
    SegState* dst = static_cast<SegState*>(ctx->seg_state);
    SegState* hst = static_cast<SegState*>(ctx->seg_host);
    cudaMemsetAsync(dst, 0, sizeof(SegState), s);
    if (hybrid) {
        cudaEventRecord(static_cast<cudaEvent_t>(ctx->seg_events[0]), s);
        cudaStreamWaitEvent(ks, static_cast<cudaEvent_t>(ctx->seg_events[0]), 0);
    }
    if (limit > 0 && n > 0 && n_small > 0) {
        SegArgs A;
        A.voff = ctx->voff;
        A.order = ctx->seg_order;
        A.G = n_small;
        A.re0 = ctx->seg_e0;
        A.rdeg = ctx->seg_deg;
        A.pe = ctx->dpe;
        A.P0 = ctx->P0;
        A.P[0] = ctx->P[0];
        A.P[1] = ctx->P[1];
        A.hash = ctx->seg_hash;
        A.cnt = ctx->cnt;
        A.slot = ctx->slot;
        A.own = ctx->seg_own;
        A.joined = ctx->seg_joined;
        for (int i = 0; i < 4; ++i) A.list[i] = ctx->seg_lists + static_cast<int64_t>(i) * n;
        A.slots = hybrid ? ctx->seg_table : ctx->rtable;
        A.rbase = ctx->rbase;
        A.rmask = ctx->rmask;
        const int hb = ctx->opt.hash_bits;
        A.hmask = hb >= 64 ? ~0ull : ((1ull << hb) - 1ull);
        A.limit = limit;
        A.fixpoint = fixpoint ? 1 : 0;
        A.st = dst;
        BISIM_SITE(site, "segment_rounds");
        // algorithmic bytes of one round over every graph: the packed row
        // (label, target: 8 B) and its partition gather (4 B) per edge, and per
        // vertex its row offsets, partition reads and writes, hash, size, slot
        // and flags (about 40 B); rounds after the first skip settled vertices,
        // so this is an upper bound (none is counted when the union's kernels,
        // timed under their own sites, take part of the batch)
        Launch L(site, ks, n, ctx->m, hybrid ? 0.0 : static_cast<double>(limit) * (12.0 * ctx->m + 40.0 * n));
        // beside the union's kernels the persistent kernel keeps one CTA per SM
        k_segments<<<seg_grid(n_small, hybrid), kSegThreads, kSegSmem, ks>>>(A);
        if ((e = cudaGetLastError())) return cuda_error(ctx, e, "launch batched rounds");
    } else if (n > 0 && !hybrid) {
        cudaMemcpyAsync(ctx->P[0], ctx->P0, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    int32_t rounds_u = 0, executed_u = 0;
    int64_t blocks_u = 0;
    bisim_status st_u = BISIM_OK;
    if (hybrid) {
        cudaEventRecord(static_cast<cudaEvent_t>(ctx->seg_events[1]), ks);
        st_u = dense_rounds_run(ctx, k, cap, s, prev_u, &rounds_u, &executed_u, &blocks_u, true);
        cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(ctx->seg_events[1]), 0);   // also when the union failed
    }
    cudaMemcpyAsync(hst, dst, sizeof(SegState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "batched rounds");
    if (st_u != BISIM_OK) return st_u;
    if (hst->error & kErrHubFull) return set_error(ctx, BISIM_ETIMEOUT, "row set passes reached their split limit");
    if (hst->error) return set_error(ctx, BISIM_ETIMEOUT, "signature table probe limit reached");
    int32_t rounds = limit, executed = 0;
    int64_t blocks = ctx->last_blocks;
    if (limit > 0 && n == 0) {
        rounds = fixpoint ? 0 : limit;                  // no vertices: P_1 = P_0 at once
        executed = 1;
    } else if (limit > 0) {
        rounds = fixpoint ? hst->rounds : limit;
        executed = hst->executed;
        blocks = static_cast<int64_t>(hst->blocks);
        if (hybrid) {
            // the union's count holds the dropped live vertices as blocks
            rounds = fixpoint ? std::max(rounds, rounds_u) : limit;
            executed = std::max(executed, executed_u);
            blocks += blocks_u - dropped;
        }
    }
    ctx->cur = 0;
    ctx->cur_k = rounds;
    ctx->stats.rounds = rounds;
    ctx->stats.rounds_executed = executed;
    ctx->stats.num_blocks = blocks;
    ctx->stats.collision_levels += static_cast<int64_t>(hst->levels);
    *out_rounds = rounds;
    *out_executed = executed;
    *out_blocks = blocks;
    return BISIM_OK;
}

void segment_release(bisim_ctx* ctx) {
    if (ctx->seg_stream) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->seg_stream));
    for (void*& ev : ctx->seg_events) {
        if (ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
        ev = nullptr;
    }
    ctx->seg_stream = nullptr;
}

}  // namespace bisim
