// One refinement round of forward k-bisimulation (Algorithm 4, Section 3.3.1),
// made exact.
//
// Per round i -> i+1 every live vertex v
//   1. gathers the pairs (l, P_i[w]) of its out-edges (SignalMessages: a pull over
//      the out-CSR instead of messages pushed along reversed edges),
//   2. removes duplicates (MergeMessages) -- by sorting for small and mid
//      degrees, by a per-hub hash set for hubs,
//   3. hashes (P_i[v], set) order-independently (Hash, with the own block in the
//      role of the paper's (self, old id) tuple),
//   4. inserts the hash into an open-addressing table whose slots keep the
//      smallest vertex id seen (FindAndMerge; canonical id = smallest member).
// A verification pass then compares every vertex's full signature with that of
// its block representative. Vertices whose signature differs (a hash
// collision) move to the next "level", where only they are re-hashed with a
// new salt; the group containing each level's smallest vertex is final, so
// every level resolves at least one group per colliding hash and the loop ends
// with the exact partition.
#include <algorithm>
#include <climits>
#include <cstring>
#include <tuple>

#include "common.cuh"
#include "prof.cuh"
#include "rows.cuh"

namespace bisim {

namespace {

constexpr int kMaxLevels = 1 << 16;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, cdiv(n, threads)));
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// ----------------------------------------------------------------------------- views

// Rows come from the CSR (row v = [rp[v], rp[v + 1]) of col / elab) or from the
// incremental path's row store (row v = rl[v] packed entries from rp[v], some
// deleted, some pointing at dead vertices: those do not count).
struct GraphView {
    const int64_t* rp;
    const int32_t* rl;                 // store row lengths (null: CSR)
    const int32_t* col;
    const int32_t* elab;
    const unsigned long long* pe;      // store entries (null: CSR)
    const int32_t* P;                  // P_i (-1 for a dead vertex)
    unsigned long long* hout;          // nullable: receives each vertex's signature hash
};

__device__ __forceinline__ int row_len(const GraphView& G, int32_t v) {
    return G.rl ? G.rl[v] : static_cast<int>(G.rp[v + 1] - G.rp[v]);
}

// Pair value of row entry e; false when the entry does not count.
__device__ __forceinline__ bool entry_value(const GraphView& G, int64_t e, unsigned long long* mv) {
    if (G.pe) {
        const unsigned long long x = __ldcs(G.pe + e);
        if (x == kRowTomb) return false;
        const int32_t p = __ldg(G.P + static_cast<int32_t>(static_cast<uint32_t>(x)));
        if (p < 0) return false;
        *mv = pair_value(static_cast<int32_t>(x >> 32), p);
        return true;
    }
    *mv = pair_value(__ldcs(G.elab + e), __ldg(G.P + __ldcs(G.col + e)));
    return true;
}

struct HubView {
    const int32_t* hub_list;   // ascending vertex ids
    int64_t n_hub;
    const int64_t* toff;
    const uint32_t* tmask;
    const unsigned long long* tab;
    const HubAcc* acc;
};

__device__ __forceinline__ int64_t hub_index(const HubView& H, int32_t v) {
    int64_t lo = 0, hi = H.n_hub - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (H.hub_list[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool hub_contains(const HubView& H, int64_t h, unsigned long long mv) {
    if (mv == 0ull) return H.acc[h].zero != 0u;
    const unsigned long long* tab = H.tab + H.toff[h];
    const uint32_t mask = H.tmask[h];
    uint32_t pos = static_cast<uint32_t>(mv) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = tab[pos];
        if (cur == mv) return true;
        if (cur == 0ull) return false;
        pos = (pos + 1) & mask;
    }
    return false;
}

// Full signature of a vertex: (P_i[v], the set of its pair values).
struct SigMode {
    static constexpr const char* kVerifySite = "verify";
    static constexpr double kVerifyBytesPerVertex = 20.0;   // slot 16 B read + P_{i+1} 4 B write
    GraphView G;
    const int32_t* cnt;
    const unsigned long long* skey;
    HubView H;
    int small_max, mid_max;

    __device__ uint64_t hash0(int32_t v) const {
        const int32_t c = cnt[v];
        const unsigned long long* l = skey + G.rp[v];
        uint64_t sum = 0;
        for (int32_t j = 0; j < c; ++j) sum += l[j];
        return sig_hash(G.P[v], static_cast<uint32_t>(c), sum);
    }

    static constexpr bool kDefers = true;

    // Exact comparison: 1 equal, 0 different, 2 left to the set comparison of
    // k_verify_deferred. Lists of vertices on the thread-per-vertex path are
    // sorted by pair value, so two of them are equal sets iff they are equal
    // element by element; every other list is in arrival order.
    __device__ int compare(int32_t v, int32_t r) const {
        if (G.P[v] != G.P[r]) return 0;
        const int32_t c = cnt[v];
        if (c != cnt[r]) return 0;
        const int64_t bv = G.rp[v], br = G.rp[r];
        const int64_t dv = row_len(G, v), dr = row_len(G, r);
        const bool sorted = (dv == 0 || dv <= small_max) && (dr == 0 || dr <= small_max);
        if (!sorted) return 2;
        const unsigned long long* lv = skey + bv;
        const unsigned long long* lr = skey + br;
        {
            // independent loads, four pairs per step, no early exit inside a step
            int32_t j = 0;
            for (; j + 4 <= c; j += 4) {
                const unsigned long long a0 = lv[j], a1 = lv[j + 1], a2 = lv[j + 2], a3 = lv[j + 3];
                const unsigned long long b0 = lr[j], b1 = lr[j + 1], b2 = lr[j + 2], b3 = lr[j + 3];
                if (((a0 ^ b0) | (a1 ^ b1) | (a2 ^ b2) | (a3 ^ b3)) != 0ull) return 0;
            }
            for (; j < c; ++j)
                if (lv[j] != lr[j]) return 0;
            return 1;
        }
    }
};

// Label partition P_0: key (graph id, vertex label).
struct LabelMode {
    static constexpr const char* kVerifySite = "label_verify";
    static constexpr double kVerifyBytesPerVertex = 20.0;
    const int32_t* vlabel;
    const int32_t* gid;   // may be null

    static constexpr bool kDefers = false;
    __device__ uint64_t hash0(int32_t v) const { return label_hash(gid ? gid[v] : 0, vlabel[v]); }
    __device__ int compare(int32_t v, int32_t r) const {
        return vlabel[v] == vlabel[r] && (gid == nullptr || gid[v] == gid[r]) ? 1 : 0;
    }
};

// ----------------------------------------------------------------------------- signature kernels

template <int D>
__device__ __forceinline__ void bitonic_regs(uint64_t (&s)[D]) {
#pragma unroll
    for (int k = 2; k <= D; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint64_t a = s[i], b = s[l];
                    const bool sw = up ? (a > b) : (a < b);
                    s[i] = sw ? b : a;
                    s[l] = sw ? a : b;
                }
            }
        }
    }
}

// One thread per vertex of out-degree <= D: the pairs live in registers and
// are sorted by a bitonic network.
template <int D>
__global__ void __launch_bounds__(128) k_sig_small(const int32_t* __restrict__ list, int64_t count,
                                                   GraphView G, int32_t* __restrict__ cnt,
                                                   unsigned long long* __restrict__ skey,
                                                   uint32_t* __restrict__ slot, TableRef t,
                                                   unsigned* err) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int32_t v = list[i];
    const int64_t b = G.rp[v];
    const int d = row_len(G, v);
    uint64_t s[D];
    int live = 0;                                   // entries that count sort first
#pragma unroll
    for (int j = 0; j < D; ++j) {
        unsigned long long mv = ~0ull;
        if (j < d && entry_value(G, b + j, &mv)) ++live;
        else mv = ~0ull;
        s[j] = mv;
    }
    bitonic_regs<D>(s);
    uint32_t u = 0;
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        if (j < live && (j == 0 || s[j] != s[j - 1])) {
            skey[b + u] = s[j];
            sum += s[j];
            ++u;
        }
    }
    cnt[v] = static_cast<int32_t>(u);
    const uint64_t h = sig_hash(G.P[v], u, sum) & t.hmask;
    if (G.hout) G.hout[v] = h;
    slot[v] = table_insert(t, h, v, err);
}

// One warp per vertex of out-degree <= N (N <= 256), eight vertices per CTA:
// duplicates are removed with a hash set in the warp's slice of shared memory
// (2N slots), so the cost is linear in the degree and needs no CTA barrier.
// The unique values are written in arrival order (the list is a set; it is
// compared as a set by the verification pass).
template <int N>
__global__ void __launch_bounds__(256) k_sig_warp(const int32_t* __restrict__ list, int64_t count, GraphView G,
                                                  int32_t* __restrict__ cnt,
                                                  unsigned long long* __restrict__ skey,
                                                  uint32_t* __restrict__ slot, TableRef t, unsigned* err) {
    constexpr int S = 2 * N;
    __shared__ unsigned long long sm_all[8 * S];
    __shared__ unsigned zero_all[8];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    unsigned long long* tab = sm_all + warp * S;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * 8 + warp;
    if (i >= count) return;                      // whole warp leaves together
#pragma unroll
    for (int j = static_cast<int>(lane); j < S; j += 32) tab[j] = 0ull;
    if (lane == 0) zero_all[warp] = 0u;
    __syncwarp();
    const int32_t v = list[i];
    const int64_t b = G.rp[v];
    const int d = row_len(G, v);
    unsigned out = 0;
    unsigned long long mys = 0;
    for (int j0 = 0; j0 < d; j0 += 32) {
        const int j = j0 + static_cast<int>(lane);
        bool fresh = false;
        unsigned long long mv = 0;
        if (j < d && entry_value(G, b + j, &mv)) fresh = smem_set_insert(tab, S - 1, &zero_all[warp], mv);
        const unsigned ball = __ballot_sync(0xffffffffu, fresh);
        if (fresh) {
            skey[b + out + __popc(ball & lanemask_lt())] = mv;
            mys += mv;
        }
        out += __popc(ball);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mys += __shfl_xor_sync(0xffffffffu, mys, o);
    if (lane == 0) {
        cnt[v] = static_cast<int32_t>(out);
        const uint64_t h = sig_hash(G.P[v], out, mys) & t.hmask;
        if (G.hout) G.hout[v] = h;
        slot[v] = table_insert(t, h, v, err);
    }
}

// One CTA of T threads per vertex of out-degree <= N: hash-set dedup in a
// shared-memory table of 2N slots, block-wide compaction of the unique values.
template <int N, int T>
__global__ void __launch_bounds__(T) k_sig_mid(const int32_t* __restrict__ list, GraphView G,
                                               int32_t* __restrict__ cnt,
                                               unsigned long long* __restrict__ skey,
                                               uint32_t* __restrict__ slot, TableRef t,
                                               unsigned* err) {
    extern __shared__ unsigned long long tab[];   // 2N slots
    __shared__ unsigned long long ws[T / 32];
    __shared__ unsigned n_out, zero;
    constexpr uint32_t mask = 2 * N - 1;
    const int32_t v = list[blockIdx.x];
    const int64_t b = G.rp[v];
    const int d = row_len(G, v);
    for (int j = threadIdx.x; j < 2 * N; j += T) tab[j] = 0ull;
    if (threadIdx.x == 0) {
        n_out = 0;
        zero = 0;
    }
    __syncthreads();
    unsigned long long mys = 0;
    for (int j0 = 0; j0 < d; j0 += T) {
        const int j = j0 + static_cast<int>(threadIdx.x);
        bool fresh = false;
        unsigned long long mv = 0;
        if (j < d && entry_value(G, b + j, &mv)) fresh = smem_set_insert(tab, mask, &zero, mv);
        const unsigned ball = __ballot_sync(0xffffffffu, fresh);
        if (ball) {
            const int leader = __ffs(ball) - 1;
            unsigned base = 0;
            if (static_cast<int>(lane_id()) == leader) base = atomicAdd(&n_out, __popc(ball));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (fresh) {
                skey[b + base + __popc(ball & lanemask_lt())] = mv;
                mys += mv;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mys += __shfl_xor_sync(0xffffffffu, mys, o);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = mys;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tsum = 0;
        for (int w = 0; w < T / 32; ++w) tsum += ws[w];
        const unsigned total = n_out;
        cnt[v] = static_cast<int32_t>(total);
        const uint64_t h = sig_hash(G.P[v], total, tsum) & t.hmask;
        if (G.hout) G.hout[v] = h;
        slot[v] = table_insert(t, h, v, err);
    }
}

// Hub path, phase 1: every CTA dedups one chunk of a hub's edges into the hub's
// global hash set; first inserters append their value to the hub's list and
// add it to the hub's order-independent sum.
__global__ void __launch_bounds__(256) k_hub_insert(const HubChunk* __restrict__ chunks, GraphView G,
                                                    const int64_t* __restrict__ toff,
                                                    const uint32_t* __restrict__ tmask,
                                                    unsigned long long* __restrict__ tab_all,
                                                    HubAcc* __restrict__ acc,
                                                    unsigned long long* __restrict__ skey,
                                                    unsigned* err) {
    __shared__ unsigned long long red[8];
    const HubChunk c = chunks[blockIdx.x];
    unsigned long long* tab = tab_all + toff[c.hub];
    const uint32_t mask = tmask[c.hub];
    const int64_t row = G.rp[c.vertex];
    unsigned long long lsum = 0;
    for (int64_t e0 = c.begin; e0 < c.end; e0 += blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        bool fresh = false;
        unsigned long long mv = 0;
        if (e < c.end && entry_value(G, e, &mv)) {
            if (mv == 0ull) {
                fresh = atomicOr(&acc[c.hub].zero, 1u) == 0u;
            } else {
                uint32_t pos = static_cast<uint32_t>(mv) & mask;
                uint32_t probe = 0;
                for (; probe <= mask; ++probe) {
                    unsigned long long cur = tab[pos];
                    if (cur == mv) break;
                    if (cur == 0ull) {
                        unsigned long long prev = atomicCAS(&tab[pos], 0ull, mv);
                        if (prev == 0ull) { fresh = true; break; }
                        if (prev == mv) break;
                    }
                    pos = (pos + 1) & mask;
                }
                if (probe > mask) atomicOr(err, kErrHubFull);
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, fresh);
        if (ball) {
            const int leader = __ffs(ball) - 1;
            unsigned base = 0;
            if (static_cast<int>(lane_id()) == leader) base = atomicAdd(&acc[c.hub].count, __popc(ball));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (fresh) {
                skey[row + base + __popc(ball & lanemask_lt())] = mv;
                lsum += mv;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane_id() == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(&acc[c.hub].sum, s);
    }
}

// Hub path, phase 2: one thread per hub finishes its signature and inserts it.
__global__ void k_hub_finalize(const int32_t* __restrict__ hubs, int64_t nh, GraphView G,
                               const HubAcc* __restrict__ acc, int32_t* __restrict__ cnt,
                               uint32_t* __restrict__ slot, TableRef t, unsigned* err) {
    const int64_t h = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int32_t v = hubs[h];
    const unsigned c = acc[h].count;
    cnt[v] = static_cast<int32_t>(c);
    const uint64_t hv = sig_hash(G.P[v], c, acc[h].sum) & t.hmask;
    if (G.hout) G.hout[v] = hv;
    slot[v] = table_insert(t, hv, v, err);
}

// ----------------------------------------------------------------------------- resolution

// Insert level-`level` hashes for every live vertex (list == null) or for the
// listed ones.
template <class Mode>
__global__ void k_resolve_insert(const int32_t* __restrict__ list, int64_t count,
                                 const uint8_t* __restrict__ alive, Mode M, uint32_t level,
                                 uint32_t* __restrict__ slot, TableRef t, unsigned* err) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int32_t v = list ? list[i] : static_cast<int32_t>(i);
    if (!list && alive && !alive[v]) return;
    const uint64_t h = level_hash(M.hash0(v), level, t.hmask);
    slot[v] = table_insert(t, h, v, err);
}

// P_0's table insert with each CTA tile's vertices combined first: a
// shared-memory map from the level-0 hash to the tile's smallest vertex with
// it, so that each distinct hash of the tile goes into the global table once
// (the few hundred labels of ten million vertices otherwise send every vertex
// to the same few slots, and their reads and atomics queue there). The table
// then keeps the smallest vertex per hash as before, and every vertex gets its
// hash's slot. A hash the map cannot place within kP0Probes slots goes into
// the table from its vertex alone.
constexpr int kP0Per = 8;
constexpr int kP0Tile = 256 * kP0Per;
constexpr int kP0Slots = 1024;
constexpr int kP0Probes = 16;
constexpr unsigned long long kP0Empty = ~0ull;
__global__ void __launch_bounds__(256) k_p0_insert(int32_t n, const uint8_t* __restrict__ alive, LabelMode M,
                                                   uint32_t* __restrict__ slot, TableRef t, unsigned* err) {
    __shared__ unsigned long long key[kP0Slots];
    __shared__ int32_t vmin[kP0Slots];
    __shared__ uint32_t gslot[kP0Slots];
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kP0Tile; base < n;
         base += static_cast<int64_t>(gridDim.x) * kP0Tile) {
        for (int i = threadIdx.x; i < kP0Slots; i += blockDim.x) {
            key[i] = kP0Empty;
            vmin[i] = INT_MAX;
        }
        __syncthreads();
        uint64_t h[kP0Per];
        int where[kP0Per];                      // map entry; -1: straight to the table; -2: nothing (dead, past n)
#pragma unroll
        for (int k = 0; k < kP0Per; ++k) {
            const int64_t v = base + static_cast<int64_t>(k) * blockDim.x + threadIdx.x;
            where[k] = -2;
            h[k] = 0;
            if (v >= n || (alive != nullptr && !alive[v])) continue;
            h[k] = level_hash(M.hash0(static_cast<int32_t>(v)), 0u, t.hmask);
            where[k] = -1;
            if (h[k] == kP0Empty) continue;
            uint32_t pos = static_cast<uint32_t>(h[k]) & (kP0Slots - 1);
            for (int probe = 0; probe < kP0Probes; ++probe) {
                const unsigned long long prev = atomicCAS(&key[pos], kP0Empty, h[k]);
                if (prev == kP0Empty || prev == h[k]) {
                    atomicMin(&vmin[pos], static_cast<int32_t>(v));
                    where[k] = static_cast<int>(pos);
                    break;
                }
                pos = (pos + 1) & (kP0Slots - 1);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kP0Slots; i += blockDim.x)
            if (key[i] != kP0Empty) gslot[i] = table_insert(t, key[i], vmin[i], err);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kP0Per; ++k) {
            const int64_t v = base + static_cast<int64_t>(k) * blockDim.x + threadIdx.x;
            if (where[k] >= 0) slot[v] = gslot[where[k]];
            else if (where[k] == -1) slot[v] = table_insert(t, h[k], static_cast<int32_t>(v), err);
        }
        __syncthreads();                          // the map is cleared for the next tile
    }
}

// Confirm each vertex against its slot's smallest vertex. Equal: that vertex is
// its block id. Different: queue it for the next level.
template <class Mode>
__global__ void k_resolve_verify(const int32_t* __restrict__ list, int64_t count,
                                 const uint8_t* __restrict__ alive, Mode M,
                                 const uint32_t* __restrict__ slot, const Slot* __restrict__ slots,
                                 int32_t* __restrict__ Pout, int32_t* __restrict__ next,
                                 int32_t* __restrict__ deferred, DevState* st, int32_t n_total) {
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x;
    const int64_t i = i0 + threadIdx.x;
    bool is_block = false, push = false, defer = false;
    int32_t v = -1;
    if (i < count) {
        v = list ? list[i] : static_cast<int32_t>(i);
        if (!list && alive && !alive[v]) {
            Pout[v] = -1;
        } else {
            const uint32_t sv = slot[v];
            const int32_t r = sv == ~0u ? -1 : table_rep(slots, sv);
            if (r < 0 || r >= n_total) {          // failed insert: reported through st->error
                atomicOr(&st->error, kErrTableFull);
                Pout[v] = -1;
            } else if (r == v) {
                Pout[v] = v;
                is_block = true;
            } else {
                const int eq = M.compare(v, r);
                if (eq == 1) Pout[v] = r;
                else if (eq == 0) push = true;
                else defer = true;
            }
        }
    }
    const unsigned bb = __ballot_sync(0xffffffffu, is_block);
    if (bb && lane_id() == static_cast<unsigned>(__ffs(bb) - 1))
        atomicAdd(&st->blocks, static_cast<unsigned long long>(__popc(bb)));
    const unsigned pb = __ballot_sync(0xffffffffu, push);
    if (pb) {
        const int leader = __ffs(pb) - 1;
        unsigned base = 0;
        if (static_cast<int>(lane_id()) == leader) base = atomicAdd(&st->unresolved, __popc(pb));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (push) next[base + __popc(pb & lanemask_lt())] = v;
    }
    const unsigned db = __ballot_sync(0xffffffffu, defer);
    if (db) {
        const int leader = __ffs(db) - 1;
        unsigned base = 0;
        if (static_cast<int>(lane_id()) == leader) base = atomicAdd(&st->deferred, __popc(db));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (defer) deferred[base + __popc(db & lanemask_lt())] = v;
    }
}

constexpr int kDeferThreads = 256;
constexpr int kDeferGrid = 304;                        // two waves of one CTA per SM
constexpr int kDeferSetSlots = 2 * kMidMaxN;           // shared-memory set for lists up to 8192
constexpr size_t kDeferSmem = sizeof(unsigned long long) * kDeferSetSlots;

// Set comparison for the vertices deferred by k_resolve_verify: equal sizes
// were already checked, so S_v == S_r iff every value of S_v is in S_r. Lists
// up to 8192 values go through a shared-memory set of S_r; longer lists belong
// to hubs (a list is never longer than the degree), whose dedup table is probed.
// A persistent grid reads the deferred count on the device, so no host
// round trip is needed between the two passes.
__global__ void __launch_bounds__(kDeferThreads) k_verify_deferred(const int32_t* __restrict__ deferred,
                                                                   SigMode M, const uint32_t* __restrict__ slot,
                                                                   const Slot* __restrict__ slots,
                                                                   int32_t* __restrict__ Pout,
                                                                   int32_t* __restrict__ next, DevState* st) {
    extern __shared__ unsigned long long tab[];
    __shared__ unsigned zero;
    const unsigned count = *reinterpret_cast<volatile unsigned*>(&st->deferred);
    for (unsigned i = blockIdx.x; i < count; i += gridDim.x) {
        const int32_t v = deferred[i];
        const int32_t r = table_rep(slots, slot[v]);
        const int32_t c = M.cnt[v];
        const unsigned long long* lv = M.skey + M.G.rp[v];
        const unsigned long long* lr = M.skey + M.G.rp[r];
        bool miss = false;
        if (c > kMidMaxN) {
            const int64_t h = hub_index(M.H, v);
            for (int32_t j = threadIdx.x; j < c && !miss; j += kDeferThreads)
                miss = !hub_contains(M.H, h, lr[j]);
        } else {
            uint32_t size = 64;
            while (size < 2u * static_cast<uint32_t>(c)) size <<= 1;
            for (uint32_t j = threadIdx.x; j < size; j += kDeferThreads) tab[j] = 0ull;
            if (threadIdx.x == 0) zero = 0u;
            __syncthreads();
            for (int32_t j = threadIdx.x; j < c; j += kDeferThreads) smem_set_insert(tab, size - 1, &zero, lr[j]);
            __syncthreads();
            for (int32_t j = threadIdx.x; j < c && !miss; j += kDeferThreads)
                miss = !smem_set_contains(tab, size - 1, zero, lv[j]);
        }
        const int any = __syncthreads_or(miss ? 1 : 0);
        if (threadIdx.x == 0) {
            if (!any) Pout[v] = r;
            else next[atomicAdd(&st->unresolved, 1u)] = v;
        }
        __syncthreads();
    }
}

__global__ void k_local_ids(const int32_t* __restrict__ P, const int32_t* __restrict__ gid,
                            const int64_t* __restrict__ voff, int32_t n, int32_t* __restrict__ out) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t p = P[v];
    out[v] = p < 0 ? -1 : static_cast<int32_t>(p - voff[gid[v]]);
}

// ----------------------------------------------------------------------------- host side

}  // namespace

TableRef next_epoch(bisim_ctx* ctx, cudaStream_t s) {
    ctx->epoch32 += 1;
    const uint32_t e = ((ctx->epoch32 - 1) % kEpochCycle) + 1u;
    if (ctx->epoch32 > 1 && e == 1)   // the epoch wrapped: start from a blank table
        cudaMemsetAsync(ctx->table, 0, sizeof(Slot) * ctx->nslots, s);
    TableRef t;
    t.slots = ctx->table;
    t.mask = ctx->nslots - 1;
    t.epoch = static_cast<uint64_t>(e) << 32;
    const int hb = ctx->opt.hash_bits;
    t.hmask = hb >= 64 ? ~0ull : ((1ull << hb) - 1ull);
    return t;
}

namespace {

template <class Mode>
void launch_deferred(bisim_ctx* ctx, const Mode& M, int32_t* Pout, int32_t* next, cudaStream_t s) {
    if constexpr (Mode::kDefers) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_verify_deferred, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kDeferSmem));
            attr_set = true;
        }
        BISIM_SITE(site, "verify_deferred");
        Launch L(site, s, 0, 0, 0.0);
        k_verify_deferred<<<kDeferGrid, kDeferThreads, kDeferSmem, s>>>(ctx->dlist, M, ctx->slot, ctx->table, Pout,
                                                                         next, ctx->dstate);
    }
}

template <class Mode>
bisim_status resolve(bisim_ctx* ctx, Mode M, int32_t* Pout, const int32_t* vlist, int64_t vcount, cudaStream_t s,
                     int64_t* blocks) {
    const int32_t n = ctx->n;
    const int64_t nv = vlist ? vcount : n;
    cudaError_t e;
    cudaMemsetAsync(ctx->dstate, 0, sizeof(DevState), s);
    if (nv > 0) {
        BISIM_SITE(site, Mode::kVerifySite);
        Launch L(site, s, nv, 0, Mode::kVerifyBytesPerVertex * nv);
        k_resolve_verify<Mode><<<grid_for(nv, 256), 256, 0, s>>>(vlist, nv, ctx->alive, M, ctx->slot,
                                                                 ctx->table, Pout, ctx->ulist[0], ctx->dlist,
                                                                 ctx->dstate, n);
    }
    if (nv > 0) launch_deferred(ctx, M, Pout, ctx->ulist[0], s);
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "verify signatures");
    int which = 0;
    uint32_t level = 0;
    while (ctx->hstate->error == 0 && ctx->hstate->unresolved > 0) {
        if (++level > static_cast<uint32_t>(kMaxLevels))
            return set_error(ctx, BISIM_ETIMEOUT, "hash collision resolution did not converge");
        const int64_t cu = ctx->hstate->unresolved;
        TableRef t = next_epoch(ctx, s);
        cudaMemsetAsync(&ctx->dstate->unresolved, 0, sizeof(unsigned), s);
        cudaMemsetAsync(&ctx->dstate->deferred, 0, sizeof(unsigned), s);
        BISIM_SITE(site_i, "collision_insert");
        BISIM_SITE(site_v, "collision_verify");
        {
            Launch L(site_i, s, cu, 0, 0.0);
            k_resolve_insert<Mode><<<grid_for(cu, 256), 256, 0, s>>>(ctx->ulist[which], cu, ctx->alive, M, level,
                                                                      ctx->slot, t, &ctx->dstate->error);
        }
        {
            Launch L(site_v, s, cu, 0, 0.0);
            k_resolve_verify<Mode><<<grid_for(cu, 256), 256, 0, s>>>(ctx->ulist[which], cu, ctx->alive, M, ctx->slot,
                                                                      ctx->table, Pout, ctx->ulist[which ^ 1],
                                                                      ctx->dlist, ctx->dstate, n);
        }
        launch_deferred(ctx, M, Pout, ctx->ulist[which ^ 1], s);
        cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "resolve hash collisions");
        which ^= 1;
        ctx->stats.collision_levels += 1;
    }
    if (ctx->hstate->error & kErrTableFull) return set_error(ctx, BISIM_ETIMEOUT, "signature table probe limit reached");
    if (ctx->hstate->error & kErrHubFull) return set_error(ctx, BISIM_ETIMEOUT, "hub dedup table probe limit reached");
    if (ctx->hstate->error) return set_error(ctx, BISIM_EINVAL, "device reported invalid input");
    *blocks = static_cast<int64_t>(ctx->hstate->blocks);
    return BISIM_OK;
}

// Algorithmic bytes of the signature kernels: per edge col 4 + label 4 + the
// gathered P_i[w] 4; per vertex row_ptr 4 + P_i[v] 4 + one 16-byte table slot.
constexpr double kSigBytesPerEdge = 12.0;
constexpr double kSigBytesPerVertex = 24.0;


template <int N>
void launch_cta_mid(bisim_ctx* ctx, const int32_t* list, int64_t count, int64_t edges, GraphView G, TableRef t,
                    cudaStream_t s);

template <int N>
void launch_mid(bisim_ctx* ctx, const int32_t* list, int64_t count, int64_t edges, GraphView G, TableRef t,
                cudaStream_t s) {
    if constexpr (N <= 256) {
        static const int site = prof_site(N == 64 ? "sig_warp_64" : N == 128 ? "sig_warp_128" : "sig_warp_256");
        Launch L(site, s, count, edges, kSigBytesPerEdge * edges + kSigBytesPerVertex * count);
        k_sig_warp<N><<<grid_for(count, 8), 256, 0, s>>>(list, count, G, ctx->cnt, ctx->skey, ctx->slot, t,
                                                         &ctx->dstate->error);
    } else {
        launch_cta_mid<N>(ctx, list, count, edges, G, t, s);
    }
}

template <int N>
void launch_cta_mid(bisim_ctx* ctx, const int32_t* list, int64_t count, int64_t edges, GraphView G, TableRef t,
                    cudaStream_t s) {
    constexpr int T = N <= 1024 ? 256 : 512;
    const size_t smem = sizeof(unsigned long long) * 2 * N;
    static bool attr_set = false;   // per process; the attribute belongs to the function
    if (!attr_set && smem > 48 * 1024) {
        cudaFuncSetAttribute(k_sig_mid<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        attr_set = true;
    }
    static const int site = prof_site(N == 64 ? "sig_mid_64" : N == 128 ? "sig_mid_128" : N == 256 ? "sig_mid_256"
                                      : N == 512 ? "sig_mid_512" : N == 1024 ? "sig_mid_1024" : N == 2048 ? "sig_mid_2048"
                                      : N == 4096 ? "sig_mid_4096" : "sig_mid_8192");
    Launch L(site, s, count, edges, kSigBytesPerEdge * edges + kSigBytesPerVertex * count);
    k_sig_mid<N, T><<<static_cast<unsigned>(count), T, smem, s>>>(list, G, ctx->cnt, ctx->skey, ctx->slot, t,
                                                                  &ctx->dstate->error);
}

}  // namespace

// The gathers of a round read P_i at random (one 4-byte id per edge); P_i is
// small enough to stay in L2, so it is marked persisting there while the
// round's tables and edge streams pass through. The persisting set-aside is a
// limit of this process's context and disappears with it.
void pin_partition_in_l2(bisim_ctx* ctx, const int32_t* P, cudaStream_t s) {
    if (!(ctx->opt.flags & BISIM_FLAG_L2_PIN)) return;
    static int max_persist[64] = {};
    static int max_window[64] = {};
    const int dev = ctx->device;
    if (dev < 0 || dev >= 64) return;
    if (max_persist[dev] == 0) {
        int mp = 0, mw = 0;
        cudaDeviceGetAttribute(&mp, cudaDevAttrMaxPersistingL2CacheSize, dev);
        cudaDeviceGetAttribute(&mw, cudaDevAttrMaxAccessPolicyWindowSize, dev);
        max_persist[dev] = mp > 0 ? mp : -1;
        max_window[dev] = mw;
        if (mp > 0) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, static_cast<size_t>(mp));
    }
    if (max_persist[dev] <= 0 || max_window[dev] <= 0) return;
    const size_t bytes = std::min(sizeof(int32_t) * static_cast<size_t>(ctx->n), static_cast<size_t>(max_window[dev]));
    cudaStreamAttrValue attr;
    std::memset(&attr, 0, sizeof(attr));
    attr.accessPolicyWindow.base_ptr = const_cast<int32_t*>(P);
    attr.accessPolicyWindow.num_bytes = bytes;
    attr.accessPolicyWindow.hitRatio = std::min(1.0f, static_cast<float>(max_persist[dev]) / static_cast<float>(bytes));
    attr.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &attr);
    cudaGetLastError();   // a stream that takes no window (the legacy stream) simply runs without it
}

void unpin_partition(bisim_ctx* ctx, cudaStream_t s) {
    if (!(ctx->opt.flags & BISIM_FLAG_L2_PIN)) return;
    cudaStreamAttrValue attr;
    std::memset(&attr, 0, sizeof(attr));
    attr.accessPolicyWindow.num_bytes = 0;
    cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &attr);
    cudaCtxResetPersistingL2Cache();
    cudaGetLastError();
}

bisim_status alloc_refine_state(bisim_ctx* ctx, cudaStream_t s) {
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    cudaError_t e;
    const size_t nv = static_cast<size_t>(std::max(n, 1));
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->P0), sizeof(int32_t) * nv, s))) return cuda_error(ctx, e, "alloc P0");
    for (int i = 0; i < 2; ++i)
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->P[i]), sizeof(int32_t) * nv, s))) return cuda_error(ctx, e, "alloc P");
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->cnt), sizeof(int32_t) * nv, s))) return cuda_error(ctx, e, "alloc cnt");
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->slot), sizeof(uint32_t) * nv, s))) return cuda_error(ctx, e, "alloc slot");
    for (int i = 0; i < 2; ++i)
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ulist[i]), sizeof(int32_t) * nv, s))) return cuda_error(ctx, e, "alloc unresolved list");
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dlist), sizeof(int32_t) * nv, s))) return cuda_error(ctx, e, "alloc deferred list");
    // the pair lists (skey) of the list-mode path are allocated when that path first runs
    (void)m;
    // load factor at most 0.6: 8 bytes per slot keeps the table near L2 size
    uint64_t ns = 1024;
    while (static_cast<double>(ns) * 0.6 < static_cast<double>(n)) ns <<= 1;
    ctx->nslots = ns;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->table), sizeof(Slot) * ns, s))) return cuda_error(ctx, e, "alloc signature table");
    cudaMemsetAsync(ctx->table, 0, sizeof(Slot) * ns, s);
    if (ctx->hub_tab) cudaMemsetAsync(ctx->hub_tab, 0, sizeof(unsigned long long) * ctx->hub_tab_words, s);
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "init refine state");
    return BISIM_OK;
}

bisim_status compute_p0(bisim_ctx* ctx, cudaStream_t s) {
    TableRef t = next_epoch(ctx, s);
    LabelMode M{ctx->vlabel, ctx->gid};
    if (ctx->n > 0) {
        BISIM_SITE(site, "label_insert");
        Launch L(site, s, ctx->n, 0, 20.0 * ctx->n);   // label 4 B + one 16-byte table slot
        k_p0_insert<<<static_cast<unsigned>(std::min<int64_t>(cdiv(ctx->n, kP0Tile), 152 * 8)), 256, 0, s>>>(
            ctx->n, ctx->alive, M, ctx->slot, t, &ctx->dstate->error);
    }
    int64_t blocks = 0;
    bisim_status st = resolve(ctx, M, ctx->P0, nullptr, 0, s, &blocks);
    if (st != BISIM_OK) return st;
    ctx->last_blocks = blocks;
    ctx->stats.num_blocks = blocks;
    return BISIM_OK;
}

Buckets ctx_buckets(const bisim_ctx* ctx) {
    Buckets B;
    B.class_list = ctx->class_list;
    for (int c = 0; c <= kNumClasses; ++c) B.begin[c] = ctx->class_begin[c];
    for (int c = 0; c < kNumClasses; ++c) B.edges[c] = ctx->class_edges[c];
    B.hub_list = ctx->hub_list;
    B.n_hub = ctx->n_hub;
    B.chunks = ctx->chunks;
    B.n_chunks = ctx->n_chunks;
    B.toff = ctx->hub_toff;
    B.tmask = ctx->hub_tmask;
    B.tab = ctx->hub_tab;
    B.tab_words = ctx->hub_tab_words;
    B.acc = ctx->hub_acc;
    return B;
}

bisim_status signature_round(bisim_ctx* ctx, const Buckets& B, const int32_t* Pin, int32_t* Pout,
                             const int32_t* vlist, int64_t vcount, unsigned long long* hout, cudaStream_t s,
                             int64_t* out_blocks) {
    const GraphView G = ctx->store_ready
                            ? GraphView{ctx->xro, ctx->xlen, nullptr, nullptr, ctx->xpe, Pin, hout}
                            : GraphView{ctx->row_ptr, nullptr, ctx->col, ctx->elab, nullptr, Pin, hout};
    TableRef t = next_epoch(ctx, s);
    if (B.n_hub > 0) {
        cudaMemsetAsync(B.tab, 0, sizeof(unsigned long long) * B.tab_words, s);
        cudaMemsetAsync(B.acc, 0, sizeof(HubAcc) * B.n_hub, s);
    }
    const int64_t* cb = B.begin;
    unsigned* err = &ctx->dstate->error;
    static const int small_site[kSmallClasses] = {prof_site("sig_small_4"), prof_site("sig_small_8"),
                                                   prof_site("sig_small_16"), prof_site("sig_small_32")};
    auto small = [&](int c, auto kern) {
        const int64_t cnt = cb[c + 1] - cb[c];
        if (cnt > 0) {
            const int64_t edges = B.edges[c];
            Launch L(small_site[c], s, cnt, edges, kSigBytesPerEdge * edges + kSigBytesPerVertex * cnt);
            kern<<<grid_for(cnt, 128), 128, 0, s>>>(B.class_list + cb[c], cnt, G, ctx->cnt, ctx->skey,
                                                   ctx->slot, t, err);
        }
    };
    small(0, k_sig_small<4>);
    small(1, k_sig_small<8>);
    small(2, k_sig_small<16>);
    small(3, k_sig_small<32>);
    auto mid = [&](int c) {
        const int k = kSmallClasses + c;
        return std::make_tuple(B.class_list + cb[k], cb[k + 1] - cb[k], B.edges[k]);
    };
    { auto [l, c, e] = mid(0); if (c > 0) launch_mid<64>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(1); if (c > 0) launch_mid<128>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(2); if (c > 0) launch_mid<256>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(3); if (c > 0) launch_mid<512>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(4); if (c > 0) launch_mid<1024>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(5); if (c > 0) launch_mid<2048>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(6); if (c > 0) launch_mid<4096>(ctx, l, c, e, G, t, s); }
    { auto [l, c, e] = mid(7); if (c > 0) launch_mid<8192>(ctx, l, c, e, G, t, s); }
    if (B.n_chunks > 0) {
        BISIM_SITE(site_hi, "hub_insert");
        BISIM_SITE(site_hf, "hub_finalize");
        const int64_t hub_edges = B.edges[kClassHub];
        {
            Launch L1(site_hi, s, 0, hub_edges, kSigBytesPerEdge * hub_edges);
            k_hub_insert<<<static_cast<unsigned>(B.n_chunks), 256, 0, s>>>(B.chunks, G, B.toff, B.tmask, B.tab, B.acc,
                                                                          ctx->skey, err);
        }
        Launch L2(site_hf, s, B.n_hub, 0, kSigBytesPerVertex * B.n_hub);
        k_hub_finalize<<<grid_for(B.n_hub, 128), 128, 0, s>>>(B.hub_list, B.n_hub, G, B.acc, ctx->cnt, ctx->slot, t,
                                                             err);
    }
    cudaError_t e;
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "launch signature kernels");
    SigMode M;
    M.G = G;
    M.cnt = ctx->cnt;
    M.skey = ctx->skey;
    M.H = HubView{B.hub_list, B.n_hub, B.toff, B.tmask, B.tab, B.acc};
    // lists of up to small_max entries are sorted (thread-per-vertex classes); the
    // incremental path sets its own limit per batch
    M.small_max = ctx->store_ready ? ctx->inc_small_max : ctx->opt.small_max_degree;
    M.mid_max = ctx->opt.mid_max_degree;
    return resolve(ctx, M, Pout, vlist, vcount, s, out_blocks);
}

bisim_status refine_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks) {
    const int32_t* P = ctx->P[ctx->cur];
    pin_partition_in_l2(ctx, P, s);
    bisim_status st = signature_round(ctx, ctx_buckets(ctx), P, ctx->P[ctx->cur ^ 1], nullptr, 0, nullptr, s,
                                      out_blocks);
    if (st != BISIM_OK) return st;
    ctx->cur ^= 1;
    return BISIM_OK;
}

void launch_local_ids(const bisim_ctx* ctx, int32_t* out, cudaStream_t s) {
    BISIM_SITE(site, "local_ids");
    Launch L(site, s, ctx->n, 0, 8.0 * ctx->n);
    if (ctx->n > 0)
        k_local_ids<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->P[ctx->cur], ctx->gid, ctx->voff, ctx->n, out);
}

}  // namespace bisim
