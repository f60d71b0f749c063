// Incremental maintenance of the k-bisimulation partition under update
// batches (Section 3.2; Theorem 2 states that the incremental summary equals
// the batch summary of the edited graph, which is what this code keeps).
//
// For every level j = 0..k the state holds, per vertex, the id of its level-j
// block, and per block its signature hash, member count and smallest member;
// a hash index maps signature hashes to block ids. Block ids are stable names:
// a block keeps its id while its membership is unchanged, so a change only
// travels to the vertices whose own level-j block really changed.
//
// A batch touches, at level j, the frontier F_j: vertices whose label or
// liveness changed (j = 0), or whose out-edge multiset changed, whose level
// j-1 block changed, or that have an out-edge into such a vertex (j >= 1; the
// cascade of the paper's incremental complexity analysis). For F_j:
//   1. its vertices leave their old blocks (block minima that left are
//      recomputed over the remaining members);
//   2. it is grouped exactly among itself with the batch round machinery
//      (signatures over the level j-1 block ids);
//   3. each group is compared exactly with the live blocks of equal hash (a
//      block's smallest member stands for it) and joins one on equality;
//   4. otherwise a group that has exactly the members of one old block keeps
//      that block's id, and any other group gets a new id.
// The output partition names each level-k block by its smallest member.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "prof.cuh"
#include "rows.cuh"

namespace bisim {

namespace {

constexpr unsigned long long kIdxEmpty = 0ull;
constexpr unsigned long long kIdxTomb = 1ull;
constexpr int32_t kUndecided = -2;
constexpr int32_t kNew = -3;
constexpr int kCmpThreads = 256;
constexpr int kCmpSmallSlots = 4096;     // shared-memory set for lists up to 2048 values
constexpr int kCmpLargeSlots = 16384;    // ... up to 8192 values
constexpr int kCmpGrid = 304;            // compare CTAs (the candidate count is read on the device)
// list classes kSmallClasses + 6 and up hold rows of more than 2^11 entries
static_assert(kCmpSmallSlots / 2 == 1 << 11, "small compare set reach and class boundary differ");

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), 1 << 20)));
}

__device__ __forceinline__ unsigned long long index_key(uint64_t h) { return h < 2 ? h + 2 : h; }
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Per-level device view.
struct Level {
    uint8_t* stale;               // levels >= 1: the vertex's block has no current index key (see k_settle_single)
    int32_t* lid;                 // block id per vertex (-1 dead)
    int32_t* lcnt;                // |S| per vertex (levels >= 1)
    unsigned long long* bkey;     // per block: signature index key
    int32_t* bcnt;                // per block: members
    int32_t* bmin;                // per block: smallest member
    unsigned long long* ikey;     // index slots: key (0 empty, 1 tombstone)
    int32_t* ibid;                // index slots: block id
    uint64_t imask;
    int32_t* free;                // block ids freed by earlier batches
    long long* fc;                // [3]: ids in `free` when the level starts, taken, freed this level
};

// Per-batch scratch shared by the levels.
struct Work {
    int32_t* old;                 // [n] previous block id of frontier vertices
    int32_t* grp;                 // [n] frontier group (smallest frontier vertex with the same signature)
    unsigned long long* h;        // [n] signature hash of frontier vertices
    int32_t* gsize;               // [n] per group representative
    int32_t* gomin;               // [n]
    int32_t* gomax;               // [n]
    int32_t* decision;            // [n] block chosen for a group representative
    int64_t* resume;              // [n] next index slot to probe
    uint32_t* cntF;               // [bcap] frontier members per old block
    uint32_t* touched;            // [bcap]
    uint32_t* dirty;              // [bcap / 32] bit per block: its smallest member left
    int32_t* tlist;               // [bcap]
    int32_t* dlist;               // [bcap]
    int32_t* cand;                // [n] representatives with a candidate block
    int32_t* candb;               // [n] the candidate block
    unsigned long long* counters; // [8]
    int32_t* F;                   // [n] frontier
    int32_t* FL;                  // [n] live frontier
    uint8_t* inF;                 // [n]
    uint8_t* changed;             // [n]
    uint8_t* next;                // [n]
    uint8_t* recomp;              // [n] vertices the next level must recompute (their block gained a member)
    int32_t n;
    int64_t bcap;
    unsigned* err;                // self-check bits: an index out of range was skipped
};

constexpr unsigned kChkGroup = 1u, kChkProbe = 2u, kChkMin = 4u, kChkCompare = 8u, kChkAssign = 16u,
                   kChkOutput = 32u, kChkSettle = 64u, kChkPurge = 128u;

// ----------------------------------------------------------------------------- frontier

__device__ __forceinline__ void warp_list_push(bool f, int32_t v, int32_t* out, unsigned long long* count) {
    const unsigned ball = __ballot_sync(0xffffffffu, f);
    if (!ball) return;
    const int leader = __ffs(ball) - 1;
    unsigned long long base = 0;
    if (static_cast<int>(lane_id()) == leader) base = atomicAdd(count, static_cast<unsigned long long>(__popc(ball)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (f) out[base + __popc(ball & ((1u << lane_id()) - 1u))] = v;
}

// 16 flag bytes starting at v (a multiple of 16) as a 16-bit mask; null
// flags nothing, a misaligned array is read byte by byte.
__device__ __forceinline__ uint32_t flag_mask16(const uint8_t* f, int64_t v) {
    if (f == nullptr) return 0u;
    uint32_t m = 0u;
    if ((reinterpret_cast<uintptr_t>(f + v) & 15u) == 0u) {
        const uint4 w = *reinterpret_cast<const uint4*>(f + v);
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if ((q[k >> 2] >> (8 * (k & 3))) & 0xffu) m |= 1u << k;
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (f[v + k]) m |= 1u << k;
    }
    return m;
}

// Appends the positions v0 + k for the set bits k of `mask` to out, one atomic per warp.
__device__ __forceinline__ void warp_push_mask(uint32_t mask, int64_t v0, int32_t* out,
                                               unsigned long long* count) {
    const unsigned lane = lane_id();
    const unsigned mine = static_cast<unsigned>(__popc(mask));
    unsigned inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= static_cast<unsigned>(o)) inc += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, inc, 31);
    if (total == 0u) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(count, static_cast<unsigned long long>(total));
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned long long at = base + inc - mine;
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1u;
        out[at++] = static_cast<int32_t>(v0 + k);
    }
}

// The level's frontier in one pass: F = vertices with any of the flags a, b,
// c, d set (a null `a` flags every vertex), split by liveness and, from level
// 1 on, by the size of the vertex's block one level down: a vertex alone in
// its level-(j-1) block is alone at level j too (each level refines the last),
// so it goes to FX and needs no signature; the other live ones go to FL.
// count: [0] |F|, [1] |FL|, [2] |FX|. Each thread takes 16 vertices; most
// have no flag set and cost one 16-byte read per flag array.
__global__ void k_frontier(const uint8_t* __restrict__ a, const uint8_t* __restrict__ b,
                           const uint8_t* __restrict__ c, const uint8_t* __restrict__ d,
                           const uint8_t* __restrict__ alive, int32_t n, const int32_t* __restrict__ lid_prev,
                           const int32_t* __restrict__ bcnt_prev, uint8_t* __restrict__ stale,
                           int32_t* __restrict__ F, int32_t* __restrict__ FL, int32_t* __restrict__ FX,
                           unsigned long long* __restrict__ count) {
    const int64_t v0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 16;
    uint32_t mf = 0u, ml = 0u, mx = 0u;
    if (v0 < n) {
        const int valid = v0 + 16 <= n ? 16 : static_cast<int>(n - v0);
        const uint32_t vm = valid == 16 ? 0xffffu : ((1u << valid) - 1u);
        if (valid == 16) {
            mf = a == nullptr ? 0xffffu : (flag_mask16(a, v0) | flag_mask16(b, v0) | flag_mask16(c, v0) |
                                           flag_mask16(d, v0));
        } else {
            for (int k = 0; k < valid; ++k) {
                const int64_t v = v0 + k;
                if (a == nullptr || a[v] || (b && b[v]) || (c && c[v]) || (d && d[v])) mf |= 1u << k;
            }
        }
        mf &= vm;
        uint32_t m = mf;
        while (m) {
            const int k = __ffs(m) - 1;
            m &= m - 1u;
            const int64_t v = v0 + k;
            if (!alive[v]) continue;
            bool alone = false;
            if (lid_prev) {
                const int32_t pb = lid_prev[v];
                alone = pb >= 0 && bcnt_prev[pb] == 1;
                stale[v] = alone ? 1 : 0;
            }
            if (alone) mx |= 1u << k;
            else ml |= 1u << k;
        }
    }
    warp_push_mask(mf, v0, F, &count[0]);
    warp_push_mask(ml, v0, FL, &count[1]);
    warp_push_mask(mx, v0, FX, &count[2]);
}

// In-row tasks of the listed vertices (those whose previous-level block changed).
__global__ void k_in_row_tasks(const int32_t* __restrict__ list, const unsigned long long* __restrict__ count,
                               const int64_t* __restrict__ yro, const int32_t* __restrict__ ylen, TierLists L) {
    const int64_t c = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(count));
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t b0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; b0 < c; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        bool has = false;
        RowTask t{0, 0, 0};
        if (i < c) {
            const int32_t w = list[i];
            has = true;
            t = RowTask{yro[w], ylen[w], w};
        }
        tier_push(L, has, t);
    }
}

// mark[u] for every source u in the in-rows (a superset of the in-neighbours).
struct MarkSources {
    const int32_t* ype;
    uint8_t* mark;
    __device__ void operator()(const RowTask&, int64_t e, bool in) const {
        if (in) mark[ype[e]] = 1;
    }
};

__global__ void k_set_flags(const int32_t* __restrict__ list, int64_t count, uint8_t* __restrict__ flag, uint8_t v) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) flag[list[i]] = v;
}

// Kernels launched before the host knows the frontier's size read it on the
// device and stride over it with a fixed grid.
constexpr int kDevGrid = 152 * 8;

__device__ __forceinline__ int64_t dev_count(const unsigned long long* c) {
    return static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(c));
}

// ----------------------------------------------------------------------------- frontier degree buckets

// A hub of the live frontier with its row bounds (read back to lay out its chunks).
struct HubInfo {
    int32_t v;
    int32_t len;
    int64_t off;
};

__device__ __forceinline__ int list_class(int64_t d, int small_max, int mid_max) {
    if (d <= small_max || d == 0) return d <= 4 ? 0 : d <= 8 ? 1 : d <= 16 ? 2 : 3;
    if (d <= mid_max) {
        int lg = 64 - __clzll(static_cast<unsigned long long>(d - 1));
        lg = lg < 6 ? 6 : lg;
        return kSmallClasses + (lg - 6);
    }
    return kClassHub;
}

// Vertices and row entries per class over the live frontier (W.counters[7]
// vertices), one atomic per class per CTA.
__global__ void __launch_bounds__(256) k_class_count(const int32_t* __restrict__ FL,
                                                     const unsigned long long* __restrict__ dfl,
                                                     const int32_t* __restrict__ rl, int small_max, int mid_max,
                                                     unsigned long long* __restrict__ ccount,
                                                     unsigned long long* __restrict__ cedges) {
    __shared__ unsigned sc[kNumClasses];
    __shared__ unsigned long long se[kNumClasses];
    if (threadIdx.x < kNumClasses) {
        sc[threadIdx.x] = 0u;
        se[threadIdx.x] = 0ull;
    }
    __syncthreads();
    const int64_t fl = dev_count(dfl);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < fl;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t d = rl[FL[i]];
        const int c = list_class(d, small_max, mid_max);
        atomicAdd(&sc[c], 1u);
        atomicAdd(&se[c], static_cast<unsigned long long>(d));
    }
    __syncthreads();
    if (threadIdx.x < kNumClasses && sc[threadIdx.x]) {
        atomicAdd(&ccount[threadIdx.x], static_cast<unsigned long long>(sc[threadIdx.x]));
        atomicAdd(&cedges[threadIdx.x], se[threadIdx.x]);
    }
}

__global__ void k_class_scan(const unsigned long long* __restrict__ ccount, int64_t* __restrict__ begin,
                             unsigned long long* __restrict__ cursor) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        begin[c] = acc;
        cursor[c] = static_cast<unsigned long long>(acc);
        acc += static_cast<int64_t>(ccount[c]);
    }
    begin[kNumClasses] = acc;
}

// Places every live frontier vertex in its class's range (any order inside a
// class); hubs also go to `hubs` with their row bounds.
__global__ void __launch_bounds__(256) k_class_scatter(const int32_t* __restrict__ FL,
                                                       const unsigned long long* __restrict__ dfl,
                                                       const int64_t* __restrict__ ro, const int32_t* __restrict__ rl,
                                                       int small_max, int mid_max,
                                                       unsigned long long* __restrict__ cursor,
                                                       int32_t* __restrict__ out, HubInfo* __restrict__ hubs,
                                                       unsigned* __restrict__ n_hubs) {
    __shared__ unsigned cnt[kNumClasses];
    __shared__ unsigned long long base[kNumClasses];
    const int64_t fl = dev_count(dfl);
    for (int64_t b0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; b0 < fl;
         b0 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (threadIdx.x < kNumClasses) cnt[threadIdx.x] = 0u;
        __syncthreads();
        const int64_t i = b0 + threadIdx.x;
        int c = -1;
        int32_t v = 0;
        unsigned rank = 0;
        if (i < fl) {
            v = FL[i];
            c = list_class(rl[v], small_max, mid_max);
            rank = atomicAdd(&cnt[c], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kNumClasses && cnt[threadIdx.x])
            base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], static_cast<unsigned long long>(cnt[threadIdx.x]));
        __syncthreads();
        if (c >= 0) {
            out[base[c] + rank] = v;
            if (c == kClassHub) hubs[atomicAdd(n_hubs, 1u)] = HubInfo{v, rl[v], ro[v]};
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- level passes

// 1. frontier vertices (W.counters[6] of them) are flagged and leave their old blocks
__global__ void k_remove(const int32_t* __restrict__ F, Level L, Work W) {
    const int64_t f = dev_count(&W.counters[6]);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < f;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = F[i];
        W.inF[v] = 1;
        const int32_t b = L.lid[v];
        W.old[v] = b;
        if (b < 0) continue;
        atomicSub(&L.bcnt[b], 1);
        atomicAdd(&W.cntF[b], 1u);
        if (atomicExch(&W.touched[b], 1u) == 0u) W.tlist[atomicAdd(&W.counters[0], 1ull)] = b;
        const unsigned bit = 1u << (b & 31);
        if (L.bmin[b] == v && (atomicOr(&W.dirty[b >> 5], bit) & bit) == 0u)
            W.dlist[atomicAdd(&W.counters[1], 1ull)] = b;
    }
}

__global__ void k_dirty_reset(const int32_t* __restrict__ dlist, Level L, Work W) {
    const int64_t nd = dev_count(&W.counters[1]);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nd;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        L.bmin[dlist[i]] = INT_MAX;
}

// smallest remaining member of every block whose minimum left (nothing to do
// when no minimum left). One pass over all vertices, four per thread: the block
// ids are read in 16-byte words and looked up in the dirty bitmap (one bit per
// block, small enough to stay in L2); only members of dirty blocks read their
// live and frontier flags.
__global__ void __launch_bounds__(256) k_rescan(int32_t n, const uint8_t* __restrict__ alive, Level L, Work W) {
    const int64_t nd = dev_count(&W.counters[1]);
    if (nd == 0) return;
    const uint32_t* __restrict__ bits = W.dirty;
    auto visit = [&](int32_t u, int32_t b) {
        if (b < 0 || b >= W.bcap || ((__ldg(&bits[b >> 5]) >> (b & 31)) & 1u) == 0u) return;
        if (!alive[u] || W.inF[u]) return;
        atomicMin(&L.bmin[b], u);
    };
    const int64_t quads = n / 4;
    const int4* lid4 = reinterpret_cast<const int4*>(L.lid);
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < quads;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int4 b = lid4[q];
        const int32_t u = static_cast<int32_t>(4 * q);
        visit(u, b.x);
        visit(u + 1, b.y);
        visit(u + 2, b.z);
        visit(u + 3, b.w);
    }
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < n - 4 * quads) visit(static_cast<int32_t>(4 * quads + t), L.lid[4 * quads + t]);
}

// group statistics of the live frontier
__global__ void k_group_init(const int32_t* __restrict__ FL, int64_t fl, Work W) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= fl) return;
    const int32_t v = FL[i];
    if (W.grp[v] != v) return;
    W.gsize[v] = 0;
    W.gomin[v] = INT_MAX;
    W.gomax[v] = INT_MIN;
    W.decision[v] = kUndecided;
    W.resume[v] = -1;
}

__global__ void k_group_stats(const int32_t* __restrict__ FL, int64_t fl, Work W) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= fl) return;
    const int32_t v = FL[i];
    const int32_t g = W.grp[v];
    if (g < 0 || g >= W.n) {
        atomicOr(W.err, kChkGroup);
        return;
    }
    atomicAdd(&W.gsize[g], 1);
    atomicMin(&W.gomin[g], W.old[v]);
    atomicMax(&W.gomax[g], W.old[v]);
}

// 3a. probe the index for the next live block with the representative's key.
// Level 0 compares labels right here; deeper levels queue a candidate.
__global__ void k_probe(const int32_t* __restrict__ FL, int64_t fl, Level L, Work W, int level,
                        const int32_t* __restrict__ vlabel, uint64_t hmask) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= fl) return;
    const int32_t g = FL[i];
    if (W.grp[g] != g || W.decision[g] != kUndecided) return;
    const unsigned long long key = index_key(W.h[g]);
    uint64_t pos = W.resume[g] >= 0 ? static_cast<uint64_t>(W.resume[g]) : (key & L.imask);
    for (uint64_t probe = 0; probe <= L.imask; ++probe) {
        const unsigned long long k = L.ikey[pos];
        if (k == kIdxEmpty) {
            W.decision[g] = kNew;
            return;
        }
        if (k == key) {
            const int32_t b = L.ibid[pos];
            if (b < 0 || b >= W.bcap) {
                atomicOr(W.err, kChkProbe);
                W.decision[g] = kNew;
                return;
            }
            if (L.bcnt[b] > 0) {
                const int32_t r = L.bmin[b];
                if (r < 0 || r >= W.n) {
                    atomicOr(W.err, kChkMin);
                    W.decision[g] = kNew;
                    return;
                }
                if (level == 0) {
                    if (vlabel[r] == vlabel[g]) {
                        W.decision[g] = b;
                        return;
                    }
                } else {
                    W.resume[g] = static_cast<int64_t>((pos + 1) & L.imask);
                    const unsigned long long c = atomicAdd(&W.counters[2], 1ull);
                    W.cand[c] = g;
                    W.candb[c] = b;
                    return;
                }
            }
        }
        pos = (pos + 1) & L.imask;
    }
    W.decision[g] = kNew;
    (void)hmask;
}

// Inserts value mv into a shared-memory set (0 = empty; value 0 flagged in *zero).
__device__ __forceinline__ void cset_insert(unsigned long long* tab, uint32_t mask, unsigned* zero,
                                            unsigned long long mv) {
    if (mv == 0ull) { *zero = 1u; return; }
    uint32_t pos = static_cast<uint32_t>(mv) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&tab[pos], 0ull, mv);
        if (prev == 0ull || prev == mv) return;
        pos = (pos + 1) & mask;
    }
}

__device__ __forceinline__ bool cset_has(const unsigned long long* tab, uint32_t mask, unsigned zero,
                                         unsigned long long mv) {
    if (mv == 0ull) return zero != 0u;
    uint32_t pos = static_cast<uint32_t>(mv) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long cur = tab[pos];
        if (cur == mv) return true;
        if (cur == 0ull) return false;
        pos = (pos + 1) & mask;
    }
    return false;
}

// Pair value of store entry e over the block ids `lid`; false for a deleted
// entry or an edge into a dead vertex (no block).
__device__ __forceinline__ bool row_entry(const unsigned long long* pe, int64_t e, const int32_t* lid,
                                          unsigned long long* mv) {
    const unsigned long long x = pe[e];
    if (x == kRowTomb) return false;
    const int32_t b = lid[static_cast<int32_t>(static_cast<uint32_t>(x))];
    if (b < 0) return false;
    *mv = pair_value(static_cast<int32_t>(x >> 32), b);
    return true;
}

// 3b. exact comparison of a representative g with a candidate block's
// smallest member r: same previous-level block, same set size, and every pair
// of r is in g's set. Lists up to SLOTS/2 values use a shared-memory set; the
// list of a hub representative (above 8192 values) is looked up in its
// dedup table. One CTA per candidate.
template <int SLOTS>
__global__ void __launch_bounds__(kCmpThreads) k_compare(const unsigned long long* dcand, Level L, Level Lprev, Work W,
                                                         const int64_t* __restrict__ ro, const int32_t* __restrict__ rl,
                                                         const unsigned long long* __restrict__ pe,
                                                         const int32_t* __restrict__ cnt,
                                                         const unsigned long long* __restrict__ skey,
                                                         const int32_t* __restrict__ hub_list, int64_t n_hub,
                                                         const int64_t* __restrict__ toff,
                                                         const uint32_t* __restrict__ tmask,
                                                         const unsigned long long* __restrict__ tab_all,
                                                         const HubAcc* __restrict__ acc, int lo_c, int hi_c) {
    extern __shared__ unsigned long long tab[];
    __shared__ unsigned zero;
    const int64_t ncand = dev_count(dcand);
    for (int64_t i = blockIdx.x; i < ncand; i += gridDim.x) {
        const int32_t g = W.cand[i];
        const int32_t b = W.candb[i];
        const int32_t c = cnt[g];
        if (c < lo_c || c > hi_c) continue;                    // uniform: handled by another launch
        const int32_t r = L.bmin[b];
        if (r < 0 || r >= W.n || g < 0 || g >= W.n) {
            if (threadIdx.x == 0) atomicOr(W.err, kChkCompare);
            continue;
        }
        bool same = Lprev.lid[g] == Lprev.lid[r] && L.lcnt[r] == c;
        if (same) {
            bool miss = false;
            if (SLOTS > 0) {
                uint32_t size = 64;
                while (size < 2u * static_cast<uint32_t>(c)) size <<= 1;
                for (uint32_t j = threadIdx.x; j < size; j += kCmpThreads) tab[j] = 0ull;
                if (threadIdx.x == 0) zero = 0u;
                __syncthreads();
                const unsigned long long* lg = skey + ro[g];
                for (int32_t j = threadIdx.x; j < c; j += kCmpThreads) cset_insert(tab, size - 1, &zero, lg[j]);
                __syncthreads();
                for (int64_t e = ro[r] + threadIdx.x; e < ro[r] + rl[r] && !miss; e += kCmpThreads) {
                    unsigned long long mv;
                    if (row_entry(pe, e, Lprev.lid, &mv)) miss = !cset_has(tab, size - 1, zero, mv);
                }
            } else {
                // hub representative: its dedup table from the frontier's hub path
                int64_t lo = 0, hi = n_hub - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (hub_list[mid] < g) lo = mid + 1; else hi = mid;
                }
                const unsigned long long* ht = tab_all + toff[lo];
                const uint32_t mask = tmask[lo];
                for (int64_t e = ro[r] + threadIdx.x; e < ro[r] + rl[r] && !miss; e += kCmpThreads) {
                    unsigned long long mv;
                    if (!row_entry(pe, e, Lprev.lid, &mv)) continue;
                    bool found = false;
                    if (mv == 0ull) {
                        found = acc[lo].zero != 0u;
                    } else {
                        uint32_t pos = static_cast<uint32_t>(mv) & mask;
                        for (uint32_t probe = 0; probe <= mask; ++probe) {
                            const unsigned long long cur = ht[pos];
                            if (cur == mv) { found = true; break; }
                            if (cur == 0ull) break;
                            pos = (pos + 1) & mask;
                        }
                    }
                    miss = !found;
                }
            }
            same = !__syncthreads_or(miss ? 1 : 0);
        }
        if (threadIdx.x == 0 && same) W.decision[g] = b;
        __syncthreads();
    }
}

// A block id for a group that needs a new one: first the ids freed by earlier
// batches (k_retire frees the ids of blocks left without members; the level's
// list holds fc[0] of them while the level runs, and fc[1] counts those
// taken), then never-used ones. An id freed by a batch is reused only from the
// next batch on: no vertex, and after the batch no block signature of the
// level above, still names it (every vertex that had an out-edge into one of
// its members was in that level's frontier).
__device__ __forceinline__ long long take_block_id(const Level& L, int64_t* bnext) {
    if (L.fc != nullptr) {
        const long long avail = L.fc[0];
        const long long p = static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long*>(&L.fc[1]), 1ull));
        if (p < avail) return L.free[avail - 1 - p];
    }
    return static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long*>(bnext), 1ull));
}

// 4. groups without a live match: keep the old id if the membership is that
// of one old block, else take a fresh id. Also (re)keys the index.
// acc[0] index tombstones made, acc[1] rebuild flags, acc[2] tombstones reused
__global__ void k_settle(const int32_t* __restrict__ FL, int64_t fl, Level L, Work W, int64_t* __restrict__ bnext,
                         int64_t bcap, unsigned long long* __restrict__ counters) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= fl) return;
    const int32_t g = FL[i];
    if (W.grp[g] != g) return;
    if (W.decision[g] >= 0) return;                        // joined a live block
    const unsigned long long key = index_key(W.h[g]);
    const int32_t ob = W.gomin[g];
    if (ob >= W.bcap) {
        atomicOr(W.err, kChkSettle);
        return;
    }
    int32_t b;
    if (ob >= 0 && ob == W.gomax[g] && L.bcnt[ob] == 0 && static_cast<int32_t>(W.cntF[ob]) == W.gsize[g]) {
        b = ob;                                            // same members as before: keep the name
        if (L.bkey[b] != key) {
            // drop the old index entry of b, then insert the new key below
            const unsigned long long okey = L.bkey[b];
            uint64_t pos = okey & L.imask;
            for (uint64_t probe = 0; probe <= L.imask; ++probe) {
                if (L.ikey[pos] == kIdxEmpty) break;
                if (L.ikey[pos] == okey && L.ibid[pos] == b) {
                    L.ikey[pos] = kIdxTomb;
                    atomicAdd(&counters[0], 1ull);
                    break;
                }
                pos = (pos + 1) & L.imask;
            }
        } else {
            W.decision[g] = b;
            L.bmin[b] = INT_MAX;
            return;
        }
    } else {
        const long long nb = take_block_id(L, bnext);
        if (nb >= bcap) {
            atomicOr(reinterpret_cast<unsigned*>(&counters[1]), 1u);   // out of block ids: rebuild
            W.decision[g] = kNew;
            return;
        }
        b = static_cast<int32_t>(nb);
        L.bcnt[b] = 0;
    }
    L.bkey[b] = key;
    L.bmin[b] = INT_MAX;
    W.decision[g] = b;
    uint64_t pos = key & L.imask;
    for (uint64_t probe = 0; probe <= L.imask; ++probe) {
        unsigned long long cur = L.ikey[pos];
        if (cur == kIdxEmpty || cur == kIdxTomb) {
            const unsigned long long prev = atomicCAS(&L.ikey[pos], cur, key);
            if (prev == cur) {
                L.ibid[pos] = b;
                if (cur == kIdxTomb) atomicAdd(&counters[2], 1ull);   // a tombstone reused
                return;
            }
            continue;                                       // lost the slot: look at it again
        }
        pos = (pos + 1) & L.imask;
    }
    atomicOr(reinterpret_cast<unsigned*>(&counters[1]), 2u);   // index full
}

// 4b. frontier vertices alone in their block one level down (FX): alone here
// too. A vertex that was its old block's only member keeps that block (and its
// index entry, now possibly stale); otherwise it gets a new block without an
// index entry. Neither can be matched wrongly (every match is an exact
// compare), and one is never missed: another vertex can share its signature
// only by joining its block one level down, which puts it back into the
// frontier (k_assign's recomp flags).
__global__ void k_settle_single(const int32_t* __restrict__ FX, int64_t fx, Level L, Work W,
                                int64_t* __restrict__ bnext, int64_t bcap, unsigned long long* __restrict__ counters) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= fx) return;
    const int32_t v = FX[i];
    const int32_t o = W.old[v];
    W.grp[v] = v;
    if (o >= W.bcap) {
        atomicOr(W.err, kChkSettle);
        W.decision[v] = kNew;
        return;
    }
    if (o >= 0 && L.bcnt[o] == 0 && W.cntF[o] == 1u) {
        W.decision[v] = o;
        L.bmin[o] = INT_MAX;
        return;
    }
    const long long nb = take_block_id(L, bnext);
    if (nb >= bcap) {
        atomicOr(reinterpret_cast<unsigned*>(&counters[1]), 1u);   // out of block ids: rebuild
        W.decision[v] = kNew;
        return;
    }
    const int32_t b = static_cast<int32_t>(nb);
    L.bcnt[b] = 0;
    L.bkey[b] = 0ull;                                      // no index entry
    L.bmin[b] = INT_MAX;
    W.decision[v] = b;
}

// 5. frontier vertices take their blocks
// Vertices whose block changed are flagged in W.changed and listed in `clist`
// (for the next level's in-neighbour search).
// A vertex that joins a block whose only member u was alone one level down
// (so u's next-level block may have no current index key) flags u in
// W.recomp for the next level (stale_next: that level's stale flags, null at
// the last level).
__global__ void k_assign(const int32_t* __restrict__ F, int64_t f, const uint8_t* __restrict__ alive, Level L,
                         Work W, const int32_t* __restrict__ cnt_now, int level, int32_t* __restrict__ clist,
                         unsigned long long* __restrict__ ccount, const uint8_t* __restrict__ stale_next) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= f) return;
    const int32_t v = F[i];
    const int32_t o = W.old[v];
    if (alive[v]) {
        const int32_t g = W.grp[v];
        if (g < 0 || g >= W.n) {
            atomicOr(W.err, kChkAssign);
            return;
        }
        const int32_t b = W.decision[g];
        if (b < 0 || b >= W.bcap) {                        // ids ran out: the host rebuilds the state
            if (b != kNew) atomicOr(W.err, kChkAssign);
            return;
        }
        L.lid[v] = b;
        atomicAdd(&L.bcnt[b], 1);
        const int32_t before = atomicMin(&L.bmin[b], v);
        if (stale_next && b != o && before != INT_MAX && before != v && stale_next[before]) W.recomp[before] = 1;
        if (level > 0 && !L.stale[v]) L.lcnt[v] = cnt_now[v];
        W.changed[v] = b != o;
        if (b != o) clist[atomicAdd(ccount, 1ull)] = v;
    } else {
        L.lid[v] = -1;
        W.changed[v] = o != -1;
        if (o != -1) clist[atomicAdd(ccount, 1ull)] = v;
    }
}

// blocks left without members lose their index entry and free their id (for
// the next batch's new blocks, after the free list's unused part); per-block
// flags reset
__global__ void k_retire(const int32_t* __restrict__ tlist, int64_t nt, Level L, Work W,
                         unsigned long long* __restrict__ counters) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int32_t b = tlist[i];
    // (counters: the level's accumulators, as for k_settle)
    W.touched[b] = 0u;
    const unsigned bit = 1u << (b & 31);
    if (W.dirty[b >> 5] & bit) atomicAnd(&W.dirty[b >> 5], ~bit);
    W.cntF[b] = 0u;
    if (L.bcnt[b] != 0) return;
    if (L.fc != nullptr) {
        const long long left = L.fc[0] - min(L.fc[0], L.fc[1]);
        const long long at = static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long*>(&L.fc[2]), 1ull));
        L.free[left + at] = b;
    }
    const unsigned long long key = L.bkey[b];
    uint64_t pos = key & L.imask;
    for (uint64_t probe = 0; probe <= L.imask; ++probe) {
        const unsigned long long k = L.ikey[pos];
        if (k == kIdxEmpty) return;
        if (k == key && L.ibid[pos] == b) {
            L.ikey[pos] = kIdxTomb;
            atomicAdd(&counters[0], 1ull);
            return;
        }
        pos = (pos + 1) & L.imask;
    }
}

// Level 0 groups the live frontier by vertex label. A label is a 32-bit key,
// so an open-addressing table that stores the label itself groups exactly in
// one pass (no fingerprint to verify, no host round trip): a slot holds
// (label << 32 | smallest vertex), ~0 when empty.
__global__ void k_label_insert(const int32_t* __restrict__ FL, int64_t fl, const int32_t* __restrict__ vlabel,
                               unsigned long long* __restrict__ tab, uint64_t mask, unsigned* err) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < fl;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = FL[i];
        const uint64_t key = static_cast<uint32_t>(vlabel[v]);
        const unsigned long long want = (key << 32) | static_cast<uint32_t>(v);
        uint64_t pos = mix64(key) & mask;
        bool placed = false;
        for (uint64_t probe = 0; probe <= mask && !placed; ++probe) {
            unsigned long long cur = tab[pos];
            if (cur == ~0ull) {
                const unsigned long long prev = atomicCAS(&tab[pos], ~0ull, want);
                if (prev == ~0ull) {
                    placed = true;
                    break;
                }
                cur = prev;
            }
            if ((cur >> 32) == key) {
                while (static_cast<uint32_t>(v) < static_cast<uint32_t>(cur)) {
                    const unsigned long long prev = atomicCAS(&tab[pos], cur, want);
                    if (prev == cur) break;
                    cur = prev;
                }
                placed = true;
                break;
            }
            pos = (pos + 1) & mask;
        }
        if (!placed) atomicOr(err, kChkGroup);
    }
}

__global__ void k_label_read(const int32_t* __restrict__ FL, int64_t fl, const int32_t* __restrict__ vlabel,
                             const unsigned long long* __restrict__ tab, uint64_t mask, int32_t* __restrict__ grp,
                             unsigned* err) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < fl;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = FL[i];
        const uint64_t key = static_cast<uint32_t>(vlabel[v]);
        uint64_t pos = mix64(key) & mask;
        int32_t g = -1;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long cur = tab[pos];
            if (cur == ~0ull) break;
            if ((cur >> 32) == key) {
                g = static_cast<int32_t>(static_cast<uint32_t>(cur));
                break;
            }
            pos = (pos + 1) & mask;
        }
        if (g < 0) atomicOr(err, kChkGroup);
        grp[v] = g;
    }
}

__global__ void k_label_keys(const int32_t* __restrict__ FL, int64_t fl, const int32_t* __restrict__ vlabel,
                             unsigned long long* __restrict__ h, uint64_t hmask) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < fl) {
        const int32_t v = FL[i];
        h[v] = label_hash(0, vlabel[v]) & hmask;
    }
}

__global__ void k_output(int32_t n, const uint8_t* __restrict__ alive, const int32_t* __restrict__ lid,
                         const int32_t* __restrict__ bmin, int64_t bcap, int32_t* __restrict__ P, unsigned* err) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t b = alive[v] ? lid[v] : -1;
    if (alive[v] && (b < 0 || b >= bcap)) {
        atomicOr(err, kChkOutput);
        P[v] = -1;
        return;
    }
    P[v] = alive[v] ? bmin[b] : -1;
}

// End of a batch: each level's free list becomes its unused part followed by
// the ids freed in the batch (one thread per level).
__global__ void k_free_commit(long long* __restrict__ fc, int levels) {
    const int j = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= levels) return;
    long long* c = fc + 3 * j;
    c[0] = c[0] - min(c[0], c[1]) + c[2];
    c[1] = 0;
    c[2] = 0;
}

// Index without tombstones: emptied (by a memset), then every block with
// members and a key enters again. Those are the index's live entries (a block
// keyed by k_settle keeps one entry under its bkey until it is re-keyed or
// retired; a block made by k_settle_single has key 0 and none), so matching
// sees the same candidates as before.
__global__ void k_index_refill(const int32_t* __restrict__ bcnt, const unsigned long long* __restrict__ bkey,
                               int64_t used, unsigned long long* __restrict__ ikey, int32_t* __restrict__ ibid,
                               uint64_t imask, unsigned* __restrict__ err) {
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < used;
         b += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const unsigned long long key = bkey[b];
        if (bcnt[b] <= 0 || key <= kIdxTomb) continue;
        uint64_t pos = key & imask;
        bool placed = false;
        for (uint64_t probe = 0; probe <= imask && !placed; ++probe) {
            if (ikey[pos] == kIdxEmpty && atomicCAS(&ikey[pos], kIdxEmpty, key) == kIdxEmpty) {
                ibid[pos] = static_cast<int32_t>(b);
                placed = true;
            }
            pos = (pos + 1) & imask;
        }
        if (!placed) atomicOr(err, kChkPurge);
    }
}

// Free list of an imported level: every id below the next never-used one
// whose block has no members.
__global__ void k_free_collect(const int32_t* __restrict__ bcnt, int64_t used, int32_t* __restrict__ free,
                               long long* __restrict__ fc) {
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < used;
         b += static_cast<int64_t>(gridDim.x) * blockDim.x)
        if (bcnt[b] == 0) free[atomicAdd(reinterpret_cast<unsigned long long*>(&fc[0]), 1ull)] = static_cast<int32_t>(b);
}

// ----------------------------------------------------------------------------- host side

Level level_view(const bisim_ctx* ctx, int j) {
    return Level{ctx->lstale[j], ctx->lid[j], ctx->lcnt[j], ctx->bkey[j], ctx->bcnt[j], ctx->bmin[j], ctx->ikey[j],
                 ctx->ibid[j], ctx->isize - 1, ctx->lfree[j], ctx->lfreec ? ctx->lfreec + 3 * j : nullptr};
}

constexpr int kHubPrefetch = 2048;     // hub records read back with the level's counts
constexpr size_t kHubStageBytes = size_t{1} << 20;   // pinned stage of a frontier's hub layout
constexpr int64_t kThreadClassOps = 20000;   // batches above this use thread-per-vertex classes

// Host copies of everything a level pass reads back, in pinned memory so that
// the copies queue behind the level's kernels and one synchronisation covers them.
struct HostStage {
    unsigned long long counters[16];
    int64_t begin[kNumClasses + 1];
    unsigned long long edges[kNumClasses];
    unsigned n_hubs;
    unsigned err;
    unsigned long long ncand;
    int64_t bnext[kMaxIncLevels + 1];
    unsigned long long acc[kMaxIncLevels + 1][4];
    long long fc[kMaxIncLevels + 1][3];
    HubInfo hubs[kHubPrefetch];
};

// Work buffers of the incremental path, kept between batches.
struct Scratch {
    char* base = nullptr;
    size_t bytes = 0;                  // device bytes of base (counted in the context's device_bytes)
    Work W{};
    int64_t* dbnext = nullptr;         // [kMaxIncLevels + 1] next unused block id per level
    unsigned long long* dacc = nullptr;   // [kMaxIncLevels + 1][4] per-level accumulators (k_settle)
    long long* dfree = nullptr;        // [kMaxIncLevels + 1][3] free-list counters (Level::fc)
    int32_t* blist = nullptr;          // [n] live frontier grouped by class
    int64_t* dbegin = nullptr;         // [kNumClasses + 1]
    unsigned long long* ccount = nullptr;   // [kNumClasses] vertices per class
    unsigned long long* cedges = nullptr;   // [kNumClasses] row entries per class
    unsigned long long* ccursor = nullptr;  // [kNumClasses]
    HubInfo* hubs = nullptr;           // [n]
    unsigned* n_hubs = nullptr;
    int32_t* clist = nullptr;          // [n] vertices whose block changed one level down
    unsigned long long* chcount = nullptr;
    TierLists tiers{};                 // in-row tasks, [n] per tier
    HostStage* h = nullptr;            // pinned
    char* hub_stage = nullptr;         // pinned: a frontier's hub chunks, offsets, masks and ids (kHubStageBytes)
    int32_t* FX = nullptr;             // [n] live frontier vertices alone in their block one level down
    unsigned long long* ltab = nullptr;   // level-0 label table, a power of two >= 2n slots
};

cudaError_t alloc_scratch(bisim_ctx* ctx, Scratch& S, cudaStream_t s) {
    const size_t n = static_cast<size_t>(std::max(ctx->n, 1));
    const size_t bc = static_cast<size_t>(ctx->bcap);
    const size_t dw = (bc + 31) / 32;                      // dirty bitmap words
    constexpr size_t L = kMaxIncLevels + 1;
    size_t bytes = 0;
    auto need = [&](size_t b) { bytes += (b + 255) & ~size_t(255); };
    need(4 * n); need(4 * n); need(8 * n); need(4 * n); need(4 * n); need(4 * n); need(4 * n); need(8 * n);
    need(4 * bc); need(4 * bc); need(4 * dw); need(4 * bc); need(4 * bc);
    need(4 * n); need(4 * n); need(8 * 16); need(4 * n); need(4 * n); need(n); need(n); need(n); need(n); need(4 * n);
    size_t lslots = 64;
    while (lslots < 2 * n) lslots <<= 1;
    need(8 * lslots);
    need(8 * L); need(32 * L); need(24 * L); need(32);
    need(4 * n); need(8 * (kNumClasses + 1)); need(8 * kNumClasses); need(8 * kNumClasses); need(8 * kNumClasses);
    need(sizeof(HubInfo) * std::max<size_t>(n, kHubPrefetch)); need(16);
    need(4 * n); need(16); need(3 * sizeof(RowTask) * n); need(16);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&S.base), bytes, s);
    if (e) return e;
    S.bytes = bytes;
    ctx->device_bytes += static_cast<int64_t>(bytes);
    if ((e = cudaHostAlloc(reinterpret_cast<void**>(&S.h), sizeof(HostStage), cudaHostAllocDefault))) {
        cudaFreeAsync(S.base, s);
        S.base = nullptr;
        return e;
    }
    if ((e = cudaHostAlloc(reinterpret_cast<void**>(&S.hub_stage), kHubStageBytes, cudaHostAllocDefault))) {
        cudaFreeHost(S.h);
        S.h = nullptr;
        cudaFreeAsync(S.base, s);
        S.base = nullptr;
        return e;
    }
    char* p = S.base;
    auto carve = [&](size_t b) { char* q = p; p += (b + 255) & ~size_t(255); return q; };
    Work& W = S.W;
    W.old = reinterpret_cast<int32_t*>(carve(4 * n));
    W.grp = reinterpret_cast<int32_t*>(carve(4 * n));
    W.h = reinterpret_cast<unsigned long long*>(carve(8 * n));
    W.gsize = reinterpret_cast<int32_t*>(carve(4 * n));
    W.gomin = reinterpret_cast<int32_t*>(carve(4 * n));
    W.gomax = reinterpret_cast<int32_t*>(carve(4 * n));
    W.decision = reinterpret_cast<int32_t*>(carve(4 * n));
    W.resume = reinterpret_cast<int64_t*>(carve(8 * n));
    W.cntF = reinterpret_cast<uint32_t*>(carve(4 * bc));
    W.touched = reinterpret_cast<uint32_t*>(carve(4 * bc));
    W.dirty = reinterpret_cast<uint32_t*>(carve(4 * dw));
    W.tlist = reinterpret_cast<int32_t*>(carve(4 * bc));
    W.dlist = reinterpret_cast<int32_t*>(carve(4 * bc));
    W.cand = reinterpret_cast<int32_t*>(carve(4 * n));
    W.candb = reinterpret_cast<int32_t*>(carve(4 * n));
    W.counters = reinterpret_cast<unsigned long long*>(carve(8 * 16));
    W.F = reinterpret_cast<int32_t*>(carve(4 * n));
    W.FL = reinterpret_cast<int32_t*>(carve(4 * n));
    W.inF = reinterpret_cast<uint8_t*>(carve(n));
    W.changed = reinterpret_cast<uint8_t*>(carve(n));
    W.next = reinterpret_cast<uint8_t*>(carve(n));
    W.recomp = reinterpret_cast<uint8_t*>(carve(n));
    S.FX = reinterpret_cast<int32_t*>(carve(4 * n));
    S.ltab = reinterpret_cast<unsigned long long*>(carve(8 * lslots));
    S.dbnext = reinterpret_cast<int64_t*>(carve(8 * L));
    S.dacc = reinterpret_cast<unsigned long long*>(carve(32 * L));
    S.dfree = reinterpret_cast<long long*>(carve(24 * L));
    ctx->lfreec = S.dfree;
    W.err = reinterpret_cast<unsigned*>(carve(32));
    W.n = ctx->n;
    W.bcap = ctx->bcap;
    S.blist = reinterpret_cast<int32_t*>(carve(4 * n));
    S.dbegin = reinterpret_cast<int64_t*>(carve(8 * (kNumClasses + 1)));
    S.ccount = reinterpret_cast<unsigned long long*>(carve(8 * kNumClasses));
    S.cedges = reinterpret_cast<unsigned long long*>(carve(8 * kNumClasses));
    S.ccursor = reinterpret_cast<unsigned long long*>(carve(8 * kNumClasses));
    S.hubs = reinterpret_cast<HubInfo*>(carve(sizeof(HubInfo) * std::max<size_t>(n, kHubPrefetch)));
    S.n_hubs = reinterpret_cast<unsigned*>(carve(16));
    S.clist = reinterpret_cast<int32_t*>(carve(4 * n));
    S.chcount = reinterpret_cast<unsigned long long*>(carve(16));
    RowTask* tasks = reinterpret_cast<RowTask*>(carve(3 * sizeof(RowTask) * n));
    S.tiers = TierLists{{tasks, tasks + n, tasks + 2 * n}, reinterpret_cast<unsigned*>(carve(16))};
    cudaMemsetAsync(W.err, 0, 32, s);
    cudaMemsetAsync(S.dbnext, 0, 8 * L, s);
    cudaMemsetAsync(S.dacc, 0, 32 * L, s);
    cudaMemsetAsync(S.dfree, 0, 24 * L, s);                 // free lists start empty
    // per-block flags start (and are kept) at zero
    cudaMemsetAsync(W.cntF, 0, 4 * bc, s);
    cudaMemsetAsync(W.touched, 0, 4 * bc, s);
    cudaMemsetAsync(W.dirty, 0, 4 * dw, s);
    cudaMemsetAsync(W.changed, 0, n, s);
    cudaMemsetAsync(W.inF, 0, n, s);                       // pool memory is recycled: start clean
    cudaMemsetAsync(W.recomp, 0, n, s);
    return cudaSuccess;
}

void free_scratch(Scratch* S, cudaStream_t s) {
    if (S->base) cudaFreeAsync(S->base, s);
    if (S->h || S->hub_stage) cudaStreamSynchronize(s);   // no copy into or out of a stage is left in flight
    if (S->h) cudaFreeHost(S->h);
    if (S->hub_stage) cudaFreeHost(S->hub_stage);
    delete S;
}

// Degree buckets of the live frontier, launched before the level's read-back.
void launch_buckets(bisim_ctx* ctx, Scratch& S, cudaStream_t s) {
    const unsigned long long* dfl = &S.W.counters[7];
    cudaMemsetAsync(S.ccount, 0, 8 * kNumClasses, s);
    cudaMemsetAsync(S.cedges, 0, 8 * kNumClasses, s);
    cudaMemsetAsync(S.n_hubs, 0, 4, s);
    BISIM_SITE(site, "inc_buckets");
    Launch L(site, s, 0, 0, 0.0);
    const int sm = ctx->inc_small_max, mm = ctx->opt.mid_max_degree;
    k_class_count<<<kDevGrid, 256, 0, s>>>(S.W.FL, dfl, ctx->xlen, sm, mm, S.ccount, S.cedges);
    k_class_scan<<<1, 32, 0, s>>>(S.ccount, S.dbegin, S.ccursor);
    k_class_scatter<<<kDevGrid, 256, 0, s>>>(S.W.FL, dfl, ctx->xro, ctx->xlen, sm, mm, S.ccursor, S.blist, S.hubs,
                                            S.n_hubs);
    cudaMemcpyAsync(S.h->begin, S.dbegin, sizeof(S.h->begin), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(S.h->edges, S.cedges, sizeof(S.h->edges), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&S.h->n_hubs, S.n_hubs, 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(S.h->hubs, S.hubs, sizeof(S.h->hubs), cudaMemcpyDeviceToHost, s);
}

// After the read-back: the Buckets view, and the hub chunks laid out on the
// host (hubs in ascending vertex order, as the hub lookups expect).
struct ListBuckets {
    Buckets B;
    void* hubmem = nullptr;
};

bisim_status finish_buckets(bisim_ctx* ctx, Scratch& S, ListBuckets& out, cudaStream_t s) {
    Buckets& B = out.B;
    cudaError_t e;
    B.class_list = S.blist;
    for (int c = 0; c <= kNumClasses; ++c) B.begin[c] = S.h->begin[c];
    for (int c = 0; c < kNumClasses; ++c) B.edges[c] = static_cast<int64_t>(S.h->edges[c]);
    B.n_hub = S.h->n_hubs;
    if (B.n_hub == 0) return BISIM_OK;
    std::vector<HubInfo> hubs(S.h->hubs, S.h->hubs + std::min<int64_t>(B.n_hub, kHubPrefetch));
    if (B.n_hub > kHubPrefetch) {
        hubs.resize(B.n_hub);
        cudaMemcpyAsync(hubs.data() + kHubPrefetch, S.hubs + kHubPrefetch, sizeof(HubInfo) * (B.n_hub - kHubPrefetch),
                        cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "read frontier hubs");
    }
    std::sort(hubs.begin(), hubs.end(), [](const HubInfo& a, const HubInfo& b) { return a.v < b.v; });
    std::vector<int32_t> ids(B.n_hub);
    std::vector<HubChunk> chunks;
    std::vector<int64_t> toff(B.n_hub);
    std::vector<uint32_t> tmask(B.n_hub);
    int64_t words = 0;
    const int64_t csz = ctx->opt.hub_chunk;
    for (int64_t h = 0; h < B.n_hub; ++h) {
        ids[h] = hubs[h].v;
        const int64_t rb = hubs[h].off, re = hubs[h].off + hubs[h].len;
        uint64_t sz = 64;
        while (sz < static_cast<uint64_t>(2 * (re - rb))) sz <<= 1;
        toff[h] = words;
        tmask[h] = static_cast<uint32_t>(sz - 1);
        words += static_cast<int64_t>(sz);
        for (int64_t b = rb; b < re; b += csz)
            chunks.push_back(HubChunk{static_cast<int32_t>(h), hubs[h].v, b, std::min(re, b + csz)});
    }
    // the host-made part (chunks, table offsets, masks, hub ids) first, so that
    // one copy from the pinned stage moves it when it fits there
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t head = r256(sizeof(HubChunk) * chunks.size()) + r256(sizeof(int64_t) * B.n_hub) +
                        r256(sizeof(uint32_t) * B.n_hub) + r256(sizeof(int32_t) * B.n_hub);
    const size_t bytes = head + r256(sizeof(unsigned long long) * words) + r256(sizeof(HubAcc) * B.n_hub);
    char* p = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&p), bytes, s))) return cuda_error(ctx, e, "alloc frontier hubs");
    out.hubmem = p;
    char* const dbase = p;
    auto carve = [&](size_t b) { char* q = p; p += r256(b); return q; };
    HubChunk* dchunks = reinterpret_cast<HubChunk*>(carve(sizeof(HubChunk) * chunks.size()));
    int64_t* dtoff = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * B.n_hub));
    uint32_t* dtmask = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * B.n_hub));
    int32_t* dids = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * B.n_hub));
    unsigned long long* dtab = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long) * words));
    HubAcc* dacc = reinterpret_cast<HubAcc*>(carve(sizeof(HubAcc) * B.n_hub));
    if (head <= kHubStageBytes) {
        // the stage's last copy has finished: the level synchronised since
        char* h = S.hub_stage;
        std::memcpy(h + (reinterpret_cast<char*>(dchunks) - dbase), chunks.data(), sizeof(HubChunk) * chunks.size());
        std::memcpy(h + (reinterpret_cast<char*>(dtoff) - dbase), toff.data(), sizeof(int64_t) * B.n_hub);
        std::memcpy(h + (reinterpret_cast<char*>(dtmask) - dbase), tmask.data(), sizeof(uint32_t) * B.n_hub);
        std::memcpy(h + (reinterpret_cast<char*>(dids) - dbase), ids.data(), sizeof(int32_t) * B.n_hub);
        cudaMemcpyAsync(dbase, h, head, cudaMemcpyHostToDevice, s);
    } else {
        // pageable sources: each copy has taken its data when the call returns
        cudaMemcpyAsync(dchunks, chunks.data(), sizeof(HubChunk) * chunks.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dtoff, toff.data(), sizeof(int64_t) * B.n_hub, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dtmask, tmask.data(), sizeof(uint32_t) * B.n_hub, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dids, ids.data(), sizeof(int32_t) * B.n_hub, cudaMemcpyHostToDevice, s);
    }
    B.hub_list = dids;
    B.chunks = dchunks;
    B.n_chunks = static_cast<int64_t>(chunks.size());
    B.toff = dtoff;
    B.tmask = dtmask;
    B.tab = dtab;
    B.tab_words = words;
    B.acc = dacc;
    return BISIM_OK;
}

// The signature lists of the list-mode kernels sit at the rows' offsets in the
// out-pool of the row store.
bisim_status ensure_skey(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->xpool <= ctx->skey_cap) return BISIM_OK;
    ctx_free(ctx, ctx->skey, sizeof(unsigned long long) * ctx->skey_cap, s);
    ctx->skey = nullptr;
    const int64_t cap = ctx->xpool;
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->skey), sizeof(unsigned long long) * cap, s)))
        return cuda_error(ctx, e, "grow signature lists");
    ctx->skey_cap = cap;
    return BISIM_OK;
}

// Frontier lists from the flags a | b | c | d (every vertex when a is null):
// F (live or dead), its live part split into FL and FX (see k_frontier);
// their sizes stay on the device (W.counters[6], [7], [8]).
void launch_frontier(bisim_ctx* ctx, Scratch& S, int j, const uint8_t* a, const uint8_t* b, const uint8_t* c,
                     const uint8_t* d, cudaStream_t s) {
    Work& W = S.W;
    const int32_t n = ctx->n;
    cudaMemsetAsync(&W.counters[6], 0, 24, s);
    if (n > 0)
        k_frontier<<<grid_for(cdiv(n, 16), 256), 256, 0, s>>>(a, b, c, d, ctx->alive, n, j > 0 ? ctx->lid[j - 1] : nullptr,
                                                    j > 0 ? ctx->bcnt[j - 1] : nullptr, ctx->lstale[j], W.F, W.FL,
                                                    S.FX, &W.counters[6]);
}

// One level over the frontier launch_frontier made. Host round trips: one
// read-back of the frontier's sizes and buckets, the signature round's own,
// and one per probe round that still has candidates. The level's block-id and
// index checks are read back once for all levels by inc_finish.
bisim_status level_pass(bisim_ctx* ctx, int j, Scratch& S, int64_t* frontier, cudaStream_t s) {
    Work& W = S.W;
    Level L = level_view(ctx, j);
    const int32_t n = ctx->n;
    cudaError_t e;
    bisim_status st;
    BISIM_SITE(site_remove, "inc_remove");
    BISIM_SITE(site_single, "inc_single");
    BISIM_SITE(site_label, "inc_label");
    BISIM_SITE(site_group, "inc_group");
    BISIM_SITE(site_probe, "inc_probe");
    BISIM_SITE(site_compare, "inc_compare");
    BISIM_SITE(site_settle, "inc_settle");
    BISIM_SITE(site_assign, "inc_assign");
    BISIM_SITE(site_retire, "inc_retire");
    // 1. frontier vertices leave their old blocks (sizes read on the device)
    cudaMemsetAsync(W.counters, 0, 8 * 6, s);
    {
        Launch Lk(site_remove, s, 0, 0, 0.0);
        k_remove<<<kDevGrid, 256, 0, s>>>(W.F, L, W);
        k_dirty_reset<<<kDevGrid, 256, 0, s>>>(W.dlist, L, W);
        k_rescan<<<kDevGrid, 256, 0, s>>>(n, ctx->alive, L, W);
    }
    if (j > 0) launch_buckets(ctx, S, s);
    cudaMemcpyAsync(S.h->counters, W.counters, sizeof(S.h->counters), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "frontier sizes");
    const int64_t ntouched = static_cast<int64_t>(S.h->counters[0]);
    const int64_t f = static_cast<int64_t>(S.h->counters[6]);
    const int64_t fl = static_cast<int64_t>(S.h->counters[7]);
    const int64_t fx = static_cast<int64_t>(S.h->counters[8]);
    *frontier = fl + fx;
    unsigned long long* acc = S.dacc + 4 * j;
    if (fx > 0) {
        // alone one level down: no signature, see k_settle_single
        Launch Lk(site_single, s, fx, 0, 16.0 * fx);
        k_settle_single<<<grid_for(fx, 256), 256, 0, s>>>(S.FX, fx, L, W, S.dbnext + j, ctx->bcap, acc);
    }
    // 2. exact groups within the live frontier
    ListBuckets LB;
    if (fl > 0) {
        if (j == 0) {
            uint64_t slots = 64;
            while (slots < 2 * static_cast<uint64_t>(fl)) slots <<= 1;
            Launch Lk(site_label, s, fl, 0, 40.0 * fl);
            cudaMemsetAsync(S.ltab, 0xff, sizeof(unsigned long long) * slots, s);
            k_label_insert<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, ctx->vlabel, S.ltab, slots - 1, W.err);
            k_label_read<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, ctx->vlabel, S.ltab, slots - 1, W.grp, W.err);
            k_label_keys<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, ctx->vlabel, W.h,
                                                          ctx->opt.hash_bits >= 64 ? ~0ull : ((1ull << ctx->opt.hash_bits) - 1));
        } else {
            if ((st = finish_buckets(ctx, S, LB, s)) != BISIM_OK) return st;
            int64_t blocks = 0;
            st = signature_round(ctx, LB.B, ctx->lid[j - 1], W.grp, W.FL, fl, W.h, s, &blocks);
            if (st != BISIM_OK) {
                if (LB.hubmem) cudaFreeAsync(LB.hubmem, s);
                return st;
            }
        }
        Launch Lk(site_group, s, fl, 0, 24.0 * fl);
        k_group_init<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, W);
        k_group_stats<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, W);
    }
    // 3. match live blocks: probe, compare the candidates (their number is read
    // on the device), probe again; the host only looks when a probe round
    // still leaves candidates (different signatures under one hash)
    const uint64_t hmask = ctx->opt.hash_bits >= 64 ? ~0ull : ((1ull << ctx->opt.hash_bits) - 1);
    if (fl > 0) {
        Launch Lk(site_probe, s, fl, 0, 32.0 * fl);
        cudaMemsetAsync(&W.counters[2], 0, 8, s);
        k_probe<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, L, W, j, ctx->vlabel, hmask);
    }
    for (int iter = 0; fl > 0 && j > 0; ++iter) {
        if (iter > 1 << 16) {
            if (LB.hubmem) cudaFreeAsync(LB.hubmem, s);
            return set_error(ctx, BISIM_ETIMEOUT, "incremental block matching did not converge");
        }
        Level Lp = level_view(ctx, j - 1);
        const Buckets& B = LB.B;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_compare<kCmpLargeSlots>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sizeof(unsigned long long) * kCmpLargeSlots));
            attr = true;
        }
        {
            Launch Lk(site_compare, s, 0, 0, 0.0);
            k_compare<kCmpSmallSlots><<<kCmpGrid, kCmpThreads, sizeof(unsigned long long) * kCmpSmallSlots, s>>>(
                &W.counters[2], L, Lp, W, ctx->xro, ctx->xlen, ctx->xpe, ctx->cnt, ctx->skey, B.hub_list, B.n_hub,
                B.toff, B.tmask, B.tab, B.acc, 0, kCmpSmallSlots / 2);
            // a representative's set is no larger than its row: the larger variants only
            // run when the frontier has rows above the small set's reach
            if (B.begin[kNumClasses] > B.begin[kSmallClasses + 6])
                k_compare<kCmpLargeSlots><<<kCmpGrid, kCmpThreads, sizeof(unsigned long long) * kCmpLargeSlots, s>>>(
                    &W.counters[2], L, Lp, W, ctx->xro, ctx->xlen, ctx->xpe, ctx->cnt, ctx->skey, B.hub_list, B.n_hub,
                    B.toff, B.tmask, B.tab, B.acc, kCmpSmallSlots / 2 + 1, kCmpLargeSlots / 2);
            if (B.n_hub > 0)
                k_compare<0><<<kCmpGrid, kCmpThreads, 0, s>>>(&W.counters[2], L, Lp, W, ctx->xro, ctx->xlen, ctx->xpe,
                                                              ctx->cnt, ctx->skey, B.hub_list, B.n_hub, B.toff, B.tmask,
                                                              B.tab, B.acc, kCmpLargeSlots / 2 + 1, INT_MAX);
            cudaMemsetAsync(&W.counters[2], 0, 8, s);
            k_probe<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, L, W, j, ctx->vlabel, hmask);
        }
        cudaMemcpyAsync(&S.h->ncand, &W.counters[2], 8, cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "probe blocks");
        if (S.h->ncand == 0) break;
    }
    if (LB.hubmem) cudaFreeAsync(LB.hubmem, s);
    // 4. keep or create ids; 5. assign; retire empty blocks
    if (fl > 0) {
        Launch Lk(site_settle, s, fl, 0, 24.0 * fl);
        k_settle<<<grid_for(fl, 256), 256, 0, s>>>(W.FL, fl, L, W, S.dbnext + j, ctx->bcap, acc);
    }
    if (f > 0) {
        Launch Lk(site_assign, s, f, 0, 24.0 * f);
        k_assign<<<grid_for(f, 256), 256, 0, s>>>(W.F, f, ctx->alive, L, W, ctx->cnt, j, S.clist, S.chcount,
                                                 j < ctx->inc_k ? ctx->lstale[j + 1] : nullptr);
        k_set_flags<<<grid_for(f, 256), 256, 0, s>>>(W.F, f, W.inF, 0);
    }
    if (ntouched > 0) {
        Launch Lk(site_retire, s, ntouched, 0, 16.0 * ntouched);
        k_retire<<<grid_for(ntouched, 256), 256, 0, s>>>(W.tlist, ntouched, L, W, acc);
    }
    return BISIM_OK;
}

// The partition P_k (smallest member of each level-k block) and every level's
// deferred checks, read back together. *rebuild is set when a level ran out of
// block ids or index room (the state must then be rebuilt).
bisim_status inc_finish(bisim_ctx* ctx, Scratch& S, bool* rebuild, cudaStream_t s) {
    const int K = ctx->inc_k;
    constexpr int L = kMaxIncLevels + 1;
    if (ctx->n > 0) {
        BISIM_SITE(site, "inc_output");
        Launch Lk(site, s, ctx->n, 0, 13.0 * ctx->n);
        cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
        k_output<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->alive, ctx->lid[K], ctx->bmin[K], ctx->bcap,
                                                      ctx->P[0], &ctx->dstate->error);
    }
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(S.h->bnext, S.dbnext, 8 * L, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(S.h->acc, S.dacc, 32 * L, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&S.h->err, S.W.err, 4, cudaMemcpyDeviceToHost, s);
    cudaMemsetAsync(S.dacc, 0, 32 * L, s);
    k_free_commit<<<1, 32, 0, s>>>(S.dfree, L);
    cudaMemcpyAsync(S.h->fc, S.dfree, 24 * L, cudaMemcpyDeviceToHost, s);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "incremental update");
    if (S.h->err) {
        char msg[96];
        std::snprintf(msg, sizeof(msg), "incremental state self-check failed (bits 0x%x)", S.h->err);
        return set_error(ctx, BISIM_EINVAL, msg);
    }
    *rebuild = false;
    for (int j = 0; j <= K; ++j) {
        ctx->itomb[j] += static_cast<int64_t>(S.h->acc[j][0]) - static_cast<int64_t>(S.h->acc[j][2]);
        if (S.h->acc[j][1]) *rebuild = true;
        ctx->bnext[j] = std::min<int64_t>(S.h->bnext[j], ctx->bcap);
        ctx->nfree[j] = S.h->fc[j][0];
    }
    if (!*rebuild && ctx->n > 0 && ctx->hstate->error)
        return set_error(ctx, BISIM_EINVAL, "incremental state inconsistent at output");
    ctx->cur = 0;
    ctx->cur_k = K;
    return BISIM_OK;
}

bisim_status write_output(bisim_ctx* ctx, cudaStream_t s) {
    const int k = ctx->inc_k;
    if (ctx->n > 0) {
        BISIM_SITE(site, "inc_output");
        Launch L(site, s, ctx->n, 0, 13.0 * ctx->n);
        cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
        k_output<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->alive, ctx->lid[k], ctx->bmin[k], ctx->bcap,
                                                      ctx->P[0], &ctx->dstate->error);
        cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) return cuda_error(ctx, e, "write partition");
        if (ctx->hstate->error) return set_error(ctx, BISIM_EINVAL, "incremental state inconsistent at output");
    }
    ctx->cur = 0;
    ctx->cur_k = k;
    return BISIM_OK;
}

}  // namespace

void inc_release(bisim_ctx* ctx, cudaStream_t s) {
    const size_t n = static_cast<size_t>(std::max(ctx->n, 1));
    if (ctx->inc_ws != nullptr) {
        ctx->device_bytes -= static_cast<int64_t>(static_cast<Scratch*>(ctx->inc_ws)->bytes);
        free_scratch(static_cast<Scratch*>(ctx->inc_ws), s);
        ctx->inc_ws = nullptr;
    }
    for (int j = 0; j <= kMaxIncLevels; ++j) {
        ctx_free(ctx, ctx->lid[j], 4 * n, s);
        ctx_free(ctx, ctx->lcnt[j], 4 * n, s);
        ctx_free(ctx, ctx->bkey[j], 8 * static_cast<size_t>(ctx->bcap), s);
        ctx_free(ctx, ctx->bcnt[j], 4 * static_cast<size_t>(ctx->bcap), s);
        ctx_free(ctx, ctx->bmin[j], 4 * static_cast<size_t>(ctx->bcap), s);
        ctx_free(ctx, ctx->ikey[j], 8 * ctx->isize, s);
        ctx_free(ctx, ctx->ibid[j], 4 * ctx->isize, s);
        ctx_free(ctx, ctx->lstale[j], n, s);
        ctx_free(ctx, ctx->lfree[j], 4 * static_cast<size_t>(ctx->bcap), s);
        ctx->lstale[j] = nullptr;
        ctx->lfree[j] = nullptr;
        ctx->lid[j] = ctx->lcnt[j] = ctx->bcnt[j] = ctx->bmin[j] = ctx->ibid[j] = nullptr;
        ctx->bkey[j] = ctx->ikey[j] = nullptr;
        ctx->bnext[j] = ctx->itomb[j] = ctx->nfree[j] = 0;
    }
    ctx->lfreec = nullptr;                                 // lives in the scratch
    ctx->inc_k = -1;
}

// The incremental state of K levels allocated but not computed: the row
// store (from the CSR), the levels' arrays at the given record and index
// sizes, and the per-batch scratch. bisim_import_state fills the levels from
// an exported state.
bisim_status inc_alloc_levels(bisim_ctx* ctx, int K, int64_t bcap, uint64_t isize, cudaStream_t s) {
    if (K < 0 || K > kMaxIncLevels) return set_error(ctx, BISIM_EINVAL, "k_incremental out of range");
    inc_release(ctx, s);
    bisim_status st;
    if ((st = store_build(ctx, s)) != BISIM_OK) return st;
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK) return st;
    if ((st = ensure_skey(ctx, s)) != BISIM_OK) return st;
    const size_t n = static_cast<size_t>(std::max(ctx->n, 1));
    ctx->bcap = bcap;
    ctx->isize = isize;
    cudaError_t e;
    for (int j = 0; j <= K; ++j) {
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lid[j]), 4 * n, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lcnt[j]), 4 * n, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->bkey[j]), 8 * static_cast<size_t>(bcap), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->bcnt[j]), 4 * static_cast<size_t>(bcap), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->bmin[j]), 4 * static_cast<size_t>(bcap), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ikey[j]), 8 * isize, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ibid[j]), 4 * isize, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lstale[j]), n, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lfree[j]), 4 * static_cast<size_t>(bcap), s))) {
            inc_release(ctx, s);
            return cuda_error(ctx, e, "alloc incremental state");
        }
    }
    ctx->inc_k = K;
    ctx->inc_small_max = ctx->opt.small_max_degree;
    Scratch* Sp = new Scratch();
    if ((e = alloc_scratch(ctx, *Sp, s))) {
        delete Sp;
        inc_release(ctx, s);
        return cuda_error(ctx, e, "alloc incremental scratch");
    }
    ctx->inc_ws = Sp;
    return BISIM_OK;
}

// Next unused block id per level, on the host and in the device counters the
// settle kernels draw new ids from, and the free lists: the ids below it whose
// blocks have no members (state import; called once the block records are in).
bisim_status inc_set_next_ids(bisim_ctx* ctx, const int64_t* bnext, cudaStream_t s) {
    if (ctx->inc_ws == nullptr) return set_error(ctx, BISIM_ESTATE, "no incremental state");
    Scratch& S = *static_cast<Scratch*>(ctx->inc_ws);
    constexpr int L = kMaxIncLevels + 1;
    for (int j = 0; j < L; ++j) ctx->bnext[j] = std::max<int64_t>(0, std::min<int64_t>(bnext[j], ctx->bcap));
    cudaError_t e = cudaMemcpyAsync(S.dbnext, ctx->bnext, sizeof(int64_t) * L, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(S.dfree, 0, 24 * L, s);
    for (int j = 0; !e && j <= ctx->inc_k; ++j)
        if (ctx->bnext[j] > 0)
            k_free_collect<<<grid_for(ctx->bnext[j], 256), 256, 0, s>>>(ctx->bcnt[j], ctx->bnext[j], ctx->lfree[j],
                                                                       S.dfree + 3 * j);
    if (!e) e = cudaMemcpyAsync(S.h->fc, S.dfree, 24 * L, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);          // the source is the context's host array
    if (e) return cuda_error(ctx, e, "restore block ids");
    for (int j = 0; j < L; ++j) ctx->nfree[j] = S.h->fc[j][0];
    return BISIM_OK;
}

// Full build of the incremental state: every live vertex is the frontier of
// an empty state at every level.
bisim_status inc_build(bisim_ctx* ctx, cudaStream_t s) {
    const int K = ctx->opt.k_incremental;
    ctx->inc_small_max = ctx->opt.small_max_degree;     // every vertex is the frontier
    if (K > kMaxIncLevels) return set_error(ctx, BISIM_EINVAL, "k_incremental exceeds 16");
    inc_release(ctx, s);
    bisim_status st;
    if ((st = store_build(ctx, s)) != BISIM_OK) return st;
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK) return st;
    if ((st = ensure_skey(ctx, s)) != BISIM_OK) return st;
    const size_t n = static_cast<size_t>(std::max(ctx->n, 1));
    ctx->bcap = 2 * static_cast<int64_t>(n) + 1024;
    uint64_t is = 1024;
    while (is < 3ull * n) is <<= 1;
    ctx->isize = is;
    cudaError_t e;
    for (int j = 0; j <= K; ++j) {
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lid[j]), 4 * n, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lcnt[j]), 4 * n, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->bkey[j]), 8 * static_cast<size_t>(ctx->bcap), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->bcnt[j]), 4 * static_cast<size_t>(ctx->bcap), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->bmin[j]), 4 * static_cast<size_t>(ctx->bcap), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ikey[j]), 8 * is, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ibid[j]), 4 * is, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lstale[j]), n, s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->lfree[j]), 4 * static_cast<size_t>(ctx->bcap), s)))
            return cuda_error(ctx, e, "alloc incremental state");
        cudaMemsetAsync(ctx->lstale[j], 0, n, s);
        cudaMemsetAsync(ctx->lid[j], 0xff, 4 * n, s);        // -1: no block yet
        cudaMemsetAsync(ctx->lcnt[j], 0, 4 * n, s);
        cudaMemsetAsync(ctx->bcnt[j], 0, 4 * static_cast<size_t>(ctx->bcap), s);
        cudaMemsetAsync(ctx->ikey[j], 0, 8 * is, s);
    }
    ctx->inc_k = K;
    Scratch* Sp = new Scratch();
    if ((e = alloc_scratch(ctx, *Sp, s))) {
        delete Sp;
        inc_release(ctx, s);
        return cuda_error(ctx, e, "alloc incremental scratch");
    }
    ctx->inc_ws = Sp;
    Scratch& S = *Sp;
    int64_t fl = 0;
    st = BISIM_OK;
    for (int j = 0; st == BISIM_OK && j <= K; ++j) {
        launch_frontier(ctx, S, j, nullptr, nullptr, nullptr, nullptr, s);
        cudaMemsetAsync(S.chcount, 0, 8, s);          // k_assign lists changed vertices (at most n)
        st = level_pass(ctx, j, S, &fl, s);
        cudaMemsetAsync(S.W.recomp, 0, static_cast<size_t>(std::max(ctx->n, 1)), s);   // every vertex was in F
    }
    bool rebuild = false;
    if (st == BISIM_OK) st = inc_finish(ctx, S, &rebuild, s);
    if (st == BISIM_OK && rebuild) st = set_error(ctx, BISIM_ENOMEM, "incremental state overflow during build");
    if (st != BISIM_OK) {
        inc_release(ctx, s);
        return st;
    }
    ctx->stats.last_frontier = fl;
    ctx->stats.state_builds += 1;
    return BISIM_OK;
}

bisim_status write_current(bisim_ctx* ctx, cudaStream_t s) {
    bisim_status st = write_output(ctx, s);
    if (st != BISIM_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    return e ? cuda_error(ctx, e, "write partition") : BISIM_OK;
}

// n_ops sizes the frontiers to expect: small batches give every frontier row at
// least a warp (thread-per-vertex classes need many rows to fill the GPU).
bisim_status inc_update(bisim_ctx* ctx, const uint8_t* vchanged, const uint8_t* rowchg, int64_t n_ops,
                        cudaStream_t s) {
    ctx->inc_small_max = n_ops > kThreadClassOps ? ctx->opt.small_max_degree : 0;
    bisim_status st;
    if ((st = ensure_skey(ctx, s)) != BISIM_OK) return st;
    const int K = ctx->inc_k;
    const int32_t n = ctx->n;
    Scratch& S = *static_cast<Scratch*>(ctx->inc_ws);
    Work& W = S.W;
    int64_t total = 0;
    for (int j = 0; st == BISIM_OK && j <= K; ++j) {
        if (j > 0) {
            // F_j: block changed one level down, out-edges changed, or an out-edge into a
            // changed vertex (its source is in the changed vertex's in-row)
            cudaMemsetAsync(W.next, 0, n, s);
            cudaMemsetAsync(S.tiers.cnt, 0, 16, s);
            if (n > 0) {
                BISIM_SITE(site, "inc_in_neighbours");
                Launch L(site, s, n, 0, 1.0 * n);
                k_in_row_tasks<<<kTierGrid, kTierThreads, 0, s>>>(S.clist, S.chcount, ctx->yro, ctx->ylen, S.tiers);
                run_tiers(S.tiers, MarkSources{ctx->ype, W.next}, s);
            }
            launch_frontier(ctx, S, j, W.next, W.changed, rowchg, W.recomp, s);
            cudaMemsetAsync(W.recomp, 0, n, s);       // this level's assign flags the next level's
        } else {
            launch_frontier(ctx, S, j, vchanged, nullptr, nullptr, nullptr, s);
        }
        cudaMemsetAsync(W.changed, 0, n, s);
        cudaMemsetAsync(S.chcount, 0, 8, s);          // the level lists its changed vertices
        int64_t fl = 0;
        st = level_pass(ctx, j, S, &fl, s);
        total += fl;
    }
    bool rebuild = false;
    if (st == BISIM_OK) st = inc_finish(ctx, S, &rebuild, s);
    if (st != BISIM_OK) {
        inc_release(ctx, s);      // the state may be half-updated: the next batch rebuilds it
        return st;
    }
    // out of block ids or index slots: start over from the current graph. The
    // next batch takes at most n ids, the free ones first; the index holds the
    // live blocks' keys and the tombstones. An index that is full mostly of
    // tombstones is refilled in place instead.
    bool full = rebuild;
    bool refilled = false;
    for (int j = 0; j <= K && !full; ++j) {
        const int64_t in_use = ctx->bnext[j] - ctx->nfree[j];
        if (ctx->bnext[j] + std::max<int64_t>(0, n - ctx->nfree[j]) >= ctx->bcap ||
            static_cast<uint64_t>(in_use) * 2 > ctx->isize) {
            full = true;
        } else if (static_cast<uint64_t>(in_use + ctx->itomb[j]) * 10 > ctx->isize * 7) {
            BISIM_SITE(site, "inc_index_refill");
            Launch Lk(site, s, in_use, 0, 12.0 * ctx->bnext[j] + 8.0 * ctx->isize);
            cudaMemsetAsync(ctx->ikey[j], 0, 8 * ctx->isize, s);
            k_index_refill<<<grid_for(ctx->bnext[j], 256), 256, 0, s>>>(ctx->bcnt[j], ctx->bkey[j], ctx->bnext[j],
                                                                       ctx->ikey[j], ctx->ibid[j], ctx->isize - 1,
                                                                       S.W.err);
            ctx->itomb[j] = 0;
            refilled = true;
        }
    }
    if (full) return inc_build(ctx, s);
    if (refilled) {
        cudaMemcpyAsync(&S.h->err, S.W.err, 4, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) {
            inc_release(ctx, s);
            return cuda_error(ctx, e, "index refill");
        }
        if (S.h->err) {
            inc_release(ctx, s);
            return set_error(ctx, BISIM_EINVAL, "incremental index refill failed its self-check");
        }
    }
    ctx->stats.last_frontier = total;
    return BISIM_OK;
}

}  // namespace bisim
