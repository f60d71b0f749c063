// Dense refinement rounds: every live vertex recomputes its signature in every
// round (Algorithm 4, Section 3.3.1, made exact as in the definition of
// Section 2.5).
//
// The out-CSR is copied once per graph version into a layout made for these
// rounds. Live vertices are grouped by out-degree class ("positions", ascending
// vertex id inside a class) and their rows are stored in position order as
// packed 8-byte words (label << 32 | target). Consecutive threads then read
// consecutive edges whatever the vertex ids are, and every class runs as one
// kind of work unit:
//   degree <= 32    one thread per vertex, the row's pair values in registers,
//                   a value counted when no earlier one equals it;
//   degree <= 256   one warp per vertex with a set in shared memory;
//   degree <= 8192  one CTA per vertex with a set in shared memory;
//   above           the row cut into chunks over many CTAs; its values are
//                   bucketed by a mix of their bits and every bucket is
//                   deduplicated by one CTA in shared memory.
// Each vertex's signature hash goes into the open-addressing table, whose slots
// keep the smallest vertex (the canonical block id). A verification pass then
// confirms every vertex against its slot's representative by recomputing both
// pair sets (no list is stored): inside the lane group for small degrees, in a
// CTA per pair otherwise. Vertices whose signature differs from their
// representative's (a hash collision) are re-hashed with a new salt in further
// levels; the smallest vertex of each level's group is final, so the loop ends
// with the exact partition.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, cdiv(n, threads)));
}

constexpr int kMaxLevels = 1 << 16;
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

__device__ __forceinline__ unsigned long long pack_edge(int32_t label, int32_t target) {
    return (static_cast<unsigned long long>(static_cast<uint32_t>(label)) << 32) | static_cast<uint32_t>(target);
}

__device__ __forceinline__ uint64_t packed_pair_value(unsigned long long pk, const int32_t* __restrict__ P) {
    return pair_value(static_cast<int32_t>(pk >> 32), __ldg(P + static_cast<uint32_t>(pk)));
}

__device__ __forceinline__ int ceil_log2(int64_t d) {
    return d <= 1 ? 0 : 64 - __clzll(static_cast<unsigned long long>(d - 1));
}

// Block-aggregated list append: one atomic per CTA rather than per warp, which
// matters when a whole grid adds to a single counter (tens of thousands of
// warps on one address serialise in L2). Every thread of the CTA must call
// it; `sh` holds kThreads / 32 + 1 words of shared memory.

template <class T>
__device__ __forceinline__ void block_push(bool flag, T value, T* list, unsigned* counter, unsigned* sh) {
    constexpr int W = kThreads / 32;
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    const int w = static_cast<int>(threadIdx.x >> 5);
    if (lane_id() == 0) sh[w] = static_cast<unsigned>(__popc(b));
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned total = 0;
        for (int q = 0; q < W; ++q) {
            const unsigned c = sh[q];
            sh[q] = total;
            total += c;
        }
        sh[W] = total ? atomicAdd(counter, total) : 0u;
    }
    __syncthreads();
    if (flag) list[sh[W] + sh[w] + __popc(b & lanemask_lt())] = value;
    __syncthreads();                                 // sh is free for the next call
}

// Exclusive scan of in[0..len) into out (which may be in) by one CTA of 1024
// threads; every thread gets the total. Chunks of 1024 values: a warp scan,
// a scan of the 32 warp sums, and a carry between chunks.
__device__ int64_t cta_exclusive_scan(const int64_t* in, int64_t* out, int64_t len) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < len; b += 1024) {
        const int64_t t = b + threadIdx.x;
        const int64_t x = t < len ? in[t] : 0;
        int64_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (static_cast<int>(lane_id()) >= o) inc += y;
        }
        if (lane_id() == 31) wsum[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            int64_t w = wsum[threadIdx.x];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (static_cast<int>(threadIdx.x) >= o) w += y;
            }
            wsum[threadIdx.x] = w;                       // inclusive over warps
        }
        __syncthreads();
        const int64_t before = carry + (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0) + inc - x;
        if (t < len) out[t] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + x;
        __syncthreads();
    }
    return carry;
}

// ----------------------------------------------------------------------------- layout kernels

__global__ void k_deg_from_rows(const int64_t* __restrict__ rp, int32_t n, int32_t* __restrict__ deg) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) deg[v] = static_cast<int32_t>(rp[v + 1] - rp[v]);
}

__global__ void k_dense_classify(const int32_t* __restrict__ deg, const uint8_t* __restrict__ alive, int32_t n,
                                 int small_max, int mid_max, uint32_t* __restrict__ keys,
                                 uint64_t* __restrict__ vals) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int64_t d = deg[v];
    uint32_t c;
    if (alive != nullptr && !alive[v]) {
        c = kDDead;
    } else if (d == 0) {
        c = 0;
    } else if (d <= small_max) {
        c = 1u + static_cast<uint32_t>(ceil_log2(d));                // 1..6
    } else if (d <= mid_max) {
        const int lg = max(6, ceil_log2(d));
        c = lg <= 8 ? static_cast<uint32_t>(kDWarp0 + (lg - 6)) : static_cast<uint32_t>(kDMid0 + (lg - 9));
    } else {
        c = kDHub;
    }
    keys[v] = c;
    vals[v] = static_cast<uint64_t>(v);
}

// begin[c] = first position of class c (classes absent in between start there too).
__global__ void k_dense_bounds(const uint32_t* __restrict__ sk, int32_t n, int64_t* __restrict__ begin) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = static_cast<int>(min(sk[i], static_cast<uint32_t>(kDClasses)));
    const int p = i == 0 ? -1 : static_cast<int>(min(sk[i - 1], static_cast<uint32_t>(kDClasses)));
    for (int q = p + 1; q <= c; ++q) begin[q] = i;
}

__global__ void k_dense_vertices(const uint64_t* __restrict__ sv, int32_t n, int32_t* __restrict__ vert,
                                 int32_t* __restrict__ vpos) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = static_cast<int32_t>(sv[i]);
    vert[i] = v;
    vpos[v] = static_cast<int32_t>(i);
}

__global__ void k_dense_degrees(const int32_t* __restrict__ vert, int64_t n_live, const int32_t* __restrict__ deg,
                                int64_t* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i > n_live) return;
    out[i] = i == n_live ? 0 : deg[vert[i]];
}

// Vertex-ordered out-degrees back from the layout (dead vertices: 0).
__global__ void k_vertex_degrees(const int32_t* __restrict__ vpos, int32_t n, int64_t n_live,
                                 const int64_t* __restrict__ prp, int64_t* __restrict__ deg) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v > n) return;
    if (v == n) {
        deg[v] = 0;
        return;
    }
    const int64_t p = vpos[v];
    deg[v] = p < n_live ? prp[p + 1] - prp[p] : 0;
}

// Vertex-ordered rows of at most 256 edges from the packed rows: one warp per
// 32 consecutive vertices. The warp's short rows are numbered consecutively
// (a warp scan of their lengths); every word finds its row by a binary search
// over the 33 prefix values in shared memory. Longer rows are left to
// k_unpack_big and k_unpack_chunks.
__global__ void __launch_bounds__(256) k_unpack_rows(const int32_t* __restrict__ vpos, int32_t n, int64_t n_live,
                                                     const int64_t* __restrict__ prp,
                                                     const unsigned long long* __restrict__ pe,
                                                     const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                                                     int32_t* __restrict__ elab) {
    __shared__ int64_t pre_all[8][33];
    __shared__ int64_t dst_all[8][32];
    __shared__ int64_t src_all[8][32];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t v0 = (static_cast<int64_t>(blockIdx.x) * 8 + warp) * 32;
    if (v0 >= n) return;                                 // whole warp leaves together
    int64_t* pre = pre_all[warp];
    int64_t* dst = dst_all[warp];
    int64_t* src = src_all[warp];
    const int64_t v = v0 + lane;
    int64_t a = 0, d = 0, sp = 0;
    if (v < n) {
        a = rp[v];
        d = rp[v + 1] - a;
        if (d > 256) d = 0;
        const int64_t p = vpos[v];
        sp = p < n_live ? prp[p] : 0;
    }
    int64_t incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (static_cast<int>(lane) >= o) incl += y;
    }
    pre[lane] = incl - d;
    dst[lane] = a;
    src[lane] = sp;
    if (lane == 31) pre[32] = incl;
    __syncwarp();
    const int64_t total = pre[32];
    for (int64_t t = lane; t < total; t += 32) {
        int lo = 0, hi = 31;                             // the last row starting at or before t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int64_t off = t - pre[lo];
        const unsigned long long w = pe[src[lo] + off];
        col[dst[lo] + off] = static_cast<int32_t>(static_cast<uint32_t>(w));
        elab[dst[lo] + off] = static_cast<int32_t>(w >> 32);
    }
}

// Longer rows (CTA classes): one CTA per position.
__global__ void k_unpack_big(const int32_t* __restrict__ vert, int64_t first, const int64_t* __restrict__ prp,
                             const unsigned long long* __restrict__ pe, const int64_t* __restrict__ rp,
                             int32_t* __restrict__ col, int32_t* __restrict__ elab) {
    const int64_t i = first + blockIdx.x;
    const int64_t o = rp[vert[i]];
    const int64_t b = prp[i], d = prp[i + 1] - b;
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
        const unsigned long long w = pe[b + j];
        col[o + j] = static_cast<int32_t>(static_cast<uint32_t>(w));
        elab[o + j] = static_cast<int32_t>(w >> 32);
    }
}

// Rows of out-degree <= 256: one warp per 32 consecutive positions. The warp's
// output range is contiguous, so it is written word by word across the lanes;
// each word finds its source row by a binary search over the warp's 33 row
// offsets in shared memory.
__global__ void __launch_bounds__(256) k_dense_pack_rows(const int32_t* __restrict__ vert, int64_t count,
                                                         const int64_t* __restrict__ prp,
                                                         const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col,
                                                         const int32_t* __restrict__ elab,
                                                         unsigned long long* __restrict__ pe) {
    __shared__ int64_t off_all[8][33];
    __shared__ int64_t src_all[8][32];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t p0 = (static_cast<int64_t>(blockIdx.x) * 8 + warp) * 32;
    if (p0 >= count) return;                             // whole warp leaves together
    int64_t* off = off_all[warp];
    int64_t* src = src_all[warp];
    const int64_t pend = min(count, p0 + 32);
    const int64_t p = p0 + lane;
    const bool act = p < count;
    off[lane] = prp[act ? p : pend];                     // rows past the end start at the end
    if (lane == 0) off[32] = prp[pend];
    src[lane] = act ? rp[vert[p]] : 0;
    __syncwarp();
    const int64_t o1 = off[32];
    for (int64_t o = off[0] + lane; o < o1; o += 32) {
        int lo = 0, hi = 31;                             // the last row starting at or before o
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= o) lo = mid; else hi = mid - 1;
        }
        const int64_t e = src[lo] + (o - off[lo]);
        pe[o] = pack_edge(elab[e], col[e]);
    }
}

// Rows of out-degree <= 8192: one CTA per position.
__global__ void k_dense_pack_big(const int32_t* __restrict__ vert, int64_t first, const int64_t* __restrict__ prp,
                                 const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ elab, unsigned long long* __restrict__ pe) {
    const int64_t i = first + blockIdx.x;
    const int32_t v = vert[i];
    const int64_t b = rp[v];
    const int64_t d = rp[v + 1] - b;
    const int64_t o = prp[i];
    for (int64_t j = threadIdx.x; j < d; j += blockDim.x) pe[o + j] = pack_edge(elab[b + j], col[b + j]);
}

// Hub rows: one CTA per chunk of a row.
__global__ void k_dense_pack_chunks(const HubChunk* __restrict__ chunks, const int32_t* __restrict__ vert,
                                    int64_t first, const int64_t* __restrict__ prp, const int64_t* __restrict__ rp,
                                    const int32_t* __restrict__ col, const int32_t* __restrict__ elab,
                                    unsigned long long* __restrict__ pe) {
    const HubChunk c = chunks[blockIdx.x];
    const int64_t pos = first + c.hub;
    const int64_t src = rp[vert[pos]] - prp[pos];        // source index = packed index + src
    for (int64_t o = c.begin + threadIdx.x; o < c.end; o += blockDim.x) pe[o] = pack_edge(elab[src + o], col[src + o]);
}

// Hub rows back to vertex order: one CTA per chunk.
__global__ void k_unpack_chunks(const HubChunk* __restrict__ chunks, const int32_t* __restrict__ vert, int64_t first,
                                const int64_t* __restrict__ prp, const unsigned long long* __restrict__ pe,
                                const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                                int32_t* __restrict__ elab) {
    const HubChunk c = chunks[blockIdx.x];
    const int64_t pos = first + c.hub;
    const int64_t dst = rp[vert[pos]] - prp[pos];        // vertex-ordered index = packed index + dst
    for (int64_t e = c.begin + threadIdx.x; e < c.end; e += blockDim.x) {
        const unsigned long long w = pe[e];
        col[dst + e] = static_cast<int32_t>(static_cast<uint32_t>(w));
        elab[dst + e] = static_cast<int32_t>(w >> 32);
    }
}

__global__ void k_dense_dead(const int32_t* __restrict__ vert, int64_t first, int64_t n, int32_t* __restrict__ Pa,
                             int32_t* __restrict__ Pb) {
    const int64_t i = first + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = vert[i];
    Pa[v] = -1;
    Pb[v] = -1;
}

// ----------------------------------------------------------------------------- round kernels

struct DenseView {
    const int32_t* vert;               // position -> vertex
    const int32_t* vpos;               // vertex -> position
    const int64_t* prp;                // position -> offset into pe
    const unsigned long long* pe;      // packed (label, target) rows
    const int32_t* P;                  // P_i, by vertex
    SigRec* sig;                       // signature hash, |S| and own block, by position
    uint32_t* slot;                    // table slot, by position
    uint8_t* joined;                   // by position: another vertex joined its block in the last round
    uint8_t* own;                      // by position: the vertex was its block's id (smallest member) in the last round
    const int32_t* gid;                // batched contexts: graph of each vertex (null: one graph)
    const int64_t* rbase;              // batched contexts: the graph's table region
    const uint32_t* rmask;
    unsigned long long* work;          // launch profiling only: rows and row entries each group processed
    const int32_t* act;                // active positions (not alone in their block), ascending
    const int64_t* aoff;               // [kDClasses + 1] class c's entries are act[aoff[c] .. aoff[c+1])
    const int32_t* round_no;           // captured loop: rounds run so far, which picks the table epoch (null: eager)
};

// Work counters of the signature kernels, filled only while launch profiling
// is on (vertices alone in their block skip their row, so the work done per
// round is known only on the device). Groups follow the launch sites: thread
// classes 8 / 16 / 32, the warp classes, the five CTA classes, the hubs; each
// counter is spread over kWorkSpread words to keep atomics off one address.
constexpr int kWorkGroups = 10;
constexpr int kWorkSpread = 16;
constexpr int kWorkWords = kWorkGroups * 2 * kWorkSpread;
constexpr int kWorkHub = 9;

__device__ __forceinline__ void work_add(const DenseView& D, int g, unsigned long long rows,
                                         unsigned long long edges) {
    const int k = static_cast<int>(blockIdx.x) & (kWorkSpread - 1);
    if (rows) atomicAdd(&D.work[(g * 2) * kWorkSpread + k], rows);
    if (edges) atomicAdd(&D.work[(g * 2 + 1) * kWorkSpread + k], edges);
}

// CTA-wide sum of the active threads' rows and entries (every thread calls it).
__device__ __forceinline__ void work_block(const DenseView& D, int g, bool active, unsigned d) {
    if (D.work == nullptr) return;                    // uniform: the same for the whole grid
    __shared__ unsigned long long esum;
    if (threadIdx.x == 0) esum = 0ull;
    unsigned long long w = active ? d : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    __syncthreads();
    if ((threadIdx.x & 31u) == 0u && w) atomicAdd(&esum, w);
    const int rows = __syncthreads_count(active);
    if (threadIdx.x == 0) work_add(D, g, static_cast<unsigned long long>(rows), esum);
}

// A vertex alone in its block of P_i stays alone in P_{i+1}: no signature is
// needed. The hub passes test this per chunk; every other kernel of a round
// walks the active list, which holds only the vertices that are not alone.
// The flags are those of the previous round until the level-0 insert clears
// the joined flags of the listed positions.
__device__ __forceinline__ bool alone_last_round(const DenseView& D, int64_t pos) {
    return D.own[pos] && !D.joined[pos];
}

__device__ __forceinline__ void finish_sig(const DenseView& D, int64_t pos, int32_t own, uint32_t c, uint64_t sum) {
    SigRec r;
    r.hash = sig_hash(own, c, sum);
    r.cnt = static_cast<int32_t>(c);
    r.own = own;
    D.sig[pos] = r;
}

// Degree <= D: one thread per active vertex of the classes [c0, c1). The row's
// pair values sit in registers; a value counts when no earlier value of the
// row equals it.
template <int D>
__global__ void __launch_bounds__(kThreads) k_dense_thread_sig(int c0, int c1, const DenseView V, int group) {
    const int64_t a0 = V.aoff[c0];
    const int64_t count = V.aoff[c1] - a0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x;
    int32_t next = base + threadIdx.x < count ? V.act[a0 + base + threadIdx.x] : 0;
    for (; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool active = i < count;
        const int64_t pos = next;
        if (i + stride < count) next = V.act[a0 + i + stride];     // the next entry's load overlaps this one
        int d = 0;
        if (active) {
            const int32_t own = V.P[V.vert[pos]];
            const int64_t e0 = V.prp[pos];
            d = static_cast<int>(V.prp[pos + 1] - e0);
            uint64_t v[D];
#pragma unroll
            for (int j = 0; j < D; ++j) v[j] = j < d ? packed_pair_value(__ldcs(V.pe + e0 + j), V.P) : 0ull;
            uint64_t sum = 0;
            uint32_t u = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                bool fresh = j < d;
#pragma unroll
                for (int q = 0; q < j; ++q) fresh = fresh && v[q] != v[j];
                if (fresh) {
                    sum += v[j];
                    ++u;
                }
            }
            finish_sig(V, pos, own, u, sum);
        }
        work_block(V, group, active, static_cast<unsigned>(d));
    }
}

// Degree <= 256: one warp per active vertex, set of up to 512 slots in the
// warp's slice of shared memory. All of the row's words are loaded, then all
// of their block ids gathered, before the first set insert, so that a warp
// keeps up to eight loads of each kind in flight.
constexpr int kWarpSlots = 512;
constexpr int kWarpChunks = 8;                         // 256 / 32
__global__ void __launch_bounds__(kThreads) k_dense_warp_sig(const DenseView D) {
    __shared__ unsigned long long sm_all[(kThreads / 32) * kWarpSlots];
    __shared__ unsigned zero_all[kThreads / 32];
    const int64_t a0 = D.aoff[kDWarp0];
    const int64_t count = D.aoff[kDMid0] - a0;
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    unsigned long long* tab = sm_all + warp * kWarpSlots;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * (kThreads / 32);
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * (kThreads / 32); base < count; base += stride) {
        const int64_t w = base + warp;
        const bool active = w < count;                 // the same for the whole warp
        int64_t pos = 0, e0 = 0;
        int d = 0;
        if (active) {
            pos = D.act[a0 + w];
            e0 = D.prp[pos];
            d = static_cast<int>(D.prp[pos + 1] - e0);
        }
        if (D.work) work_block(D, 3, active && lane == 0, active ? static_cast<unsigned>(d) : 0u);
        if (!active) continue;
        const int32_t own = lane == 0 ? D.P[D.vert[pos]] : 0;
        uint64_t mv[kWarpChunks];
#pragma unroll
        for (int k = 0; k < kWarpChunks; ++k) {
            const int j = k * 32 + static_cast<int>(lane);
            mv[k] = j < d ? __ldcs(D.pe + e0 + j) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < kWarpChunks; ++k)
            if (k * 32 + static_cast<int>(lane) < d) mv[k] = packed_pair_value(mv[k], D.P);
        uint32_t S = 64;
        while (S < 2u * static_cast<uint32_t>(d)) S <<= 1;
        for (uint32_t j = lane; j < S; j += 32) tab[j] = 0ull;
        if (lane == 0) zero_all[warp] = 0u;
        __syncwarp();
        unsigned out = 0;
        uint64_t mys = 0;
#pragma unroll
        for (int k = 0; k < kWarpChunks; ++k) {
            if (k * 32 >= d) break;                    // the same for the whole warp
            const int j = k * 32 + static_cast<int>(lane);
            const bool fresh = j < d && smem_set_insert(tab, S - 1, &zero_all[warp], mv[k]);
            out += static_cast<unsigned>(__popc(__ballot_sync(0xffffffffu, fresh)));
            if (fresh) mys += mv[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mys += __shfl_xor_sync(0xffffffffu, mys, o);
        if (lane == 0) finish_sig(D, pos, own, out, mys);
        __syncwarp();                                  // the slice is cleared for the warp's next vertex
    }
}

// Degree <= N (N = 512 .. 8192): one CTA of T threads per active vertex of
// class `cls`, set of 2N slots; each thread loads four words before it
// gathers and inserts them.
constexpr int kMidUnroll = 4;
template <int N, int T>
__global__ void __launch_bounds__(T) k_dense_mid_sig(int cls, const DenseView D, int group) {
    extern __shared__ unsigned long long tab[];
    __shared__ unsigned long long wsum[T / 32];
    __shared__ unsigned wcnt[T / 32];
    __shared__ unsigned zero;
    constexpr uint32_t mask = 2 * N - 1;
    const int64_t a0 = D.aoff[cls];
    const int64_t count = D.aoff[cls + 1] - a0;
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        const int64_t pos = D.act[a0 + it];
        const int64_t e0 = D.prp[pos];
        const int d = static_cast<int>(D.prp[pos + 1] - e0);
        if (D.work && threadIdx.x == 0) work_add(D, group, 1, static_cast<unsigned long long>(d));
        for (int j = threadIdx.x; j < 2 * N; j += T) tab[j] = 0ull;
        if (threadIdx.x == 0) zero = 0u;
        __syncthreads();
        uint64_t mys = 0;
        unsigned myc = 0;
        for (int j0 = threadIdx.x; j0 < d; j0 += kMidUnroll * T) {
            uint64_t mv[kMidUnroll];
#pragma unroll
            for (int k = 0; k < kMidUnroll; ++k) {
                const int j = j0 + k * T;
                mv[k] = j < d ? __ldcs(D.pe + e0 + j) : 0ull;
            }
#pragma unroll
            for (int k = 0; k < kMidUnroll; ++k)
                if (j0 + k * T < d) mv[k] = packed_pair_value(mv[k], D.P);
#pragma unroll
            for (int k = 0; k < kMidUnroll; ++k) {
                if (j0 + k * T < d && smem_set_insert(tab, mask, &zero, mv[k])) {
                    mys += mv[k];
                    ++myc;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mys += __shfl_xor_sync(0xffffffffu, mys, o);
            myc += __shfl_xor_sync(0xffffffffu, myc, o);
        }
        if (lane_id() == 0) {
            wsum[threadIdx.x >> 5] = mys;
            wcnt[threadIdx.x >> 5] = myc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t sm = 0;
            unsigned c = 0;
            for (int w = 0; w < T / 32; ++w) {
                sm += wsum[w];
                c += wcnt[w];
            }
            finish_sig(D, pos, D.P[D.vert[pos]], c, sm);
        }
        __syncthreads();                               // the set is cleared for the CTA's next vertex
    }
}

// Hub rows (above the CTA classes) are cut into chunks over many CTAs. Every
// hub has an open-addressing table in global memory with two slots per row
// entry: the chunk of packed edges [b, e) owns slots [2b, 2e), counted from
// the first hub edge, so the tables need no layout of their own and are never
// more than half full. A round first clears the tables of the listed hubs
// (k_hub_clear); then every chunk filters its pair values through a small
// shared-memory set and inserts the values new to the chunk into its hub's
// table (k_hub_insert). The inserter that finds a value's slot empty adds the
// value to the hub's count and sum, so a value repeated within a chunk or
// across chunks is counted once: count and sum are those of the hub's set.
struct HubSets {
    int64_t first;                 // position of the first hub
    int64_t n_hub;
    unsigned long long* tab;       // two slots per hub edge (0 = empty; the value 0 is acc[h].zero)
    int64_t e0;                    // first hub edge in the packed rows
    HubAcc* acc;
};

// No hub is listed this round (every hub is alone in its block): the hub
// passes, whose resident grids stride over all chunks, return at once.
__device__ __forceinline__ bool no_hub_listed(const DenseView& D) {
    return D.aoff[kDHub + 1] == D.aoff[kDHub];
}

// Sub-ranges of a salted mix of the pair values, taken by the set comparison
// of two long rows when one shared-memory set cannot hold a row.
constexpr uint64_t kSaltBucket = 0x452821e638d01377ull;
constexpr int kHubMaxSplits = 1 << 12;          // sub-ranges tried before the comparison gives up

__device__ __forceinline__ uint64_t bucket_mix(uint64_t mv) { return mix64(mv ^ kSaltBucket); }

// Sub-range `sub` of `splits`: the top bits of the mix after its first `shift`.
__device__ __forceinline__ uint32_t split_of(uint64_t mixed, int shift, uint32_t splits) {
    return splits <= 1 ? 0u : static_cast<uint32_t>((mixed << shift) >> (64 - __ffs(splits) + 1));
}

// Pass 1: the listed hubs' table slots are cleared, chunk by chunk (16 bytes
// per edge, the two slots it owns).
__global__ void __launch_bounds__(kThreads) k_hub_clear(const HubChunk* __restrict__ chunks, int64_t n_chunks,
                                                        const DenseView D, const HubSets H) {
    if (no_hub_listed(D)) return;
    for (int64_t ci = blockIdx.x; ci < n_chunks; ci += gridDim.x) {
        const HubChunk c = chunks[ci];
        if (alone_last_round(D, H.first + c.hub)) continue;          // the same for the whole CTA
        ulonglong2* t = reinterpret_cast<ulonglong2*>(H.tab + 2 * (c.begin - H.e0));
        const int64_t cnt = c.end - c.begin;
        for (int64_t j = threadIdx.x; j < cnt; j += kThreads) t[j] = make_ulonglong2(0ull, 0ull);
    }
}

// Insert of a nonzero pair value into a hub's table of `size` slots (linear
// probing from hub_slot, the value's high half scaled to the table). Slots
// only go from empty to a value within a round, so a plain read that sees the
// value is final and one that sees an empty slot is settled by the
// compare-and-swap. `first` is the caller's read of the first slot (so that a
// thread's reads for several values are in flight together). True for the
// inserter that placed the value.
__device__ __forceinline__ uint64_t hub_slot(unsigned long long mv, uint64_t size) {
    return ((mv >> 32) * size) >> 32;
}

__device__ __forceinline__ bool hub_table_insert(unsigned long long* tab, uint64_t size, unsigned long long mv,
                                                 unsigned long long first, unsigned* err) {
    uint64_t at = hub_slot(mv, size);
    for (uint64_t probe = 0; probe < size; ++probe) {
        const unsigned long long cur = probe == 0 ? first : tab[at];
        if (cur == mv) return false;
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&tab[at], 0ull, mv);
            if (prev == 0ull) return true;
            if (prev == mv) return false;
        }
        if (++at == size) at = 0;
    }
    atomicOr(err, kErrHubFull);                        // unreachable: the table has two slots per edge
    return false;
}

// Pass 2: per chunk, its values go through a shared-memory set of
// kHubLocalSlots slots (a filter only: once it holds kHubLocalLimit values,
// the rest go to the table directly); the values new to the set, and those
// that bypass it, are inserted into the hub's table, the first table reads of
// a thread's kHubUnroll values in flight together. The CTA adds its new
// values' count and sum to the hub's accumulator once per chunk. The filter
// is small on purpose: eight CTAs per SM hide the table reads' latency, and
// on the 10M-vertex power-law graph a 32 KB filter (six CTAs per SM) made the
// pass 2.5 times slower than this 16 KB one, and no filter 15% slower.
constexpr int kHubUnroll = 4;
constexpr int kHubLocalSlots = 2048;                   // 16 KB
constexpr int kHubLocalLimit = 512;                    // checked once per iteration of kThreads * kHubUnroll values
static_assert(kHubLocalLimit + kThreads * kHubUnroll <= 3 * kHubLocalSlots / 4, "hub filter can fill up");
constexpr size_t kHubInsertSmem = sizeof(unsigned long long) * kHubLocalSlots;
__global__ void __launch_bounds__(kThreads) k_hub_insert(const HubChunk* __restrict__ chunks, int64_t n_chunks,
                                                         const DenseView D, const HubSets H, unsigned* err) {
    extern __shared__ unsigned long long set[];                    // kHubLocalSlots
    __shared__ unsigned zero, used;
    __shared__ unsigned long long wsum[kThreads / 32];
    __shared__ unsigned wcnt[kThreads / 32];
    if (no_hub_listed(D)) return;
    for (int64_t ci = blockIdx.x; ci < n_chunks; ci += gridDim.x) {
        const HubChunk c = chunks[ci];
        const int64_t hp = H.first + c.hub;
        if (alone_last_round(D, hp)) continue;                       // the same for the whole CTA
        if (D.work && threadIdx.x == 0)
            work_add(D, kWorkHub, c.begin == D.prp[hp] ? 1 : 0, static_cast<unsigned long long>(c.end - c.begin));
        for (int j = threadIdx.x; j < kHubLocalSlots; j += kThreads) set[j] = 0ull;
        if (threadIdx.x == 0) {
            zero = 0u;
            used = 0u;
        }
        const int64_t rb = D.prp[hp];
        const uint64_t size = 2 * static_cast<uint64_t>(D.prp[hp + 1] - rb);
        unsigned long long* tab = H.tab + 2 * (rb - H.e0);
        HubAcc* acc = H.acc + c.hub;
        __syncthreads();
        uint64_t sum = 0;
        unsigned cnt = 0;
        for (int64_t b0 = c.begin; b0 < c.end; b0 += static_cast<int64_t>(kThreads) * kHubUnroll) {
            // loads, then gathers, then the filter, then the first table reads of
            // all the thread's values, before any value waits on its own chain
            uint64_t mv[kHubUnroll];
            bool send[kHubUnroll];
#pragma unroll
            for (int k = 0; k < kHubUnroll; ++k) {
                const int64_t e = b0 + static_cast<int64_t>(k) * kThreads + threadIdx.x;
                mv[k] = e < c.end ? __ldcs(D.pe + e) : 0ull;
            }
#pragma unroll
            for (int k = 0; k < kHubUnroll; ++k) {
                send[k] = b0 + static_cast<int64_t>(k) * kThreads + threadIdx.x < c.end;
                if (send[k]) mv[k] = packed_pair_value(mv[k], D.P);
            }
            const bool room = *reinterpret_cast<volatile unsigned*>(&used) < static_cast<unsigned>(kHubLocalLimit);
            unsigned added = 0;
#pragma unroll
            for (int k = 0; k < kHubUnroll; ++k) {
                if (!send[k]) continue;
                if (mv[k] == 0ull) {
                    send[k] = false;
                    if (atomicExch(&acc->zero, 1u) == 0u) ++cnt;         // the value 0 adds nothing to the sum
                } else if (room) {
                    send[k] = smem_set_insert(set, kHubLocalSlots - 1, &zero, mv[k]);
                    added += send[k] ? 1u : 0u;
                }
            }
            // one shared add per warp for the filter's fill
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) added += __shfl_xor_sync(0xffffffffu, added, o);
            if (lane_id() == 0 && added) atomicAdd(&used, added);
            unsigned long long first[kHubUnroll];
#pragma unroll
            for (int k = 0; k < kHubUnroll; ++k) first[k] = send[k] ? tab[hub_slot(mv[k], size)] : 0ull;
#pragma unroll
            for (int k = 0; k < kHubUnroll; ++k) {
                if (send[k] && hub_table_insert(tab, size, mv[k], first[k], err)) {
                    sum += mv[k];
                    ++cnt;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane_id() == 0) {
            wsum[threadIdx.x >> 5] = sum;
            wcnt[threadIdx.x >> 5] = cnt;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t s2 = 0;
            unsigned c2 = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                s2 += wsum[w];
                c2 += wcnt[w];
            }
            if (c2) {
                atomicAdd(&acc->sum, static_cast<unsigned long long>(s2));
                atomicAdd(&acc->count, c2);
            }
        }
        __syncthreads();                               // the set and the sums are reused by the next chunk
    }
}

// Hubs, phase 2: one thread per hub finishes its signature (the value 0, when
// present, was counted by its first inserter).
__global__ void k_dense_hub_finalize(const DenseView D, const HubSets H) {
    const int64_t h = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (h >= H.n_hub) return;
    if (no_hub_listed(D)) return;
    const int64_t pos = H.first + h;
    if (alone_last_round(D, pos)) return;
    finish_sig(D, pos, D.P[D.vert[pos]], H.acc[h].count, H.acc[h].sum);
}


// Hub chunks from the hub rows' offsets rows[0..nh] (device): hub h's row
// [rows[h], rows[h+1]) in chunks of csz entries, hubs in order. One CTA of
// 1024 threads; off[nh] is scratch for the chunk counts and their offsets.
__global__ void __launch_bounds__(1024) k_hub_chunks(const int64_t* __restrict__ rows, int64_t nh, int64_t csz,
                                                     int64_t* __restrict__ off, HubChunk* __restrict__ out) {
    for (int64_t h = threadIdx.x; h < nh; h += blockDim.x) off[h] = (rows[h + 1] - rows[h] + csz - 1) / csz;
    __syncthreads();
    cta_exclusive_scan(off, off, nh);
    __syncthreads();
    for (int64_t h = threadIdx.x; h < nh; h += blockDim.x) {
        const int64_t rb = rows[h], re = rows[h + 1];
        int64_t c = off[h];
        for (int64_t b = rb; b < re; b += csz, ++c) {
            HubChunk k;
            k.hub = static_cast<int32_t>(h);
            k.vertex = -1;
            k.begin = b;
            k.end = b + csz < re ? b + csz : re;
            out[c] = k;
        }
    }
}

// Start of a round: the status word, with the vertices that are not listed
// (alone in their block of P_i, hence alone in P_{i+1}) already counted as
// blocks and the list's length as the positions that need the table.
__global__ void k_round_begin(DevState* st, const int64_t* __restrict__ aoff, int64_t n_live) {
    const int64_t listed = aoff[kDClasses];
    DevState z{};
    z.blocks = static_cast<unsigned long long>(n_live - listed);
    z.listed = static_cast<unsigned>(listed);
    *st = z;
}

// Table insert of the listed positions with the level's salted hash. The count
// is read on the device when `dcount` is given (level 0), else it is `count`.
// Level 0 also clears the listed positions' joined flags, which this round's
// verification sets again. One entry per thread and iteration: the kernel is
// bound by the latency of its dependent loads (list, hash, table slot), and
// taking several entries per thread to overlap their chains was measured
// slower (0.58 against 0.27 ms for 10M positions), because the registers that
// needs halve the resident warps (the same holds for the verification, 108
// registers and a quarter of the warps at four entries per thread).
constexpr int kPersistGrid = 152 * 8;            // full occupancy of 256-thread CTAs
constexpr int kIlp = 1;
__global__ void __launch_bounds__(kThreads) k_dense_insert(const int32_t* __restrict__ list, int64_t count,
                                                           const unsigned* dcount, const DenseView D, uint32_t level,
                                                           const TableRef t, unsigned* err) {
    if (dcount) count = *reinterpret_cast<const volatile unsigned*>(dcount);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * kIlp;
    TableRef tt = t;
    if (D.round_no) tt.epoch = static_cast<uint64_t>((*D.round_no % kEpochCycle) + 1u) << 32;
    // the insert reads its slot before any atomic, so the many vertices of a
    // popular signature mostly find a smaller vertex recorded and leave
    // without one (combining equal hashes within a warp first, with
    // match_any, was measured twice as slow)
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x * kIlp + threadIdx.x; b < count; b += stride) {
        int32_t pos[kIlp], v[kIlp];
        uint64_t h[kIlp], base[kIlp], mask[kIlp];
        unsigned long long first[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const int64_t i = b + static_cast<int64_t>(k) * blockDim.x;
            pos[k] = i < count ? list[i] : -1;
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            if (pos[k] < 0) continue;
            v[k] = D.vert[pos[k]];
            h[k] = level_hash(D.sig[pos[k]].hash, level, tt.hmask);
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            if (pos[k] < 0) continue;
            base[k] = 0;
            mask[k] = tt.mask;
            if (D.gid) {
                // batched graphs: each graph has its own region of the table, so
                // that the inserts of one graph's vertices stay close together
                const int32_t g = D.gid[v[k]];
                base[k] = static_cast<uint64_t>(D.rbase[g]);
                mask[k] = D.rmask[g];
            }
            first[k] = table_read(tt, base[k] + (h[k] & mask[k]));
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            if (pos[k] < 0) continue;
            D.slot[pos[k]] = table_insert_at(tt, h[k], v[k], base[k], mask[k], first[k], err);
            if (level == 0) D.joined[pos[k]] = 0;
        }
    }
}

struct VerifyOut {
    int32_t* Pout;
    int2* pairs;           // (position, representative's position) for k_dense_compare_cta
    int2* small;           // the same for rows of at most 32 edges: k_dense_compare_warp
    int32_t* next;         // positions for the next collision level
    DevState* st;
};

// Confirms every listed position against its slot's representative r (its
// smallest vertex). r itself: a block id. Different own block or set size: the
// position moves to the next level. Equal sizes of at most one pair: the full
// hashes decide exactly. Otherwise the sets are compared: here when both rows
// have at most two edges, else in a warp (rows <= 32) or a CTA. The three
// lists and the block count of a CTA's iteration share one scan: per warp four
// ballot counts, one pass of four threads over the warps (one atomic per
// list) and two barriers; the shared words alternate between iterations.
__global__ void __launch_bounds__(kThreads) k_dense_verify(const int32_t* __restrict__ list, int64_t count,
                                                           const unsigned* dcount, const DenseView D,
                                                           const Slot* __restrict__ slots, const VerifyOut O,
                                                           int32_t n_total) {
    constexpr int W = kThreads / 32;
    __shared__ unsigned sh[2][4][W + 1];
    if (dcount) count = *reinterpret_cast<const volatile unsigned*>(dcount);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int warp = static_cast<int>(threadIdx.x >> 5);
    const unsigned lt = lanemask_lt();
    int par = 0;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < count; base += stride, par ^= 1) {
        const int64_t i = base + threadIdx.x;
        bool own = false, push = false, small = false, big = false;
        int32_t pos = -1, rpos = -1;
        if (i < count) pos = list[i];
        if (pos >= 0) {
            const int32_t v = D.vert[pos];
            const uint32_t sv = D.slot[pos];
            const int32_t r = sv == ~0u ? -1 : table_rep(slots, sv);
            if (r < 0 || r >= n_total) {                     // failed insert, reported through st->error
                atomicOr(&O.st->error, kErrTableFull);
                O.Pout[v] = -1;
            } else if (r == v) {
                O.Pout[v] = v;
                D.own[pos] = 1;
                own = true;
            } else {
                rpos = D.vpos[r];
                D.own[pos] = 0;
                const SigRec a = D.sig[pos], c = D.sig[rpos];
                bool join = false;
                if (a.own != c.own || a.cnt != c.cnt) {
                    push = true;
                } else if (a.cnt <= 1) {
                    // |S| <= 1: with equal own blocks and sizes the hashes are
                    // equal iff the sums of the pair values are (sig_hash is a
                    // bijection of the sum), and a one-value sum is the pair
                    // value itself, a bijection of (label, block): equal full
                    // hashes are equal signatures
                    join = a.hash == c.hash;
                    push = !join;
                } else {
                    const int64_t ev = D.prp[pos], dv = D.prp[pos + 1] - ev;
                    const int64_t er = D.prp[rpos], dr = D.prp[rpos + 1] - er;
                    if (dv <= 2 && dr <= 2) {
                        // S_v inside S_r with equal sizes means equal sets
                        uint64_t b0 = 0, b1 = 0;
                        if (dr > 0) b0 = packed_pair_value(D.pe[er], D.P);
                        if (dr > 1) b1 = packed_pair_value(D.pe[er + 1], D.P);
                        bool ok = true;
                        for (int64_t j = 0; j < dv; ++j) {
                            const uint64_t x = packed_pair_value(D.pe[ev + j], D.P);
                            ok = ok && ((dr > 0 && x == b0) || (dr > 1 && x == b1));
                        }
                        join = ok;
                        push = !ok;
                    } else if (dv <= 32 && dr <= 32) {
                        small = true;
                    } else {
                        big = true;
                    }
                }
                if (join) {
                    O.Pout[v] = r;
                    D.joined[rpos] = 1;
                }
            }
        }
        const unsigned bo = __ballot_sync(0xffffffffu, own), bp = __ballot_sync(0xffffffffu, push);
        const unsigned bs = __ballot_sync(0xffffffffu, small), bb = __ballot_sync(0xffffffffu, big);
        unsigned (*c)[W + 1] = sh[par];
        if (lane_id() == 0) {
            c[0][warp] = static_cast<unsigned>(__popc(bo));
            c[1][warp] = static_cast<unsigned>(__popc(bp));
            c[2][warp] = static_cast<unsigned>(__popc(bs));
            c[3][warp] = static_cast<unsigned>(__popc(bb));
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            const int q = static_cast<int>(threadIdx.x);
            unsigned tot = 0;
            for (int w2 = 0; w2 < W; ++w2) {
                const unsigned x = c[q][w2];
                c[q][w2] = tot;
                tot += x;
            }
            unsigned at = 0;
            if (tot) {
                if (q == 0) atomicAdd(&O.st->blocks, static_cast<unsigned long long>(tot));
                else at = atomicAdd(q == 1 ? &O.st->unresolved : q == 2 ? &O.st->pairs : &O.st->deferred, tot);
            }
            c[q][W] = at;
        }
        __syncthreads();
        if (push) O.next[c[1][W] + c[1][warp] + __popc(bp & lt)] = pos;
        if (small) O.small[c[2][W] + c[2][warp] + __popc(bs & lt)] = make_int2(pos, rpos);
        if (big) O.pairs[c[3][W] + c[3][warp] + __popc(bb & lt)] = make_int2(pos, rpos);
    }
}

// ----------------------------------------------------------------------------- active list

// End of a round (after its collision levels): every listed vertex's
// P_{i+1} goes into the input buffer (the two buffers already agree on every
// vertex that is not listed), and the list keeps the positions that are still
// not alone in their block, in order. Tiles of kActTile entries, four
// consecutive entries per thread (eight left most CTAs idle once the list is
// short: 2.725 against 2.679 ms for the five rounds of the 10M-vertex graph);
// `stop` (the captured loop's decision, null for host-driven rounds) skips all
// of it when the host must first resolve the round's hash collisions.
constexpr int kActPer = 4;
constexpr int kActTile = kThreads * kActPer;

struct ClassBounds {
    int64_t b[kDClasses + 1];
};

// First packed edge of every class: prp at the classes' first positions.
__global__ void k_class_edge_begin(const int64_t* __restrict__ prp, const ClassBounds cb, int64_t* __restrict__ out) {
    const int c = static_cast<int>(threadIdx.x);
    if (c <= kDClasses) out[c] = prp[cb.b[c]];
}

__device__ __forceinline__ bool stays_listed(const DenseView& D, int64_t pos) {
    return !alone_last_round(D, pos);
}

// Pass 1: copy P_{i+1} back for the listed vertices, count each tile's
// survivors and each class's. When every live position is listed (round 1)
// the whole array is copied in order instead of vertex by vertex.
__global__ void __launch_bounds__(kThreads) k_active_count(const DenseView D, const int32_t* __restrict__ Pout,
                                                           int32_t* __restrict__ Pin, int64_t n, int64_t n_live,
                                                           int64_t* __restrict__ tcount,
                                                           unsigned long long* __restrict__ ccount,
                                                           const ClassBounds cb, const int32_t* stop) {
    __shared__ unsigned wsum[kThreads / 32];
    __shared__ unsigned csum[kDClasses];
    if (stop != nullptr && *stop >= 2) return;
    const int64_t count = D.aoff[kDClasses];
    const bool full = count == n_live;
    if (full) {
        const int64_t st = static_cast<int64_t>(gridDim.x) * blockDim.x;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += st) Pin[i] = Pout[i];
    }
    if (threadIdx.x < kDClasses) csum[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t tiles = (count + kActTile - 1) / kActTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kActTile + static_cast<int64_t>(threadIdx.x) * kActPer;
        // every load of the thread's entries is issued before the first store
        // (the copy's stores would otherwise order the next entry's loads)
        int32_t pos[kActPer], v[kActPer], pv[kActPer];
        bool stay[kActPer];
#pragma unroll
        for (int k = 0; k < kActPer; ++k) pos[k] = e0 + k < count ? D.act[e0 + k] : -1;
#pragma unroll
        for (int k = 0; k < kActPer; ++k) {
            stay[k] = pos[k] >= 0 && stays_listed(D, pos[k]);
            v[k] = pos[k] >= 0 && !full ? D.vert[pos[k]] : -1;
        }
#pragma unroll
        for (int k = 0; k < kActPer; ++k) pv[k] = v[k] >= 0 ? Pout[v[k]] : 0;
        unsigned keep = 0;
        int c = 0;
#pragma unroll
        for (int k = 0; k < kActPer; ++k) {
            if (v[k] >= 0) Pin[v[k]] = pv[k];
            if (stay[k]) {
                ++keep;
                while (c + 1 < kDClasses && pos[k] >= cb.b[c + 1]) ++c;      // entries ascend: c only grows
                atomicAdd(&csum[c], 1u);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
        if (lane_id() == 0) wsum[threadIdx.x >> 5] = keep;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) tot += wsum[w];
            tcount[t] = tot;
        }
        __syncthreads();
    }
    if (threadIdx.x < kDClasses && csum[threadIdx.x])
        atomicAdd(&ccount[threadIdx.x], static_cast<unsigned long long>(csum[threadIdx.x]));
}

// Pass 2 (one CTA): exclusive scan of the tile counts; the new length goes to tcount[slot_total].
__global__ void __launch_bounds__(1024) k_active_scan(const int64_t* __restrict__ aoff, int64_t* __restrict__ tcount,
                                                      int64_t slot_total, const int32_t* stop) {
    if (stop != nullptr && *stop >= 2) return;
    const int64_t tiles = (aoff[kDClasses] + kActTile - 1) / kActTile;
    const int64_t total = cta_exclusive_scan(tcount, tcount, tiles);
    if (threadIdx.x == 0) tcount[slot_total] = total;
}

// Pass 3: every tile writes its survivors at its offset into the next list.
__global__ void __launch_bounds__(kThreads) k_active_scatter(const DenseView D, const int64_t* __restrict__ toff,
                                                             int32_t* __restrict__ next, const int32_t* stop) {
    __shared__ unsigned wpre[kThreads / 32];
    if (stop != nullptr && *stop >= 2) return;
    const int64_t count = D.aoff[kDClasses];
    const int64_t tiles = (count + kActTile - 1) / kActTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kActTile + static_cast<int64_t>(threadIdx.x) * kActPer;
        int32_t p[kActPer];
        unsigned keepm = 0;
#pragma unroll
        for (int k = 0; k < kActPer; ++k) {
            p[k] = e0 + k < count ? D.act[e0 + k] : -1;
            if (p[k] >= 0 && stays_listed(D, p[k])) keepm |= 1u << k;
        }
        const unsigned mine = static_cast<unsigned>(__popc(keepm));
        unsigned inc = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane_id() >= static_cast<unsigned>(o)) inc += y;
        }
        if (lane_id() == 31) wpre[threadIdx.x >> 5] = inc;
        __syncthreads();
        unsigned wbase = 0;
        for (int w = 0; w < static_cast<int>(threadIdx.x >> 5); ++w) wbase += wpre[w];
        int64_t at = toff[t] + wbase + inc - mine;
#pragma unroll
        for (int k = 0; k < kActPer; ++k)
            if (keepm & (1u << k)) next[at++] = p[k];
        __syncthreads();
    }
}

// Pass 4: the next list replaces the current one; its class offsets from the
// classes' survivor counts (which are cleared for the next round).
__global__ void __launch_bounds__(kThreads) k_active_finish(const int32_t* __restrict__ next, int32_t* __restrict__ act,
                                                            int64_t* __restrict__ aoff, const int64_t* __restrict__ total,
                                                            unsigned long long* __restrict__ ccount, const int32_t* stop) {
    if (stop != nullptr && *stop >= 2) return;
    const int64_t len = *total;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t run = 0;
        for (int c = 0; c < kDClasses; ++c) {
            aoff[c] = run;
            run += static_cast<int64_t>(ccount[c]);
            ccount[c] = 0ull;
        }
        aoff[kDClasses] = len;
    }
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < len; i += stride) act[i] = next[i];
}

// Batched contexts: the positions of the graphs left out are marked alone in
// their block (the next compaction drops them from the list, and no round
// kernel touches them); DevState.blocks counts them and DevState.aux those
// that are their own P_0 block id (P_0's blocks among them).
__global__ void k_keep_graphs(const int32_t* __restrict__ vert, const int32_t* __restrict__ gid,
                              const uint8_t* __restrict__ keep, const int32_t* __restrict__ P0, int64_t n_live,
                              uint8_t* __restrict__ own, uint8_t* __restrict__ joined, DevState* st) {
    unsigned long long dropped = 0, blocks0 = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_live; p += stride) {
        const int32_t v = vert[p];
        if (keep[gid[v]]) continue;
        own[p] = 1;
        joined[p] = 0;
        ++dropped;
        if (P0[v] == v) ++blocks0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dropped += __shfl_xor_sync(0xffffffffu, dropped, o);
        blocks0 += __shfl_xor_sync(0xffffffffu, blocks0, o);
    }
    if (lane_id() == 0 && dropped) {
        atomicAdd(&st->blocks, dropped);
        atomicAdd(&st->aux, blocks0);
    }
}

// Start of a run of rounds: every live position is listed.
__global__ void k_active_init(int32_t* __restrict__ act, int64_t n_live, int64_t* __restrict__ aoff,
                              unsigned long long* __restrict__ ccount, const ClassBounds cb) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t0 <= kDClasses) aoff[t0] = cb.b[t0];
    if (t0 < kDClasses) ccount[t0] = 0ull;
    for (int64_t i = t0; i < n_live; i += stride) act[i] = static_cast<int32_t>(i);
}

constexpr int kCompareGrid = 304;                      // persistent grids: two CTAs per SM
constexpr int kCompareWarpGrid = 1216;                 // eight per SM: a warp per pair, all warps in flight

// Pairs whose rows have at most 32 edges: one warp per pair. Lane j holds the
// j-th pair value of each row; S_v is inside S_r iff every value of v's row
// matches one of r's. The pair count is read on the device.
__global__ void __launch_bounds__(kThreads) k_dense_compare_warp(const int2* __restrict__ pairs, const DenseView D,
                                                                 int32_t* __restrict__ Pout,
                                                                 int32_t* __restrict__ next, DevState* st) {
    const unsigned count = *reinterpret_cast<volatile unsigned*>(&st->pairs);
    const unsigned lane = lane_id();
    const unsigned warps = gridDim.x * (kThreads / 32);
    for (unsigned i = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); i < count; i += warps) {
        const int2 pr = pairs[i];
        const int64_t ev = D.prp[pr.x], dv = D.prp[pr.x + 1] - ev;
        const int64_t er = D.prp[pr.y], dr = D.prp[pr.y + 1] - er;
        const bool ha = lane < dv, hb = lane < dr;
        const uint64_t a = ha ? packed_pair_value(D.pe[ev + lane], D.P) : 0ull;
        const uint64_t b = hb ? packed_pair_value(D.pe[er + lane], D.P) : 0ull;
        if (lane == 0) atomicAdd(&st->aux, static_cast<unsigned long long>(dv + dr));
        bool found = false;
        for (int k = 0; k < static_cast<int>(dr); ++k) {
            const uint64_t bk = __shfl_sync(0xffffffffu, b, k);   // every lane takes part in every shuffle
            found = found || bk == a;
        }
        const bool miss = __any_sync(0xffffffffu, ha && !found);
        if (lane == 0) {
            if (!miss) {
                Pout[D.vert[pr.x]] = D.vert[pr.y];
                D.joined[pr.y] = 1;
            }
            else next[atomicAdd(&st->unresolved, 1u)] = pr.x;
        }
    }
}

constexpr int kCompareSlots = 2 * kMidMaxN;          // shared-memory set of 16384 slots
constexpr int kCompareLimit = 3 * kMidMaxN / 2;       // distinct values one pass may hold
constexpr size_t kCompareSmem = sizeof(unsigned long long) * kCompareSlots;

// Longer rows: one CTA per pair; S_v == S_r iff every value of v's row is in
// S_r (the sizes are equal).
__global__ void __launch_bounds__(kThreads) k_dense_compare_cta(const int2* __restrict__ pairs, const DenseView D,
                                                                const HubSets H, int32_t* __restrict__ Pout,
                                                                int32_t* __restrict__ next, DevState* st) {
    extern __shared__ unsigned long long tab[];
    __shared__ unsigned zero, used, over;
    volatile unsigned* overv = &over;
    const unsigned count = *reinterpret_cast<volatile unsigned*>(&st->deferred);
    for (unsigned i = blockIdx.x; i < count; i += gridDim.x) {
        const int2 pr = pairs[i];
        const int32_t c = D.sig[pr.y].cnt;
        const int64_t ev = D.prp[pr.x], dv = D.prp[pr.x + 1] - ev;
        const int64_t er = D.prp[pr.y], dr = D.prp[pr.y + 1] - er;
        bool miss = false;
        // S_r is rebuilt in shared memory, in sub-ranges of the value mix when
        // it is too large for one set (a hub): each pass takes the values of
        // both rows in one sub-range; more sub-ranges when a pass overflows
        uint32_t splits = 1;
        while (splits * static_cast<uint32_t>(kCompareLimit) < static_cast<uint32_t>(c)) splits <<= 1;
        bool done = false;
        for (; splits <= static_cast<uint32_t>(kHubMaxSplits) && !done && !miss; splits <<= 1) {
            bool o = false;
            for (uint32_t sub = 0; sub < splits && !o && !miss; ++sub) {
                for (int j = threadIdx.x; j < kCompareSlots; j += kThreads) tab[j] = 0ull;
                if (threadIdx.x == 0) {
                    zero = 0u;
                    used = 0u;
                    over = 0u;
                }
                __syncthreads();
                for (int64_t j = threadIdx.x; j < dr; j += kThreads) {
                    if (*overv) break;
                    const uint64_t mv = packed_pair_value(D.pe[er + j], D.P);
                    if (split_of(bucket_mix(mv), 0, splits) != sub) continue;
                    if (smem_set_insert(tab, kCompareSlots - 1, &zero, mv) && mv != 0ull &&
                        atomicAdd(&used, 1u) + 1u > static_cast<unsigned>(kCompareLimit))
                        *overv = 1u;
                }
                __syncthreads();
                o = *overv != 0u;
                bool my_miss = false;
                if (!o) {
                    for (int64_t j = threadIdx.x; j < dv && !my_miss; j += kThreads) {
                        const uint64_t mv = packed_pair_value(D.pe[ev + j], D.P);
                        if (split_of(bucket_mix(mv), 0, splits) != sub) continue;
                        my_miss = !smem_set_contains(tab, kCompareSlots - 1, zero, mv);
                    }
                }
                miss = __syncthreads_or(my_miss ? 1 : 0) != 0;
            }
            done = !o;
        }
        if (!done && !miss) {            // no split fits: report instead of guessing
            if (threadIdx.x == 0) atomicOr(&st->error, kErrHubFull);
            miss = true;
        }
        const int any = __syncthreads_or(miss ? 1 : 0);
        if (threadIdx.x == 0) {
            atomicAdd(&st->aux, static_cast<unsigned long long>((dv + dr) * static_cast<int64_t>(splits > 1 ? splits / 2 : 1)));
            if (!any) {
                Pout[D.vert[pr.x]] = D.vert[pr.y];
                D.joined[pr.y] = 1;
            }
            else next[atomicAdd(&st->unresolved, 1u)] = pr.x;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- device-side round loop

// State of the round loop run by the captured graph (device memory).
struct LoopState {
    unsigned long long prev_blocks;   // block count of the partition the next round refines
    unsigned long long blocks;        // block count after the last round
    int32_t executed;                 // rounds run
    int32_t limit;                    // rounds allowed
    int32_t fixpoint;                 // 1: stop as soon as a round keeps the block count
    int32_t rounds;                   // the result r (k, or the fixpoint round)
    int32_t stop;                     // 0 go on, 1 done, 2 a hash collision to resolve on the host, 3 error
    int32_t pad;
};

// After a round: decide whether the loop goes on (the while condition of the graph).
__global__ void k_round_check(const DevState* __restrict__ st, LoopState* L, cudaGraphConditionalHandle cond) {
    const unsigned long long blocks = st->blocks;
    const int32_t executed = L->executed + 1;
    int32_t stop = 0;
    if (st->error != 0u) {
        stop = 3;
    } else if (st->unresolved != 0u) {
        stop = 2;                     // the host finishes this round's collision levels
    } else if (blocks == L->prev_blocks) {
        stop = 1;                     // P_{i+1} refines P_i with as many blocks: the fixpoint
        L->rounds = L->fixpoint ? executed - 1 : L->limit;
    } else if (executed >= L->limit) {
        stop = 1;
        L->rounds = L->limit;
    }
    if (stop < 2) L->prev_blocks = blocks;
    L->blocks = blocks;
    L->executed = executed;
    L->stop = stop;
    cudaGraphSetConditional(cond, stop == 0 ? 1u : 0u);
}

// Start of a captured round: the table is blanked when the epoch of this
// round (rounds run % 15, plus one) starts a new cycle, so a slot written by
// any earlier round of the cycle carries another epoch and counts as free.
__global__ void __launch_bounds__(kThreads) k_table_clear_round(const LoopState* __restrict__ L, Slot* slots,
                                                                uint64_t nslots) {
    if (L->executed % static_cast<int32_t>(kEpochCycle) != 0) return;
    uint4* w = reinterpret_cast<uint4*>(slots);          // two slots per 16-byte store
    const uint64_t words = nslots / 2;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < words; i += stride)
        w[i] = make_uint4(0u, 0u, 0u, 0u);
}

// ----------------------------------------------------------------------------- host helpers

HubSets hub_sets(const bisim_ctx* ctx) {
    return HubSets{ctx->dbegin[kDHub], ctx->n_dhub, ctx->htab, ctx->dedge_begin[kDHub], ctx->dacc};
}

template <class K>
void allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

// Algorithmic bytes: the signature kernels move per edge the packed (label,
// target) word 8 + the gathered P_i[w] 4, per vertex the list entry 4, the row
// offset 8, the vertex id 4, P_i[v] 4 and the 16-byte signature record written
// (minus the 4-byte list entry: 32); the insert moves per vertex the hash 8,
// the vertex id 4, one 8-byte table slot and the 4-byte slot index; the
// verification the slot index 4, the vertex id 4, one table slot 8 and
// P_{i+1}[v] 4.
constexpr double kEdgeBytes = 12.0;
constexpr double kSigVertexBytes = 32.0;
constexpr double kInsertVertexBytes = 24.0;
constexpr double kVerifyVertexBytes = 20.0;

// Persistent grids: as many CTAs as stay resident on all SMs at once (from the
// occupancy calculator, per kernel and dynamic shared memory size), so that no
// CTA waits for a second wave. Looked up before any capture (set_attributes)
// and cached.
unsigned resident_grid(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void*, size_t>, unsigned>> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto& c : cache)
        if (c.first.first == kernel && c.first.second == smem) return c.second;
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const unsigned g = static_cast<unsigned>(std::max(1, sms) * per_sm);
    cache.push_back({{kernel, smem}, g});
    return g;
}

template <class K>
unsigned persistent_grid(K kernel, int threads, size_t smem, int64_t ctas_needed) {
    const unsigned g = resident_grid(reinterpret_cast<const void*>(kernel), threads, smem);
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(g, ctas_needed)));
}

// The grids of the list-driven kernels are sized for the whole class (the
// list of round 1) and capped at the resident grid; each kernel reads its
// class's current entries on the device and strides over them.
template <int N, int T>
void launch_mid(bisim_ctx* ctx, int cls, const DenseView& D, cudaStream_t s, int site) {
    const int64_t count = ctx->dbegin[cls + 1] - ctx->dbegin[cls];
    if (count <= 0) return;
    const size_t smem = sizeof(unsigned long long) * 2 * N;
    Launch L(site, s, 0, 0, 0.0);                          // work and bytes: from the round's work counters
    const unsigned grid = persistent_grid(k_dense_mid_sig<N, T>, T, smem, count);
    k_dense_mid_sig<N, T><<<grid, T, smem, s>>>(cls, D, 4 + (cls - kDMid0));
}

// Kernel attributes (shared memory above 48 KB), set once before any launch or capture.
void set_attributes() {
    static std::once_flag once;
    std::call_once(once, []() {
        allow_smem(k_dense_mid_sig<512, 256>, sizeof(unsigned long long) * 2 * 512);
        allow_smem(k_dense_mid_sig<1024, 256>, sizeof(unsigned long long) * 2 * 1024);
        allow_smem(k_dense_mid_sig<2048, 512>, sizeof(unsigned long long) * 2 * 2048);
        allow_smem(k_dense_mid_sig<4096, 512>, sizeof(unsigned long long) * 2 * 4096);
        allow_smem(k_dense_mid_sig<8192, 512>, sizeof(unsigned long long) * 2 * 8192);
        allow_smem(k_dense_compare_cta, kCompareSmem);
        persistent_grid(k_hub_clear, kThreads, 0, 1);
        persistent_grid(k_hub_insert, kThreads, kHubInsertSmem, 1);
        persistent_grid(k_dense_thread_sig<8>, kThreads, 0, 1);
        persistent_grid(k_dense_thread_sig<16>, kThreads, 0, 1);
        persistent_grid(k_dense_thread_sig<32>, kThreads, 0, 1);
        persistent_grid(k_dense_warp_sig, kThreads, 0, 1);
        persistent_grid(k_dense_mid_sig<512, 256>, 256, sizeof(unsigned long long) * 2 * 512, 1);
        persistent_grid(k_dense_mid_sig<1024, 256>, 256, sizeof(unsigned long long) * 2 * 1024, 1);
        persistent_grid(k_dense_mid_sig<2048, 512>, 512, sizeof(unsigned long long) * 2 * 2048, 1);
        persistent_grid(k_dense_mid_sig<4096, 512>, 512, sizeof(unsigned long long) * 2 * 4096, 1);
        persistent_grid(k_dense_mid_sig<8192, 512>, 512, sizeof(unsigned long long) * 2 * 8192, 1);
        persistent_grid(k_dense_insert, kThreads, 0, 1);
        persistent_grid(k_dense_verify, kThreads, 0, 1);
        persistent_grid(k_active_count, kThreads, 0, 1);
        persistent_grid(k_active_finish, kThreads, 0, 1);
        persistent_grid(k_table_clear_round, kThreads, 0, 1);
    });
}

// The table the rounds insert into: the global one, or the per-graph regions of a batched context.
Slot* round_slots(const bisim_ctx* ctx) { return ctx->rtable ? ctx->rtable : ctx->table; }

// A fresh level of the renumbering: a new epoch of the global table, or a
// cleared region table (epoch 1) for batched contexts.
TableRef level_table(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->rtable == nullptr) return next_epoch(ctx, s);
    cudaMemsetAsync(ctx->rtable, 0, sizeof(Slot) * ctx->n_rslots, s);
    TableRef t;
    t.slots = ctx->rtable;
    t.mask = ctx->n_rslots - 1;     // not used by region inserts
    t.epoch = uint64_t{1} << 32;
    const int hb = ctx->opt.hash_bits;
    t.hmask = hb >= 64 ? ~0ull : ((1ull << hb) - 1ull);
    return t;
}

// Insert, verification and set comparisons of one level (level 0: the active
// list, whose length is read on the device; then the listed unresolved
// positions). Unresolved positions go to `next`.
void launch_level(bisim_ctx* ctx, cudaStream_t s, const DenseView& D, const TableRef& t, uint32_t level,
                  const int32_t* list, int64_t count, int32_t* next) {
    BISIM_SITE(site_in, "dense_insert");
    BISIM_SITE(site_v, "dense_verify");
    BISIM_SITE(site_cw, "dense_compare_warp");
    BISIM_SITE(site_cc, "dense_compare_cta");
    if (count <= 0) return;
    int32_t* Pout = ctx->P[1];
    const VerifyOut O{Pout, ctx->dpairs, ctx->dsmall, next, ctx->dstate};
    const HubSets H = hub_sets(ctx);
    if (level == 0) {
        // `count` bounds the grid; the kernels read the list's length, and
        // their bytes follow it (added after the round)
        const unsigned* dcount = &ctx->dstate->listed;
        {
            Launch L(site_in, s, 0, 0, 0.0);
            k_dense_insert<<<persistent_grid(k_dense_insert, kThreads, 0, cdiv(count, kThreads)), kThreads, 0, s>>>(
                ctx->dact, 0, dcount, D, 0, t, &ctx->dstate->error);
        }
        Launch L(site_v, s, 0, 0, 0.0);
        k_dense_verify<<<persistent_grid(k_dense_verify, kThreads, 0, cdiv(count, kThreads)), kThreads, 0, s>>>(
            ctx->dact, 0, dcount, D, round_slots(ctx), O, ctx->n);
    } else {
        {
            Launch L(site_in, s, count, 0, kInsertVertexBytes * count);
            k_dense_insert<<<grid_for(count, kThreads), kThreads, 0, s>>>(list, count, nullptr, D, level, t,
                                                                         &ctx->dstate->error);
        }
        Launch L(site_v, s, count, 0, kVerifyVertexBytes * count);
        k_dense_verify<<<grid_for(count, kThreads), kThreads, 0, s>>>(list, count, nullptr, D, round_slots(ctx), O,
                                                                     ctx->n);
    }
    {
        Launch L(site_cw, s, 0, 0, 0.0);
        k_dense_compare_warp<<<kCompareWarpGrid, kThreads, 0, s>>>(ctx->dsmall, D, Pout, next, ctx->dstate);
    }
    Launch L(site_cc, s, 0, 0, 0.0);
    k_dense_compare_cta<<<kCompareGrid, kThreads, kCompareSmem, s>>>(ctx->dpairs, D, H, Pout, next, ctx->dstate);
}

// Survivor counts per class at the end of a round: the words after the tile
// counts and the list's new length in dtile.
unsigned long long* class_counts(const bisim_ctx* ctx) {
    return reinterpret_cast<unsigned long long*>(ctx->dtile + ctx->n_tiles + 2);
}

ClassBounds class_bounds(const bisim_ctx* ctx) {
    ClassBounds cb;
    for (int c = 0; c <= kDClasses; ++c) cb.b[c] = ctx->dbegin[c];
    return cb;
}

// End of a round: P_{i+1} of the listed vertices into the input buffer and the
// list compacted to the vertices still not alone (see k_active_count). `stop`
// is the captured loop's decision, or null for host-driven rounds.
void launch_round_end(bisim_ctx* ctx, cudaStream_t s, const DenseView& D, const int32_t* stop,
                      const int32_t* Pfrom = nullptr) {
    BISIM_SITE(site, "active_compact");
    const int64_t n_live = ctx->dbegin[kDClasses];
    if (n_live <= 0) return;
    const unsigned grid = persistent_grid(k_active_count, kThreads, 0, cdiv(n_live, kActTile));
    const int64_t slot_total = ctx->n_tiles;
    // bytes: per listed entry the list 4 + vertex 4 + P read 4 + P written 4 + two flags,
    // then the list and flags again, and 8 per survivor (written, copied)
    Launch L(site, s, 0, 0, 0.0);
    unsigned long long* ccount = class_counts(ctx);
    k_active_count<<<grid, kThreads, 0, s>>>(D, Pfrom ? Pfrom : ctx->P[1], ctx->P[0], ctx->n, n_live, ctx->dtile, ccount,
                                             class_bounds(ctx), stop);
    k_active_scan<<<1, 1024, 0, s>>>(ctx->daoff, ctx->dtile, slot_total, stop);
    k_active_scatter<<<grid, kThreads, 0, s>>>(D, ctx->dtile, ctx->dact2, stop);
    k_active_finish<<<persistent_grid(k_active_finish, kThreads, 0, cdiv(n_live, kThreads)), kThreads, 0, s>>>(
        ctx->dact2, ctx->dact, ctx->daoff, ctx->dtile + slot_total, ccount, stop);
}

DenseView dense_view(bisim_ctx* ctx) {
    const bool regions = ctx->rtable != nullptr;
    return DenseView{ctx->dvert, ctx->dvpos, ctx->dprp, ctx->dpe, ctx->P[0], ctx->dsig, ctx->dslot,
                     ctx->djoined, ctx->downs, regions ? ctx->gid : nullptr, ctx->rbase, ctx->rmask,
                     prof_enabled() ? ctx->dwork : nullptr, ctx->dact, ctx->daoff, nullptr};
}


// Everything of one round P[0] -> P[1] that needs no host decision:
// signatures of the listed vertices of every class, then level 0 of the
// renumbering. P[1] already holds P_i (the end of the previous round copied
// it back, and in round 1 every vertex is listed), so vertices alone in
// their block need no write.
void launch_round(bisim_ctx* ctx, cudaStream_t s, const TableRef& t, const int32_t* round_no = nullptr) {
    DenseView D = dense_view(ctx);
    D.round_no = round_no;
    const HubSets H = hub_sets(ctx);
    unsigned* err = &ctx->dstate->error;
    BISIM_SITE(site_rb, "round_begin");
    {
        Launch L(site_rb, s, 0, 0, 0.0);
        k_round_begin<<<1, 1, 0, s>>>(ctx->dstate, ctx->daoff, ctx->dbegin[kDClasses]);
    }
    if (ctx->n_dhub > 0) {
        cudaMemsetAsync(ctx->dacc, 0, sizeof(HubAcc) * ctx->n_dhub, s);
    }
    const int64_t* db = ctx->dbegin;
    BISIM_SITE(site_t8, "dense_thread_sig_8");
    BISIM_SITE(site_t16, "dense_thread_sig_16");
    BISIM_SITE(site_t32, "dense_thread_sig_32");
    BISIM_SITE(site_w, "dense_warp_sig");
    static const int site_mid[5] = {prof_site("dense_mid_512"), prof_site("dense_mid_1024"),
                                    prof_site("dense_mid_2048"), prof_site("dense_mid_4096"),
                                    prof_site("dense_mid_8192")};
    BISIM_SITE(site_hc, "hub_clear");
    BISIM_SITE(site_hi, "hub_insert");
    BISIM_SITE(site_hf, "dense_hub_finalize");
    // classes 0..4 (degree <= 8), 5 (<= 16) and 6 (<= 32): one thread per vertex
    if (D.work) cudaMemsetAsync(D.work, 0, sizeof(unsigned long long) * kWorkWords, s);
    // the signature kernels' bytes are added after the round from the work counters
    auto thread_sig = [&](int c0, int c1, auto kernel, int site, int group) {
        const int64_t verts = db[c1] - db[c0];
        if (verts <= 0) return;
        Launch L(site, s, 0, 0, 0.0);
        kernel<<<persistent_grid(kernel, kThreads, 0, cdiv(verts, kThreads)), kThreads, 0, s>>>(c0, c1, D, group);
    };
    thread_sig(0, 5, k_dense_thread_sig<8>, site_t8, 0);
    thread_sig(5, 6, k_dense_thread_sig<16>, site_t16, 1);
    thread_sig(6, 7, k_dense_thread_sig<32>, site_t32, 2);
    if (db[kDMid0] > db[kDWarp0]) {
        const int64_t verts = db[kDMid0] - db[kDWarp0];
        Launch L(site_w, s, 0, 0, 0.0);
        k_dense_warp_sig<<<persistent_grid(k_dense_warp_sig, kThreads, 0, cdiv(verts, kThreads / 32)), kThreads, 0, s>>>(D);
    }
    launch_mid<512, 256>(ctx, kDMid0 + 0, D, s, site_mid[0]);
    launch_mid<1024, 256>(ctx, kDMid0 + 1, D, s, site_mid[1]);
    launch_mid<2048, 512>(ctx, kDMid0 + 2, D, s, site_mid[2]);
    launch_mid<4096, 512>(ctx, kDMid0 + 3, D, s, site_mid[3]);
    launch_mid<8192, 512>(ctx, kDMid0 + 4, D, s, site_mid[4]);
    if (ctx->n_dhub > 0) {
        if (ctx->n_dchunks > 0) {
            {
                Launch L(site_hc, s, 0, 0, 0.0);
                k_hub_clear<<<persistent_grid(k_hub_clear, kThreads, 0, ctx->n_dchunks), kThreads, 0, s>>>(
                    ctx->dchunks, ctx->n_dchunks, D, H);
            }
            Launch L(site_hi, s, 0, 0, 0.0);
            k_hub_insert<<<persistent_grid(k_hub_insert, kThreads, kHubInsertSmem, ctx->n_dchunks), kThreads,
                           kHubInsertSmem, s>>>(ctx->dchunks, ctx->n_dchunks, D, H, err);
        }
        Launch L(site_hf, s, 0, 0, 0.0);
        k_dense_hub_finalize<<<grid_for(ctx->n_dhub, 128), 128, 0, s>>>(D, H);
    }
    launch_level(ctx, s, D, t, 0, nullptr, ctx->dbegin[kDClasses], ctx->ulist[0]);
}

// Reads the state of a round whose level 0 has been launched, runs the
// collision levels that are needed, and moves the current partition on.
// Launch profiling: the signature kernels' algorithmic bytes from the rows and
// row entries they processed this round (vertices alone in their block are
// skipped), the level-0 table passes' from the positions listed for them.
void add_round_work(bisim_ctx* ctx, double listed) {
    unsigned long long w[kWorkWords];
    if (cudaMemcpy(w, ctx->dwork, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return;
    double rows[kWorkGroups] = {}, edges[kWorkGroups] = {};
    for (int g = 0; g < kWorkGroups; ++g)
        for (int k = 0; k < kWorkSpread; ++k) {
            rows[g] += static_cast<double>(w[(g * 2) * kWorkSpread + k]);
            edges[g] += static_cast<double>(w[(g * 2 + 1) * kWorkSpread + k]);
        }
    static const int sites[9] = {prof_site("dense_thread_sig_8"), prof_site("dense_thread_sig_16"),
                                 prof_site("dense_thread_sig_32"), prof_site("dense_warp_sig"),
                                 prof_site("dense_mid_512"), prof_site("dense_mid_1024"), prof_site("dense_mid_2048"),
                                 prof_site("dense_mid_4096"), prof_site("dense_mid_8192")};
    for (int g = 0; g < 9; ++g) {
        prof_add_bytes(sites[g], kSigVertexBytes * rows[g] + kEdgeBytes * edges[g]);
        prof_add_work(sites[g], static_cast<int64_t>(rows[g]), static_cast<int64_t>(edges[g]));
    }
    BISIM_SITE(site_hi, "hub_insert");
    BISIM_SITE(site_hf, "dense_hub_finalize");
    // the hub rows' algorithmic bytes are those of reading them; clearing the
    // tables is overhead of this design (no bytes)
    const double he = edges[kWorkHub];
    prof_add_bytes(site_hi, kEdgeBytes * he);
    prof_add_bytes(site_hf, kSigVertexBytes * rows[kWorkHub]);
    prof_add_work(site_hi, 0, static_cast<int64_t>(he));
    prof_add_work(site_hf, static_cast<int64_t>(rows[kWorkHub]), 0);
    BISIM_SITE(site_in, "dense_insert");
    BISIM_SITE(site_v, "dense_verify");
    prof_add_bytes(site_in, kInsertVertexBytes * listed);
    prof_add_bytes(site_v, kVerifyVertexBytes * listed);
    prof_add_work(site_in, static_cast<int64_t>(listed), 0);
    prof_add_work(site_v, static_cast<int64_t>(listed), 0);
}

// Algorithmic bytes of the end of a round over `listed` entries with `kept` survivors:
// per entry the list 4, the vertex id 4, P_{i+1} read 4 and written back 4 and the
// two flags 2, read again by the scatter (list 4, flags 2); per survivor the
// position written 4, read and copied 8.
double round_end_bytes(double listed, double kept) { return 24.0 * listed + 12.0 * kept; }

bisim_status finish_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks) {
    cudaError_t e;
    const DenseView D = dense_view(ctx);
    int which = 0;                    // level 0 pushed its unresolved positions to ulist[0]
    for (uint32_t level = 1;; ++level) {
        cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, level > 1 ? "resolve hash collisions" : "dense round");
        if (ctx->hstate->error != 0 || ctx->hstate->unresolved == 0) break;
        if (level > static_cast<uint32_t>(kMaxLevels))
            return set_error(ctx, BISIM_ETIMEOUT, "hash collision resolution did not converge");
        const int64_t count = ctx->hstate->unresolved;
        TableRef t = level_table(ctx, s);
        cudaMemsetAsync(&ctx->dstate->unresolved, 0, sizeof(unsigned), s);
        cudaMemsetAsync(&ctx->dstate->deferred, 0, sizeof(unsigned), s);
        cudaMemsetAsync(&ctx->dstate->pairs, 0, sizeof(unsigned), s);
        launch_level(ctx, s, D, t, level, ctx->ulist[which], count, ctx->ulist[which ^ 1]);
        which ^= 1;
        ctx->stats.collision_levels += 1;
    }
    if (prof_enabled()) {
        // the exact comparisons' work is known only now: 12 bytes per row word read
        // (packed word + gathered block id) plus two row offsets per pair
        BISIM_SITE(site_cmp, "dense_compare_warp");
        const double pairs = static_cast<double>(ctx->hstate->pairs) + static_cast<double>(ctx->hstate->deferred);
        prof_add_bytes(site_cmp, 12.0 * static_cast<double>(ctx->hstate->aux) + 32.0 * pairs);
        add_round_work(ctx, static_cast<double>(ctx->hstate->listed));
    }
    if (ctx->hstate->error & kErrTableFull) return set_error(ctx, BISIM_ETIMEOUT, "signature table probe limit reached");
    if (ctx->hstate->error & kErrHubFull) return set_error(ctx, BISIM_ETIMEOUT, "hub set probe limit reached");
    if (ctx->hstate->error) return set_error(ctx, BISIM_EINVAL, "device reported invalid input");
    *out_blocks = static_cast<int64_t>(ctx->hstate->blocks);
    launch_round_end(ctx, s, D, nullptr);
    if (prof_enabled() && ctx->dbegin[kDClasses] > 0) {
        int64_t kept = 0;
        cudaMemcpyAsync(&kept, ctx->dtile + ctx->n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "compact the active list");
        BISIM_SITE(site_ac, "active_compact");
        prof_add_bytes(site_ac, round_end_bytes(static_cast<double>(ctx->hstate->listed), static_cast<double>(kept)));
    }
    return BISIM_OK;
}

}  // namespace

namespace {

bisim_status alloc_round_state(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->dvert != nullptr) return BISIM_OK;
    const size_t nv = static_cast<size_t>(std::max(ctx->n, 1));
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dvert), sizeof(int32_t) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dvpos), sizeof(int32_t) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dprp), sizeof(int64_t) * (nv + 1), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dslot), sizeof(uint32_t) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dsig), sizeof(SigRec) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dpairs), sizeof(int2) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dsmall), sizeof(int2) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dwork), sizeof(unsigned long long) * kWorkWords, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->djoined), nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->downs), nv, s)))
        return cuda_error(ctx, e, "alloc dense round state");
    ctx->n_tiles = cdiv(static_cast<int64_t>(nv), kActTile);
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dact), sizeof(int32_t) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dact2), sizeof(int32_t) * nv, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->daoff), sizeof(int64_t) * (kDClasses + 1), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dtile), sizeof(int64_t) * (ctx->n_tiles + 2 + kDClasses), s)))
        return cuda_error(ctx, e, "alloc active list");
    return BISIM_OK;
}

void free_hub_layout(bisim_ctx* ctx, cudaStream_t s) {
    ctx_free(ctx, ctx->dchunks, sizeof(HubChunk) * ctx->n_dchunks, s);
    ctx_free(ctx, ctx->htab, 2 * sizeof(unsigned long long) * ctx->hub_edges, s);
    ctx_free(ctx, ctx->dacc, sizeof(HubAcc) * ctx->n_dhub, s);
    ctx->dchunks = nullptr;
    ctx->htab = nullptr;
    ctx->dacc = nullptr;
    ctx->n_dchunks = ctx->n_dhub = ctx->hub_edges = 0;
}

// Copies the rows of the vertex-ordered CSR into the packed rows (all but hubs).
void pack_rows_from_csr(bisim_ctx* ctx, cudaStream_t s) {
    BISIM_SITE(site_p, "dense_pack");
    const int64_t* begin = ctx->dbegin;
    const int64_t small = begin[kDMid0];                 // rows of at most 256 edges: a warp per 32 rows
    const int64_t mid = begin[kDHub] - small;
    const int64_t edges = ctx->dedge_begin[kDHub];
    Launch L(site_p, s, begin[kDHub], edges, 16.0 * edges + 20.0 * begin[kDHub]);
    if (small > 0)
        k_dense_pack_rows<<<grid_for(small, 256), 256, 0, s>>>(ctx->dvert, small, ctx->dprp, ctx->row_ptr, ctx->col,
                                                              ctx->elab, ctx->dpe);
    if (mid > 0)
        k_dense_pack_big<<<static_cast<unsigned>(mid), 256, 0, s>>>(ctx->dvert, small, ctx->dprp, ctx->row_ptr,
                                                                   ctx->col, ctx->elab, ctx->dpe);
}

}  // namespace

bisim_status dense_layout_positions(bisim_ctx* ctx, const int32_t* deg, cudaStream_t s) {
    const int32_t n = ctx->n;
    const size_t nv = static_cast<size_t>(std::max(n, 1));
    cudaError_t e;
    bisim_status st;
    if ((st = alloc_round_state(ctx, s)) != BISIM_OK) return st;
    free_hub_layout(ctx, s);
    const size_t tmp_words = std::max(radix_temp_words(n), scan_temp_words(static_cast<int64_t>(n) + 1));
    // every piece starts on a 256-byte boundary: the allocation is the sum of the rounded sizes
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t bytes = 2 * r256(sizeof(uint32_t) * nv) + 2 * r256(sizeof(uint64_t) * nv) +
                         r256(sizeof(int64_t) * (nv + 1)) + r256(sizeof(int64_t) * tmp_words) +
                         r256(sizeof(int64_t) * (kDClasses + 1));
    char* scratch = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s))) return cuda_error(ctx, e, "alloc layout scratch");
    char* base = scratch;
    auto carve = [&](size_t b) { char* p = scratch; scratch += r256(b); return p; };
    uint32_t* k0 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * nv));
    uint32_t* k1 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * nv));
    uint64_t* v0 = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * nv));
    uint64_t* v1 = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * nv));
    int64_t* pdeg = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * (nv + 1)));
    int64_t* tmp = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * tmp_words));
    int64_t* dbeg = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * (kDClasses + 1)));
    int64_t begin[kDClasses + 1];
    for (int c = 0; c <= kDClasses; ++c) begin[c] = n;
    cudaMemcpyAsync(dbeg, begin, sizeof(begin), cudaMemcpyHostToDevice, s);
    BISIM_SITE(site_c, "dense_classify");
    if (n > 0) {
        {
            Launch L(site_c, s, n, 0, 12.0 * n);
            k_dense_classify<<<grid_for(n, 256), 256, 0, s>>>(deg, ctx->alive, n, ctx->opt.small_max_degree,
                                                             ctx->opt.mid_max_degree, k0, v0);
        }
        const int which = radix_sort_pairs(k0, v0, k1, v1, n, 5, tmp, s, "class_radix");
        const uint32_t* sk = which ? k1 : k0;
        const uint64_t* sv = which ? v1 : v0;
        {
            Launch L(site_c, s, n, 0, 8.0 * n);
            k_dense_bounds<<<grid_for(n, 256), 256, 0, s>>>(sk, n, dbeg);
        }
        Launch L(site_c, s, n, 0, 12.0 * n);
        k_dense_vertices<<<grid_for(n, 256), 256, 0, s>>>(sv, n, ctx->dvert, ctx->dvpos);
    }
    cudaMemcpyAsync(begin, dbeg, sizeof(begin), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(base, s);
        return cuda_error(ctx, e, "classify vertices");
    }
    for (int c = kDClasses - 1; c >= 0; --c) begin[c] = std::min(begin[c], begin[c + 1]);
    for (int c = 0; c <= kDClasses; ++c) ctx->dbegin[c] = begin[c];
    const int64_t n_live = begin[kDClasses];
    ctx->stats.n_small = begin[kDWarp0] - begin[0];
    ctx->stats.n_mid = begin[kDHub] - begin[kDWarp0];
    ctx->stats.n_hub = begin[kDHub + 1] - begin[kDHub];
    {
        Launch L(site_c, s, n_live, 0, 12.0 * n_live);
        k_dense_degrees<<<grid_for(n_live + 1, 256), 256, 0, s>>>(ctx->dvert, n_live, deg, pdeg);
    }
    exclusive_scan_i64(pdeg, ctx->dprp, n_live + 1, tmp, s);
    // the classes' first edges in one read-back (dbeg is free again)
    k_class_edge_begin<<<1, 32, 0, s>>>(ctx->dprp, class_bounds(ctx), dbeg);
    cudaMemcpyAsync(ctx->dedge_begin, dbeg, sizeof(int64_t) * (kDClasses + 1), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(base, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "row offsets");
    return BISIM_OK;
}

bisim_status dense_layout_hubs(bisim_ctx* ctx, bool pack_from_csr, cudaStream_t s) {
    cudaError_t e;
    const int64_t* begin = ctx->dbegin;
    const int64_t m = ctx->m;
    const int64_t nh = begin[kDHub + 1] - begin[kDHub];
    BISIM_SITE(site_p, "dense_pack");
    if (nh > 0) {
        // the chunks are laid out on the device from the rows' offsets (read
        // back only to size them): a host-to-device copy here would wait behind
        // any upload of another context in flight on the copy engine
        std::vector<int64_t> rows(nh + 1);
        cudaMemcpyAsync(rows.data(), ctx->dprp + begin[kDHub], sizeof(int64_t) * (nh + 1), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "read hub rows");
        const int64_t csz = std::max(256, ctx->opt.hub_chunk);
        int64_t n_chunks = 0;
        for (int64_t h = 0; h < nh; ++h) n_chunks += (rows[h + 1] - rows[h] + csz - 1) / csz;
        ctx->n_dhub = nh;
        ctx->n_dchunks = n_chunks;
        ctx->hub_edges = std::max<int64_t>(rows[nh] - rows[0], 1);
        int64_t* off = nullptr;
        if ((n_chunks > 0 &&
             (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dchunks), sizeof(HubChunk) * n_chunks, s))) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->htab), 2 * sizeof(unsigned long long) * ctx->hub_edges,
                           s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dacc), sizeof(HubAcc) * nh, s)) ||
            (e = cudaMallocAsync(reinterpret_cast<void**>(&off), sizeof(int64_t) * nh, s)))
            return cuda_error(ctx, e, "alloc hub tables");
        k_hub_chunks<<<1, 1024, 0, s>>>(ctx->dprp + begin[kDHub], nh, csz, off, ctx->dchunks);
        cudaFreeAsync(off, s);
        if (pack_from_csr && n_chunks > 0) {
            // hub rows are copied chunk by chunk, like the rounds read them
            const int64_t edges = m - ctx->dedge_begin[kDHub];
            Launch L(site_p, s, nh, edges, 16.0 * edges);
            k_dense_pack_chunks<<<static_cast<unsigned>(n_chunks), 256, 0, s>>>(
                ctx->dchunks, ctx->dvert, begin[kDHub], ctx->dprp, ctx->row_ptr, ctx->col, ctx->elab, ctx->dpe);
        }
    }
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "build dense layout");
    ctx->dense_ready = true;
    ++ctx->layout_version;
    ctx->stats.device_bytes = ctx->device_bytes;
    return BISIM_OK;
}

// Executable round graphs are destroyed on a thread of their own: the call
// waits for copies in flight on other streams (a 1.2 GB upload of another
// context held it for the upload's whole length), and neither the context
// that drops its graph nor its caller has a reason to wait for them. The
// state is never freed, so the idle thread outlives nothing it uses; at
// process exit a handler waits (at most ten seconds) until the queue is
// empty, so that no destroy runs while the CUDA runtime shuts down.
struct GraphReaper {
    std::mutex mu;
    std::condition_variable cv;       // work queued
    std::condition_variable idle;     // queue empty and no destroy running
    std::vector<std::pair<int, cudaGraphExec_t>> queue;
    bool started = false;
    bool busy = false;
};

GraphReaper& graph_reaper() {
    static GraphReaper* r = new GraphReaper();
    return *r;
}

void reap_graphs() {
    GraphReaper& R = graph_reaper();
    for (;;) {
        std::pair<int, cudaGraphExec_t> job;
        {
            std::unique_lock<std::mutex> lk(R.mu);
            R.cv.wait(lk, [&] { return !R.queue.empty(); });
            job = R.queue.back();
            R.queue.pop_back();
            R.busy = true;
        }
        cudaSetDevice(job.first);
        cudaGraphExecDestroy(job.second);
        {
            std::lock_guard<std::mutex> lk(R.mu);
            R.busy = false;
        }
        R.idle.notify_all();
    }
}

void drain_graph_reaper() {
    GraphReaper& R = graph_reaper();
    std::unique_lock<std::mutex> lk(R.mu);
    R.idle.wait_for(lk, std::chrono::seconds(10), [&] { return R.queue.empty() && !R.busy; });
}

void drop_round_graph(bisim_ctx* ctx) {
    if (ctx->round_graph == nullptr) return;
    GraphReaper& R = graph_reaper();
    {
        std::lock_guard<std::mutex> lk(R.mu);
        if (!R.started) {
            std::thread(reap_graphs).detach();
            std::atexit(drain_graph_reaper);
            R.started = true;
        }
        R.queue.push_back({ctx->device, static_cast<cudaGraphExec_t>(ctx->round_graph)});
    }
    R.cv.notify_one();
    ctx->round_graph = nullptr;
}

bisim_status dense_prepare(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->dense_ready) return BISIM_OK;
    drop_round_graph(ctx);                     // captured for the previous layout
    bisim_status st;
    if ((st = ensure_vertex_csr(ctx, s)) != BISIM_OK) return st;
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    cudaError_t e;
    if (m > ctx->dpe_cap || ctx->dpe == nullptr) {
        ctx_free(ctx, ctx->dpe, sizeof(unsigned long long) * ctx->dpe_cap, s);
        ctx->dpe = nullptr;
        const int64_t cap = std::max<int64_t>(m, 1);
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dpe), sizeof(unsigned long long) * cap, s))) return cuda_error(ctx, e, "alloc packed rows");
        ctx->dpe_cap = cap;
    }
    int32_t* deg = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&deg), sizeof(int32_t) * std::max(n, 1), s))) return cuda_error(ctx, e, "alloc degrees");
    if (n > 0) k_deg_from_rows<<<grid_for(n, 256), 256, 0, s>>>(ctx->row_ptr, n, deg);
    st = dense_layout_positions(ctx, deg, s);
    cudaFreeAsync(deg, s);
    if (st != BISIM_OK) return st;
    pack_rows_from_csr(ctx, s);
    return dense_layout_hubs(ctx, true, s);
}

bisim_status dense_region_table(bisim_ctx* ctx, const int64_t* voff_host, int32_t n_graphs, cudaStream_t s) {
    std::vector<int64_t> base(n_graphs);
    std::vector<uint32_t> mask(n_graphs);
    uint64_t total = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const int64_t ng = voff_host[g + 1] - voff_host[g];
        uint64_t sz = 64;
        while (static_cast<double>(sz) * 0.6 < static_cast<double>(ng)) sz <<= 1;
        base[g] = static_cast<int64_t>(total);
        mask[g] = static_cast<uint32_t>(sz - 1);
        total += sz;
    }
    if (total >= (uint64_t{1} << 32)) return BISIM_OK;     // slot indices are 32-bit: keep the global table
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->rtable), sizeof(Slot) * total, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->rbase), sizeof(int64_t) * n_graphs, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->rmask), sizeof(uint32_t) * n_graphs, s)))
        return cuda_error(ctx, e, "alloc table regions");
    ctx->n_rslots = total;
    cudaMemcpyAsync(ctx->rbase, base.data(), sizeof(int64_t) * n_graphs, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(ctx->rmask, mask.data(), sizeof(uint32_t) * n_graphs, cudaMemcpyHostToDevice, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "upload table regions");
    return BISIM_OK;
}

bisim_status ensure_vertex_csr(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->csr_stale) return csr_from_store(ctx, s);     // batches edited the row store
    if (ctx->row_ptr != nullptr) return BISIM_OK;
    if (!ctx->dense_ready) return set_error(ctx, BISIM_ESTATE, "no graph layout to rebuild the CSR from");
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->row_ptr), sizeof(int64_t) * (n + 1), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->col), sizeof(int32_t) * std::max<int64_t>(m, 1), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->elab), sizeof(int32_t) * std::max<int64_t>(m, 1), s)))
        return cuda_error(ctx, e, "alloc vertex-ordered CSR");
    const size_t tmp_words = scan_temp_words(static_cast<int64_t>(n) + 1);
    int64_t* scratch = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(int64_t) * (n + 1 + tmp_words), s)))
        return cuda_error(ctx, e, "alloc CSR scratch");
    const int64_t n_live = ctx->dbegin[kDClasses];
    BISIM_SITE(site, "csr_from_layout");
    {
        Launch L(site, s, n, 0, 24.0 * n);
        k_vertex_degrees<<<grid_for(n + 1, 256), 256, 0, s>>>(ctx->dvpos, n, n_live, ctx->dprp, scratch);
    }
    exclusive_scan_i64(scratch, ctx->row_ptr, n + 1, scratch + n + 1, s);
    {
        Launch L(site, s, n, m, 16.0 * m);
        if (n > 0)
            k_unpack_rows<<<grid_for(n, 256), 256, 0, s>>>(ctx->dvpos, n, n_live, ctx->dprp, ctx->dpe, ctx->row_ptr,
                                                          ctx->col, ctx->elab);
        const int64_t mid = ctx->dbegin[kDHub] - ctx->dbegin[kDMid0];
        if (mid > 0)
            k_unpack_big<<<static_cast<unsigned>(mid), 256, 0, s>>>(ctx->dvert, ctx->dbegin[kDMid0], ctx->dprp, ctx->dpe,
                                                                   ctx->row_ptr, ctx->col, ctx->elab);
        if (ctx->n_dchunks > 0)
            k_unpack_chunks<<<static_cast<unsigned>(ctx->n_dchunks), 256, 0, s>>>(
                ctx->dchunks, ctx->dvert, ctx->dbegin[kDHub], ctx->dprp, ctx->dpe, ctx->row_ptr, ctx->col, ctx->elab);
    }
    cudaFreeAsync(scratch, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "rebuild vertex-ordered CSR");
    ctx->stats.device_bytes = ctx->device_bytes;
    return BISIM_OK;
}

void dense_start(bisim_ctx* ctx, cudaStream_t s) {
    // P_0's block sizes are not known: every live position is listed, and no
    // hub counts as alone in the first round
    if (ctx->n > 0) cudaMemsetAsync(ctx->djoined, 1, static_cast<size_t>(ctx->n), s);
    const int64_t n_live = ctx->dbegin[kDClasses];
    BISIM_SITE(site, "active_init");
    Launch L(site, s, n_live, 0, 4.0 * n_live);
    k_active_init<<<static_cast<unsigned>(std::min<int64_t>(kPersistGrid, cdiv(std::max<int64_t>(n_live, kDClasses + 1),
                                                                                kThreads))),
                    kThreads, 0, s>>>(ctx->dact, n_live, ctx->daoff, class_counts(ctx), class_bounds(ctx));
    dense_mark_dead(ctx, s);
}

void dense_mark_dead(bisim_ctx* ctx, cudaStream_t s) {
    const int64_t n_live = ctx->dbegin[kDClasses];
    if (n_live >= ctx->n) return;
    BISIM_SITE(site, "dense_dead");
    Launch L(site, s, ctx->n - n_live, 0, 12.0 * (ctx->n - n_live));
    k_dense_dead<<<grid_for(ctx->n - n_live, 256), 256, 0, s>>>(ctx->dvert, n_live, ctx->n, ctx->P[0], ctx->P[1]);
}

bisim_status dense_keep_graphs(bisim_ctx* ctx, cudaStream_t s, const uint8_t* keep_graph, int64_t* prev,
                               int64_t* dropped) {
    const int64_t n_live = ctx->dbegin[kDClasses];
    if (n_live <= 0 || ctx->gid == nullptr) return BISIM_OK;
    cudaMemsetAsync(ctx->dstate, 0, sizeof(DevState), s);
    BISIM_SITE(site, "active_init");
    {
        Launch L(site, s, n_live, 0, 13.0 * n_live);
        k_keep_graphs<<<static_cast<unsigned>(std::min<int64_t>(kPersistGrid, cdiv(n_live, kThreads))), kThreads, 0,
                        s>>>(ctx->dvert, ctx->gid, keep_graph, ctx->P0, n_live, ctx->downs, ctx->djoined, ctx->dstate);
    }
    // the list keeps the other positions; both partition buffers hold P_0 there
    launch_round_end(ctx, s, dense_view(ctx), nullptr, ctx->P[0]);
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "list the kept graphs");
    *dropped = static_cast<int64_t>(ctx->hstate->blocks);
    *prev = *prev - static_cast<int64_t>(ctx->hstate->aux) + *dropped;
    return BISIM_OK;
}

bisim_status dense_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks) {
    set_attributes();
    const TableRef t = level_table(ctx, s);
    launch_round(ctx, s, t);
    return finish_round(ctx, s, out_blocks);
}

bisim_status dense_finish_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks) {
    return finish_round(ctx, s, out_blocks);
}

namespace {

// The table of the captured rounds. Its epoch field is only a placeholder: the
// insert takes round r's epoch (r % 15 + 1) from the loop state, and the table
// is blanked whenever that epoch starts a new cycle (k_table_clear_round).
TableRef fixed_table(const bisim_ctx* ctx) {
    TableRef t;
    t.slots = round_slots(ctx);
    t.mask = ctx->rtable ? ctx->n_rslots - 1 : ctx->nslots - 1;
    t.epoch = uint64_t{1} << 32;
    const int hb = ctx->opt.hash_bits;
    t.hmask = hb >= 64 ? ~0ull : ((1ull << hb) - 1ull);
    return t;
}

// The round loop as one graph: a while node whose body is one round (table
// clear when the epoch cycle restarts, signatures and level 0 of the
// renumbering over the active list), the loop check, and the end of the round
// (P_{i+1} of the listed vertices copied into the input buffer, the list
// compacted). The body reads P[0] and writes P[1].
bisim_status build_round_graph(bisim_ctx* ctx) {
    set_attributes();
    cudaError_t e;
    if (ctx->capture_stream == nullptr &&
        (e = cudaStreamCreateWithFlags(reinterpret_cast<cudaStream_t*>(&ctx->capture_stream), cudaStreamNonBlocking)))
        return cuda_error(ctx, e, "create capture stream");
    if (ctx->dloop == nullptr) {
        if ((e = ctx_alloc(ctx, &ctx->dloop, sizeof(LoopState), nullptr))) return cuda_error(ctx, e, "alloc loop state");
        static_assert(sizeof(LoopState) <= 256, "pinned blocks hold 256 bytes");
        if ((ctx->hloop = pinned_take()) == nullptr) return set_error(ctx, BISIM_ENOMEM, "pinned loop state mirror");
    }
    cudaStream_t cs = static_cast<cudaStream_t>(ctx->capture_stream);
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0))) return cuda_error(ctx, e, "create round graph");
    cudaGraphConditionalHandle cond;
    // the node parameters are a union without a default constructor: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
    std::memset(pbuf, 0, sizeof(pbuf));
    cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(pbuf);
    cudaGraphNode_t node;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault))) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "create loop condition");
    }
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p))) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "add loop node");
    }
    cudaGraph_t body = p.conditional.phGraph_out[0];
    const int cur = ctx->cur;
    ctx->cur = 0;
    const int64_t before = bisim_launch_count();
    BISIM_SITE(site_ck, "round_check");
    BISIM_SITE(site_tc, "table_clear");
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal))) {
        ctx->cur = cur;
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "capture round");
    }
    LoopState* L = static_cast<LoopState*>(ctx->dloop);
    {
        const uint64_t ns = ctx->rtable ? ctx->n_rslots : ctx->nslots;     // a power of two >= 64
        Launch Lk(site_tc, cs, 0, 0, 0.0);
        k_table_clear_round<<<persistent_grid(k_table_clear_round, kThreads, 0,
                                              static_cast<int64_t>((ns / 2 + kThreads - 1) / kThreads)),
                              kThreads, 0, cs>>>(L, round_slots(ctx), ns);
    }
    launch_round(ctx, cs, fixed_table(ctx), &L->executed);
    {
        Launch Lk(site_ck, cs, 0, 0, 0.0);
        k_round_check<<<1, 1, 0, cs>>>(ctx->dstate, L, cond);
    }
    launch_round_end(ctx, cs, dense_view(ctx), &L->stop);
    e = cudaStreamEndCapture(cs, &body);
    ctx->cur = cur;
    ctx->round_graph_launches = bisim_launch_count() - before;
    prof_add_launches(-ctx->round_graph_launches);      // counted when the rounds run
    if (e == cudaSuccess) {
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        ctx->round_graph = exec;
    }
    cudaGraphDestroy(g);
    if (e) {
        ctx->round_graph = nullptr;
        return cuda_error(ctx, e, "instantiate round graph");
    }
    return BISIM_OK;
}

}  // namespace

bool dense_graph_usable(const bisim_ctx* ctx) {
    return ctx->dense_ready && ctx->n > 0 && !prof_enabled() &&
           !(ctx->opt.flags & (BISIM_FLAG_EAGER | BISIM_FLAG_L2_PIN));
}

bisim_status dense_graph_rounds(bisim_ctx* ctx, cudaStream_t s, int32_t limit, bool fixpoint, int64_t prev_blocks,
                                GraphRounds* out) {
    bisim_status st;
    if (ctx->round_graph == nullptr && (st = build_round_graph(ctx)) != BISIM_OK) return st;
    LoopState* h = static_cast<LoopState*>(ctx->hloop);
    std::memset(h, 0, sizeof(*h));
    h->prev_blocks = static_cast<unsigned long long>(prev_blocks);
    h->limit = limit;
    h->fixpoint = fixpoint ? 1 : 0;
    h->rounds = limit;
    cudaError_t e;
    cudaMemcpyAsync(ctx->dloop, h, sizeof(LoopState), cudaMemcpyHostToDevice, s);
    if ((e = cudaGraphLaunch(static_cast<cudaGraphExec_t>(ctx->round_graph), s))) return cuda_error(ctx, e, "launch round graph");
    cudaMemcpyAsync(h, ctx->dloop, sizeof(LoopState), cudaMemcpyDeviceToHost, s);
    // the loop's slots carry epochs of its own: the next host-driven level of
    // the global table (next_epoch) must start from a blank table
    ctx->epoch32 = kEpochCycle;
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "round graph");
    prof_add_launches(ctx->round_graph_launches * h->executed);
    out->executed = h->executed;
    out->rounds = h->rounds;
    out->blocks = static_cast<int64_t>(h->blocks);
    out->stop = h->stop;
    return BISIM_OK;
}

void dense_release(bisim_ctx* ctx) {
    drop_round_graph(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->capture_stream));
    pinned_give(ctx->hloop);
    ctx->round_graph = nullptr;
    ctx->capture_stream = nullptr;
    ctx->hloop = nullptr;
}

}  // namespace bisim
